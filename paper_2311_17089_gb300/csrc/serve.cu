// Render server: resident scenes, memory admission from one device arena,
// continuous batching of requests over a pool of CUDA streams.
//
// One scheduler thread owns the queue.  It admits the request at the head
// of the FIFO when fewer than max_inflight requests are on the device and
// the request's buffers fit in the arena (first fit over a free list of
// offset ranges), together with later queued requests of the same scene
// and mode whose buffers fit too (up to max_batch_views); while requests
// are in flight, a head with such company waits until enough slots are
// free for them all.  The batch's
// cameras are projected in one ms_project_views pass on the first
// request's stream; every request then waits for that pass on its own
// stream and enqueues ms_bin -> ms_raster plus the copies of the duplicate
// counts (and, if asked, of the image), ending its stream's work with a
// host function that hands the request back.  Host functions run in stream order after the request's
// kernels, so the arena range is free for reuse by then.  A completed
// request that overflowed its duplicate capacity goes back to the head of
// the queue with the exact count.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "arena.h"
#include "common.cuh"
#include "raster_ws.cuh"

namespace msgs {

namespace {

constexpr size_t kAlign = 256;
inline size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

double now_s() {
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

struct Layout {  // byte offsets of one request's buffers inside its range
    size_t rec, rect, n_tiles, depth, stats, gidx, ranges, counts, bin_ws, bin_ws_bytes, rws,
        rws_bytes, image, total;
};

bool request_layout(int64_t n, int64_t tiles, int64_t cap, int64_t pixels, bool own_image,
                    Layout &L) {
    const size_t bws = ms_bin_workspace_bytes(n, tiles, cap);
    const size_t rws = ms_raster_workspace_bytes(tiles, cap);
    if (!bws || !rws) return false;
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    size_t o = 0;
    L.rec = o;
    o = up(o + nn * 48);
    L.rect = o;
    o = up(o + nn * 8);
    L.n_tiles = o;
    o = up(o + nn * 4);
    L.depth = o;
    o = up(o + nn * 4);
    L.stats = o;
    o = up(o + MS_STATS_WORDS * 4);
    L.gidx = o;
    o = up(o + (size_t)cap * 4);
    L.ranges = o;
    o = up(o + (size_t)tiles * 8);
    L.counts = o;
    o = up(o + 4 * 8);
    L.bin_ws = o;
    L.bin_ws_bytes = bws;
    o = up(o + bws);
    L.rws = o;
    L.rws_bytes = rws;
    o = up(o + rws);
    L.image = o;
    if (own_image) o = up(o + (size_t)pixels * 12);
    L.total = o;
    return true;
}

}  // namespace

struct RequestKey {
    int32_t scene, mode, tiles;
    bool operator<(const RequestKey &o) const {
        if (scene != o.scene) return scene < o.scene;
        if (mode != o.mode) return mode < o.mode;
        return tiles < o.tiles;
    }
};

struct Request {
    ms_server *srv = nullptr;
    bool timed = false;  // first request of its batch: owns the pass's timing events
    uint64_t ticket = 0;
    ms_request_t r{};
    int32_t status = MS_PENDING;
    int32_t retries = 0;
    int64_t cap = 0, dups = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    size_t off = 0, bytes = 0;
    int slot = -1;  // index of its pinned counts row while on the device
    bool done = false;
};

}  // namespace msgs

struct ms_server {
    ms_serve_cfg_t cfg{};
    std::vector<cudaStream_t> streams;
    char *arena_base = nullptr;
    msgs::Arena arena;
    uint64_t *pinned_counts = nullptr;  // [max_inflight][4]
    std::vector<cudaEvent_t> proj_done;  // per slot: the batch's projection pass is done
    std::vector<cudaEvent_t> proj_t0, proj_t1;  // per slot: timing of the pass
    std::vector<int> free_slots;
    std::vector<ms_scene_t> scenes;
    std::map<msgs::RequestKey, int64_t> dup_hist;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<msgs::Request *> queue;
    std::vector<msgs::Request *> finished_gpu;  // handed back by host functions
    std::unordered_map<uint64_t, msgs::Request *> reqs;
    uint64_t next_ticket = 1;
    int inflight = 0, peak_inflight = 0, next_stream = 0;
    int64_t submitted = 0, completed = 0, failed = 0, retries = 0, renders = 0;
    int64_t proj_passes = 0;
    double issue_s = 0, proj_s = 0;
    bool stop = false;
    int max_batch = 1;  // requests per projection pass
    std::thread sched;
};

namespace msgs {
namespace {

void CUDART_CB on_gpu_done(void *p) {
    Request *q = static_cast<Request *>(p);
    ms_server *s = q->srv;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->finished_gpu.push_back(q);
    }
    s->cv_sched.notify_one();
}

int64_t capacity_for(ms_server *s, const Request *q) {
    if (q->cap > 0) return q->cap;
    const int tiles = ((q->r.cam.width + 15) / 16) * ((q->r.cam.height + 15) / 16);
    auto it = s->dup_hist.find({q->r.scene, q->r.mode, tiles});
    int64_t cap;
    if (it != s->dup_hist.end()) {
        cap = it->second + it->second / 8 + 4096;
    } else if (s->cfg.initial_capacity > 0) {
        cap = s->cfg.initial_capacity;
    } else {
        cap = std::max<int64_t>(65536, 2 * s->scenes[q->r.scene].n);
    }
    return std::min<int64_t>(std::max<int64_t>(cap, 1024), (1ll << 30) - 1);
}

// The request's buffers inside its arena range.
bool request_buffers(ms_server *s, const Request *q, ms_proj_t &proj, ms_bins_t &bins,
                     float *&image, Layout &L) {
    const ms_scene_t &sc = s->scenes[q->r.scene];
    const ms_camera_t &cam = q->r.cam;
    const int64_t tiles = (int64_t)((cam.width + 15) / 16) * ((cam.height + 15) / 16);
    const int64_t pixels = (int64_t)cam.width * cam.height;
    if (!request_layout(sc.n, tiles, q->cap, pixels, q->r.image_dev == nullptr, L)) return false;
    char *b = s->arena_base + q->off;
    proj.rec = reinterpret_cast<float *>(b + L.rec);
    proj.rect = reinterpret_cast<uint32_t *>(b + L.rect);
    proj.n_tiles = reinterpret_cast<uint32_t *>(b + L.n_tiles);
    proj.depth = reinterpret_cast<uint32_t *>(b + L.depth);
    proj.cover = nullptr;
    proj.mask = nullptr;
    proj.stats = reinterpret_cast<uint32_t *>(b + L.stats);
    proj.n = std::max<int64_t>(sc.n, 1);
    bins.gauss_idx = reinterpret_cast<uint32_t *>(b + L.gidx);
    bins.ranges = reinterpret_cast<uint32_t *>(b + L.ranges);
    bins.counts = reinterpret_cast<uint64_t *>(b + L.counts);
    bins.dup_capacity = q->cap;
    image = q->r.image_dev ? q->r.image_dev : reinterpret_cast<float *>(b + L.image);
    return true;
}

// Enqueues a batch's renders (requests of one scene and mode, each with its
// stream): one projection pass for all of their cameras on the first
// request's stream, then each request's binning, blend and copies on its
// own stream after that pass.  Called without the lock.
int launch(ms_server *s, const std::vector<Request *> &batch,
           const std::vector<cudaStream_t> &st) {
    const int nb = (int)batch.size();
    const Request *q0 = batch[0];
    const ms_scene_t &sc = s->scenes[q0->r.scene];
    ms_proj_t proj[MS_MAX_PROJ_VIEWS];
    ms_bins_t bins[MS_MAX_PROJ_VIEWS];
    ms_camera_t cams[MS_MAX_PROJ_VIEWS];
    float *image[MS_MAX_PROJ_VIEWS];
    Layout L[MS_MAX_PROJ_VIEWS];
    for (int i = 0; i < nb; i++) {
        if (!request_buffers(s, batch[i], proj[i], bins[i], image[i], L[i]))
            return fail(MS_ERR_INVALID_ARG, "request sizes out of range");
        cams[i] = batch[i]->r.cam;
    }
    const int slot0 = q0->slot;
    int rc;
    if ((rc = cuda_check(cudaEventRecord(s->proj_t0[slot0], st[0]), "event record"))) return rc;
    if (nb == 1) {
        if ((rc = ms_project(&sc, &cams[0], (ms_mode_t)q0->r.mode, &proj[0], st[0]))) return rc;
    } else if ((rc = ms_project_views(&sc, cams, nb, (ms_mode_t)q0->r.mode, proj, st[0]))) {
        return rc;
    }
    if ((rc = cuda_check(cudaEventRecord(s->proj_t1[slot0], st[0]), "event record"))) return rc;
    if ((rc = cuda_check(cudaEventRecord(s->proj_done[slot0], st[0]), "event record"))) return rc;
    for (int i = 0; i < nb; i++) {
        Request *q = batch[i];
        const ms_camera_t &cam = cams[i];
        const int64_t pixels = (int64_t)cam.width * cam.height;
        char *b = s->arena_base + q->off;
        if (st[i] != st[0] &&
            (rc = cuda_check(cudaStreamWaitEvent(st[i], s->proj_done[slot0], 0), "stream wait")))
            return rc;
        if ((rc = ms_bin(&proj[i], sc.n, &cam, &bins[i], b + L[i].bin_ws, L[i].bin_ws_bytes,
                         st[i])))
            return rc;
        if ((rc = ms_raster(&proj[i], &bins[i], &cam, image[i], nullptr, nullptr, nullptr,
                            b + L[i].rws, L[i].rws_bytes, st[i])))
            return rc;
        if ((rc = cuda_check(cudaMemcpyAsync(s->pinned_counts + 4 * q->slot, bins[i].counts, 32,
                                             cudaMemcpyDeviceToHost, st[i]),
                             "counts copy")))
            return rc;
        if (q->r.image_host &&
            (rc = cuda_check(cudaMemcpyAsync(q->r.image_host, image[i], (size_t)pixels * 12,
                                             cudaMemcpyDeviceToHost, st[i]),
                             "image copy")))
            return rc;
        if ((rc = cuda_check(cudaLaunchHostFunc(st[i], on_gpu_done, q), "host function")))
            return rc;
    }
    return MS_OK;
}

size_t bytes_for(ms_server *s, const Request *q) {
    const ms_camera_t &cam = q->r.cam;
    const int64_t tiles = (int64_t)((cam.width + 15) / 16) * ((cam.height + 15) / 16);
    Layout L;
    if (!request_layout(s->scenes[q->r.scene].n, tiles, q->cap, (int64_t)cam.width * cam.height,
                        q->r.image_dev == nullptr, L))
        return 0;
    return L.total;
}

void finish(ms_server *s, Request *q, int status) {  // with the lock held
    q->status = status;
    q->t_done = now_s();
    q->done = true;
    if (status == MS_OK) s->completed++;
    else s->failed++;
}

// Takes back requests whose GPU work ended; with the lock held.
void reap(ms_server *s) {
    std::vector<Request *> fin;
    fin.swap(s->finished_gpu);
    for (Request *q : fin) {
        if (q->timed) {
            // the first request's stream ran the pass before this request's
            // work, so both events have completed
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, s->proj_t0[q->slot], s->proj_t1[q->slot]) == cudaSuccess)
                s->proj_s += 1e-3 * ms;
            q->timed = false;
        }
        const uint64_t *h = s->pinned_counts + 4 * q->slot;
        const int64_t d = (int64_t)h[kCntDup];
        const uint64_t status = h[kCntStatus];
        s->arena.release(q->off, q->bytes);
        s->free_slots.push_back(q->slot);
        q->slot = -1;
        s->inflight--;
        q->dups = d;
        const int tiles = ((q->r.cam.width + 15) / 16) * ((q->r.cam.height + 15) / 16);
        int64_t &hist = s->dup_hist[{q->r.scene, q->r.mode, tiles}];
        hist = std::max(hist, d);
        if (status & kStatusTimeout) {
            finish(s, q, MS_ERR_TIMEOUT);
        } else if ((status & kStatusOverflow) || d > q->cap) {
            q->retries++;
            s->retries++;
            q->cap = d + d / 16 + 1024;
            s->queue.push_front(q);
        } else {
            finish(s, q, MS_OK);
        }
    }
    if (!fin.empty()) s->cv_done.notify_all();
}

void scheduler(ms_server *s) {
    cudaSetDevice(s->cfg.device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        reap(s);
        if (s->stop && s->inflight == 0) break;
        bool progressed = false;
        while (!s->stop && !s->queue.empty() && s->inflight < s->cfg.max_inflight) {
            Request *q = s->queue.front();
            q->cap = capacity_for(s, q);
            q->bytes = bytes_for(s, q);
            size_t off = 0;
            if (q->bytes == 0 || q->bytes > s->arena.size()) {
                s->queue.pop_front();
                finish(s, q, MS_ERR_OOM);  // can never fit
                s->cv_done.notify_all();
                progressed = true;
                continue;
            }
            if (s->max_batch > 1 && s->inflight > 0) {
                // when several queued requests share the head's scene and
                // mode, wait (the GPU busy with the requests in flight) until
                // enough slots are free to project them in one pass
                int want = 1;
                int scanned = 0;
                for (auto it = std::next(s->queue.begin());
                     it != s->queue.end() && want < s->max_batch && scanned < 64; ++it, ++scanned)
                    if ((*it)->r.scene == q->r.scene && (*it)->r.mode == q->r.mode) want++;
                if (s->cfg.max_inflight - s->inflight < want) break;
            }
            if (!s->arena.alloc(q->bytes, off)) break;  // wait for memory
            s->queue.pop_front();
            q->off = off;
            // later queued requests of the same scene and mode whose buffers
            // fit now join the head's projection pass (FIFO order among them)
            std::vector<Request *> batch{q};
            const int maxb = std::min(s->max_batch, s->cfg.max_inflight - s->inflight);
            for (auto it = s->queue.begin(); it != s->queue.end() && (int)batch.size() < maxb;) {
                Request *r = *it;
                if (r->r.scene != q->r.scene || r->r.mode != q->r.mode) {
                    ++it;
                    continue;
                }
                r->cap = capacity_for(s, r);
                r->bytes = bytes_for(s, r);
                size_t roff = 0;
                if (r->bytes == 0 || r->bytes > s->arena.size() || !s->arena.alloc(r->bytes, roff)) {
                    ++it;
                    continue;
                }
                r->off = roff;
                it = s->queue.erase(it);
                batch.push_back(r);
            }
            std::vector<cudaStream_t> sts;
            for (Request *r : batch) {
                r->slot = s->free_slots.back();
                s->free_slots.pop_back();
                s->inflight++;
                if (r->t_start == 0) r->t_start = now_s();
                sts.push_back(s->streams[s->next_stream]);
                s->next_stream = (s->next_stream + 1) % (int)s->streams.size();
            }
            s->peak_inflight = std::max(s->peak_inflight, s->inflight);
            batch[0]->timed = true;
            lk.unlock();
            const double t_issue = now_s();
            const int rc = launch(s, batch, sts);
            const double t_issued = now_s();
            lk.lock();
            s->renders += (int64_t)batch.size();
            s->proj_passes++;
            s->issue_s += t_issued - t_issue;
            if (rc != MS_OK) {
                // whatever was enqueued before the failure may still run:
                // keep the ranges until the streams have drained
                lk.unlock();
                for (cudaStream_t st : sts) cudaStreamSynchronize(st);
                lk.lock();
                for (Request *r : batch) {
                    s->arena.release(r->off, r->bytes);
                    s->free_slots.push_back(r->slot);
                    r->slot = -1;
                    r->timed = false;
                    s->inflight--;
                    finish(s, r, rc);
                }
                // host functions of requests enqueued before the failure
                // must not hand them back a second time
                s->finished_gpu.erase(
                    std::remove_if(s->finished_gpu.begin(), s->finished_gpu.end(),
                                   [&batch](Request *r) {
                                       return std::find(batch.begin(), batch.end(), r) !=
                                              batch.end();
                                   }),
                    s->finished_gpu.end());
                s->cv_done.notify_all();
            }
            progressed = true;
        }
        if (progressed) continue;
        s->cv_sched.wait(lk, [s] {
            return !s->finished_gpu.empty() ||
                   (s->stop && s->inflight == 0) ||
                   (!s->stop && !s->queue.empty() && s->inflight < s->cfg.max_inflight &&
                    s->queue.front()->cap == 0);
        });
    }
}

void fill(const Request *q, ms_result_t *res) {
    res->status = q->done ? q->status : MS_PENDING;
    res->retries = q->retries;
    res->duplicates = q->dups;
    res->capacity = q->cap;
    res->bytes = q->bytes;
    res->t_submit = q->t_submit;
    res->t_start = q->t_start;
    res->t_done = q->t_done;
}

}  // namespace
}  // namespace msgs

using namespace msgs;

extern "C" double ms_serve_clock(void) { return now_s(); }

extern "C" int ms_serve_create(const ms_serve_cfg_t *cfg, ms_server_t **out) {
    if (!out) return fail(MS_ERR_INVALID_ARG, "NULL out");
    *out = nullptr;
    if (!cfg) return fail(MS_ERR_INVALID_ARG, "NULL cfg");
    // the binning sorts up to 2^30 - 1 items per pass
    if (cfg->max_gaussians < 1 || cfg->max_gaussians > (1ll << 30) - 1)
        return fail(MS_ERR_INVALID_ARG, "max_gaussians must be 1..2^30-1");
    if (cfg->max_width < 1 || cfg->max_height < 1 || cfg->max_width > 32768 ||
        cfg->max_height > 32768)
        return fail(MS_ERR_INVALID_ARG, "max image size must be 1..32768");
    if (cfg->max_inflight < 1 || cfg->max_inflight > 1024)
        return fail(MS_ERR_INVALID_ARG, "max_inflight must be 1..1024");
    if (cfg->n_streams < 1 || cfg->n_streams > cfg->max_inflight)
        return fail(MS_ERR_INVALID_ARG, "n_streams must be 1..max_inflight");
    if (cfg->mem_budget_bytes < (1u << 20))
        return fail(MS_ERR_INVALID_ARG, "mem_budget_bytes must be at least 1 MiB");
    if (cfg->initial_capacity < 0 || cfg->initial_capacity > (1ll << 30) - 1)
        return fail(MS_ERR_INVALID_ARG, "initial_capacity must be 0..2^30-1");
    if (cfg->max_batch_views < 0 || cfg->max_batch_views > MS_MAX_PROJ_VIEWS)
        return fail(MS_ERR_INVALID_ARG, "max_batch_views must be 0..MS_MAX_PROJ_VIEWS");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev)
        return fail(MS_ERR_NO_DEVICE, "no such CUDA device");
    int rc;
    if ((rc = cuda_check(cudaSetDevice(cfg->device), "set device"))) return rc;
    ms_server *s = new ms_server();
    s->cfg = *cfg;
    s->max_batch = cfg->max_batch_views > 0 ? cfg->max_batch_views : MS_MAX_PROJ_VIEWS;
    auto cleanup = [s](int code) {
        for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
        for (auto *v : {&s->proj_done, &s->proj_t0, &s->proj_t1})
            for (cudaEvent_t e : *v) cudaEventDestroy(e);
        if (s->arena_base) cudaFree(s->arena_base);
        if (s->pinned_counts) cudaFreeHost(s->pinned_counts);
        delete s;
        return code;
    };
    const size_t arena = cfg->mem_budget_bytes & ~(kAlign - 1);
    if (cudaMalloc(&s->arena_base, arena) != cudaSuccess) {
        cudaGetLastError();
        s->arena_base = nullptr;
        return cleanup(fail(MS_ERR_OOM, "arena allocation of mem_budget_bytes failed"));
    }
    s->arena.init(arena);
    if ((rc = cuda_check(cudaMallocHost(&s->pinned_counts, (size_t)cfg->max_inflight * 32),
                         "pinned counts")))
        return cleanup(rc);
    for (int i = 0; i < cfg->max_inflight; i++) {
        s->free_slots.push_back(cfg->max_inflight - 1 - i);
        cudaEvent_t e0, e1, e2;
        if ((rc = cuda_check(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming), "event"))) 
            return cleanup(rc);
        s->proj_done.push_back(e0);
        if ((rc = cuda_check(cudaEventCreate(&e1), "event"))) return cleanup(rc);
        s->proj_t0.push_back(e1);
        if ((rc = cuda_check(cudaEventCreate(&e2), "event"))) return cleanup(rc);
        s->proj_t1.push_back(e2);
    }
    for (int i = 0; i < cfg->n_streams; i++) {
        cudaStream_t st;
        if ((rc = cuda_check(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream")))
            return cleanup(rc);
        s->streams.push_back(st);
    }
    s->sched = std::thread(scheduler, s);
    *out = s;
    return MS_OK;
}

extern "C" int ms_serve_add_scene(ms_server_t *s, const ms_scene_t *scene, int32_t *scene_id) {
    if (!s || !scene || !scene_id) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    if (scene->n < 0 || scene->n > s->cfg.max_gaussians)
        return fail(MS_ERR_INVALID_ARG, "scene larger than max_gaussians");
    int rc;
    if ((rc = cuda_check(cudaSetDevice(s->cfg.device), "set device"))) return rc;
    cudaStream_t st = s->streams[0];
    if ((rc = ms_scene_prepare(scene, st))) return rc;
    if ((rc = cuda_check(cudaStreamSynchronize(st), "scene prepare"))) return rc;
    std::lock_guard<std::mutex> lk(s->mu);
    s->scenes.push_back(*scene);
    *scene_id = (int32_t)s->scenes.size() - 1;
    return MS_OK;
}

extern "C" int ms_serve_submit(ms_server_t *s, const ms_request_t *req, uint64_t *ticket) {
    if (!s || !req || !ticket) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    const ms_camera_t &c = req->cam;
    if (c.width < 1 || c.height < 1 || c.width > s->cfg.max_width || c.height > s->cfg.max_height)
        return fail(MS_ERR_INVALID_ARG, "request image larger than the configured maximum");
    if (req->mode < MS_SELECTIVE || req->mode > MS_FILTER_SMALL)
        return fail(MS_ERR_INVALID_ARG, "unknown mode");
    if (req->image_dev && !aligned(req->image_dev, 16))
        return fail(MS_ERR_INVALID_ARG, "image_dev must be 16-byte aligned");
    Request *q = new Request();
    q->srv = s;
    q->r = *req;
    q->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (req->scene < 0 || req->scene >= (int32_t)s->scenes.size()) {
            delete q;
            return fail(MS_ERR_INVALID_ARG, "unknown scene id");
        }
        if (s->stop) {
            delete q;
            return fail(MS_ERR_INVALID_ARG, "server is shutting down");
        }
        q->ticket = s->next_ticket++;
        s->reqs[q->ticket] = q;
        s->queue.push_back(q);
        s->submitted++;
        *ticket = q->ticket;
    }
    s->cv_sched.notify_one();
    return MS_OK;
}

extern "C" int ms_serve_poll(ms_server_t *s, uint64_t ticket, ms_result_t *res) {
    return ms_serve_wait(s, ticket, 0.0, res);
}

extern "C" int ms_serve_wait(ms_server_t *s, uint64_t ticket, double timeout_s,
                             ms_result_t *res) {
    if (!s || !res) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(MS_ERR_INVALID_ARG, "unknown ticket");
    Request *q = it->second;
    if (!q->done && timeout_s > 0)
        s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [q] { return q->done; });
    fill(q, res);
    if (q->done) {
        s->reqs.erase(it);
        delete q;
    }
    return MS_OK;
}

extern "C" int ms_serve_stats(ms_server_t *s, ms_serve_stats_t *st) {
    if (!s || !st) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->failed = s->failed;
    st->retries = s->retries;
    st->queued = (int32_t)s->queue.size();
    st->inflight = s->inflight;
    st->peak_inflight = s->peak_inflight;
    st->scenes = (int32_t)s->scenes.size();
    st->arena_bytes = s->arena.size();
    st->arena_used = s->arena.used();
    st->arena_peak = s->arena.peak();
    st->renders = s->renders;
    st->issue_seconds = s->issue_s;
    st->proj_passes = s->proj_passes;
    st->proj_seconds = s->proj_s;
    return MS_OK;
}

extern "C" int ms_serve_destroy(ms_server_t *s) {
    if (!s) return MS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Request *q : s->queue) finish(s, q, MS_ERR_INVALID_ARG);
        s->queue.clear();
    }
    s->cv_sched.notify_all();
    if (s->sched.joinable()) s->sched.join();
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto &kv : s->reqs) delete kv.second;
    for (auto *v : {&s->proj_done, &s->proj_t0, &s->proj_t1})
        for (cudaEvent_t e : *v) cudaEventDestroy(e);
    if (s->arena_base) cudaFree(s->arena_base);
    if (s->pinned_counts) cudaFreeHost(s->pinned_counts);
    delete s;
    return MS_OK;
}

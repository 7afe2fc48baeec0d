// Front-to-back blending per 16x16 tile (Sec. 3.1; Eq. 3 with incremental
// transmittance T_k): one 256-thread CTA walks a chunk of a tile's sorted
// list, one thread per pixel.
//
// Long lists (low resolutions put thousands of splats on one tile; Sec. 3.2,
// item 2) are cut into chunks of kChunk records that different CTAs blend
// concurrently.  The blend stays exactly sequential:
//   - a chunk whose predecessor has already finished starts from the
//     predecessor's per-pixel (C, T) and applies the termination rule
//     directly;
//   - otherwise it blends from T = 1 into local (C_l, T_l), then waits for
//     the predecessor's (C_in, T_in).  If no termination can fall inside the
//     chunk (T_in T_l >= 1e-4, T being monotone) the result is
//     C_in + T_in C_l, T_in T_l; otherwise the chunk is re-walked from
//     shared memory starting at T_in, which finds the exact stopping point.
// Records reach shared memory by per-record bulk copies (cp.async.bulk)
// completing on an mbarrier; each persistent CTA prefetches its next chunk
// into the second buffer while it blends the current one.  Every wait is
// bounded; a wait that gives up sets a status bit and the CTA carries on.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace msgs {

constexpr int kRasterThreads = 256;
constexpr int kChunk = 512;                  // records per chunk
constexpr int kRecBytes = 48;                // one raster record
constexpr int kBufBytes = kChunk * kRecBytes;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTStop = 1e-4f;
constexpr uint32_t kTermBit = 0x80000000u;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

struct RasterArgs {
    const uint32_t *ranges;
    const uint32_t *gidx;
    const float4 *rec;
    uint32_t n_rec;
    int W, H, tiles_x, tiles;
    float bg0, bg1, bg2;
    float *image;
    float *final_t;
    uint32_t *n_contrib;
    uint32_t *n_eval;
    uint32_t *chunk_off;  // [tiles + 1]
    uint32_t *ticket;
    uint32_t *flags;      // [max_chunks]
    float4 *state;        // [max_chunks][256] (C0, C1, C2, T)
    uint2 *state2;        // [max_chunks][256] (n_contrib, n_eval | term bit)
    unsigned long long *err;
};

struct Chunk {
    uint32_t t, k, nk, start, cnt;
};

__device__ __forceinline__ Chunk chunk_of(const RasterArgs &a, uint32_t c) {
    int lo = 0, hi = a.tiles;  // chunk_off[lo] <= c < chunk_off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (a.chunk_off[mid] <= c) lo = mid;
        else hi = mid;
    }
    Chunk ch;
    ch.t = lo;
    ch.k = c - a.chunk_off[lo];
    ch.nk = a.chunk_off[lo + 1] - a.chunk_off[lo];
    uint32_t s = a.ranges[2 * lo], e = a.ranges[2 * lo + 1];
    ch.start = s + ch.k * kChunk;
    uint32_t stop = min(e, ch.start + kChunk);
    ch.cnt = stop > ch.start ? stop - ch.start : 0;
    return ch;
}

// Number of chunks of every tile (at least one, so empty tiles still write
// the background), exclusive-scanned by one block.
__global__ void __launch_bounds__(1024)
chunk_offsets_kernel(const uint32_t *__restrict__ ranges, int tiles, uint32_t *__restrict__ off) {
    __shared__ uint32_t s_warp[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (tiles + 1023) / 1024;
    const int t0 = tid * per;
    uint32_t sum = 0;
    for (int t = t0; t < t0 + per && t < tiles; t++) {
        uint32_t len = ranges[2 * t + 1] - ranges[2 * t];
        sum += len > 0 ? (len + kChunk - 1) / kChunk : 1u;
    }
    uint32_t x = sum;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = s_warp[lane];
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        s_warp[lane] = v;
    }
    __syncthreads();
    uint32_t run = x - sum + (warp > 0 ? s_warp[warp - 1] : 0u);
    for (int t = t0; t < t0 + per && t < tiles; t++) {
        off[t] = run;
        uint32_t len = ranges[2 * t + 1] - ranges[2 * t];
        run += len > 0 ? (len + kChunk - 1) / kChunk : 1u;
    }
    if (tid == 1023) off[tiles] = run;
}

struct PixelState {
    float C0, C1, C2, T;
    uint32_t last, evals;
    bool term;
};

// Blend records [0, cnt) of a staged chunk into s, starting from s's state.
// pos0 is the list position of record 0 of the chunk.
__device__ __forceinline__ void blend_chunk(const float4 *__restrict__ buf, uint32_t cnt,
                                            uint32_t pos0, float fx, float fy, PixelState &s) {
    for (uint32_t i = 0; i < cnt; i++) {
        const float4 r0 = buf[3 * i];
        const float4 r1 = buf[3 * i + 1];
        const float dx = fx - r0.x, dy = fy - r0.y;
        const float u = fmaf(r0.w, dy, r0.z * dx);
        const float p = fmaf(r1.x * dy, dy, dx * u);
        if (p > 0.0f) continue;
        const float al = fminf(kAlphaMax, r1.y * ex2_approx(p));
        if (al < kAlphaMin) continue;
        const float Tn = fmaf(-al, s.T, s.T);
        if (Tn < kTStop) {
            s.term = true;
            s.evals = pos0 + i + 1;
            return;
        }
        const float w = al * s.T;
        const float rb = reinterpret_cast<const float *>(buf)[12 * i + 8];
        s.C0 = fmaf(w, r1.z, s.C0);
        s.C1 = fmaf(w, r1.w, s.C1);
        s.C2 = fmaf(w, rb, s.C2);
        s.T = Tn;
        s.last = pos0 + i + 1;
    }
    s.evals = pos0 + cnt;
}

// All threads: arm the buffer's mbarrier with the chunk's byte count, then
// each thread issues bulk copies of its share of the gathered records.
__device__ __forceinline__ void issue_chunk(const RasterArgs &a, const Chunk &ch, float4 *buf,
                                            uint64_t *bar) {
    if (ch.cnt == 0) return;
    if (threadIdx.x == 0) mbar_expect_tx(bar, ch.cnt * kRecBytes);
    __syncthreads();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (uint32_t i = threadIdx.x; i < ch.cnt; i += kRasterThreads) {
        uint32_t g = a.gidx[ch.start + i];
        if (g >= a.n_rec) g = 0;  // unreachable unless binning reported an error
        bulk_copy_g2s(buf + 3 * i, a.rec + 3 * (size_t)g, kRecBytes, bar);
    }
}

__device__ __forceinline__ bool wait_chunk(const RasterArgs &a, uint64_t *bar, uint32_t parity) {
    for (uint32_t spins = 0; spins < kSpinLimit; spins++)
        if (mbar_try_wait(bar, parity)) return true;
    atomicOr(a.err, (unsigned long long)kStatusTimeout);
    for (uint32_t spins = 0; spins < kSpinLimit; spins++)  // copies still in flight
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ PixelState load_state(const RasterArgs &a, uint32_t c) {
    float4 st = __ldcg(a.state + (size_t)c * kRasterThreads + threadIdx.x);
    uint2 st2 = __ldcg(a.state2 + (size_t)c * kRasterThreads + threadIdx.x);
    PixelState s = {st.x, st.y, st.z, st.w, st2.x, st2.y & ~kTermBit, (st2.y & kTermBit) != 0};
    return s;
}

__global__ void __launch_bounds__(kRasterThreads)
raster_kernel(RasterArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t s_next;
    __shared__ uint32_t s_flag;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_next = atomicAdd(a.ticket, 1u);
    }
    __syncthreads();
    const uint32_t total = a.chunk_off[a.tiles];
    uint32_t cur = s_next;
    uint32_t parity = 0u;  // bit b: phase parity of buffer b's mbarrier
    int b = 0;
    auto buf = [&](int i) { return reinterpret_cast<float4 *>(smem + i * kBufBytes); };
    Chunk ch = {0, 0, 0, 0, 0};
    if (cur < total) {
        ch = chunk_of(a, cur);
        issue_chunk(a, ch, buf(b), &bars[b]);
    }
    while (cur < total) {
        // prefetch the next chunk into the other buffer
        __syncthreads();
        if (tid == 0) s_next = atomicAdd(a.ticket, 1u);
        __syncthreads();
        const uint32_t nxt = s_next;
        Chunk nch = {0, 0, 0, 0, 0};
        if (nxt < total) {
            nch = chunk_of(a, nxt);
            issue_chunk(a, nch, buf(b ^ 1), &bars[b ^ 1]);
        }
        if (ch.cnt > 0) {
            if (!wait_chunk(a, &bars[b], (parity >> b) & 1u)) return;
            parity ^= 1u << b;
        }
        // ---- blend this chunk
        const int tx = ch.t % a.tiles_x, ty = ch.t / a.tiles_x;
        const int px = tx * 16 + (tid & 15), py = ty * 16 + (tid >> 4);
        const bool inside = px < a.W && py < a.H;
        const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
        const uint32_t pos0 = ch.k * kChunk;
        PixelState s = {0.0f, 0.0f, 0.0f, 1.0f, 0u, pos0, false};
        bool exact = ch.k == 0;
        const uint32_t prev = cur - 1;
        if (!exact) {
            if (tid == 0) s_flag = ld_acquire(a.flags + prev);
            __syncthreads();
            if (s_flag) {
                exact = true;
                s = load_state(a, prev);
            }
        }
        if (inside && !s.term) blend_chunk(buf(b), ch.cnt, pos0, fx, fy, s);
        if (!exact) {
            // wait for the predecessor's inclusive state, then merge
            if (tid == 0) {
                uint32_t spins = 0;
                while (ld_acquire(a.flags + prev) == 0) {
                    if (++spins > kSpinLimit) {
                        atomicOr(a.err, (unsigned long long)kStatusTimeout);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __syncthreads();
            PixelState in = load_state(a, prev);
            if (in.term) {
                s = in;
            } else if (!s.term && in.T * s.T >= kTStop) {
                s.C0 = fmaf(in.T, s.C0, in.C0);
                s.C1 = fmaf(in.T, s.C1, in.C1);
                s.C2 = fmaf(in.T, s.C2, in.C2);
                s.T = in.T * s.T;
                if (s.last <= pos0) s.last = in.last;
            } else {
                s = in;
                if (inside) blend_chunk(buf(b), ch.cnt, pos0, fx, fy, s);
            }
        }
        if (ch.k + 1 < ch.nk) {
            a.state[(size_t)cur * kRasterThreads + tid] = make_float4(s.C0, s.C1, s.C2, s.T);
            a.state2[(size_t)cur * kRasterThreads + tid] =
                make_uint2(s.last, s.evals | (s.term ? kTermBit : 0u));
            __threadfence();
            __syncthreads();
            if (tid == 0) st_release(a.flags + cur, 1u);
        } else if (inside) {
            const size_t p = (size_t)py * a.W + px, plane = (size_t)a.W * a.H;
            a.image[p] = fmaf(s.T, a.bg0, s.C0);
            a.image[plane + p] = fmaf(s.T, a.bg1, s.C1);
            a.image[2 * plane + p] = fmaf(s.T, a.bg2, s.C2);
            if (a.final_t) a.final_t[p] = s.T;
            if (a.n_contrib) a.n_contrib[p] = s.last;
            if (a.n_eval) a.n_eval[p] = s.evals;
        }
        cur = nxt;
        ch = nch;
        b ^= 1;
    }
}

struct RasterLayout {
    size_t ticket, chunk_off, flags, state, state2, total, zero_bytes;
    int64_t max_chunks;
};

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static bool raster_layout(int64_t tiles, int64_t cap, RasterLayout &L) {
    if (tiles < 1 || tiles > 65536 || cap < 1 || cap > (1ll << 30)) return false;
    L.max_chunks = tiles + ceil_div(cap, kChunk);
    size_t o = 0;
    L.ticket = o;
    o = al256(o + 4);
    L.flags = o;
    o = al256(o + (size_t)L.max_chunks * 4);
    L.zero_bytes = o;
    L.chunk_off = o;
    o = al256(o + (size_t)(tiles + 1) * 4);
    L.state = o;
    o = al256(o + (size_t)L.max_chunks * kRasterThreads * sizeof(float4));
    L.state2 = o;
    o = al256(o + (size_t)L.max_chunks * kRasterThreads * sizeof(uint2));
    L.total = o;
    return true;
}

static int raster_grid() {
    static int blocks_per_sm = 0;
    if (blocks_per_sm == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, raster_kernel, kRasterThreads,
                                                          2 * kBufBytes) != cudaSuccess ||
            v < 1)
            v = 1;
        blocks_per_sm = v;
    }
    return blocks_per_sm * num_sms();
}

}  // namespace msgs

using namespace msgs;

extern "C" size_t ms_raster_workspace_bytes(int64_t tiles, int64_t dup_capacity) {
    RasterLayout L;
    if (!raster_layout(tiles, dup_capacity, L)) return 0;
    return L.total;
}

extern "C" int ms_raster(const ms_proj_t *proj, const ms_bins_t *bins, const ms_camera_t *cam,
                         float *image, float *final_t, uint32_t *n_contrib, uint32_t *n_eval,
                         void *ws, size_t ws_bytes, void *stream) {
    if (!proj || !bins || !cam || !image) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
        return fail(MS_ERR_INVALID_ARG, "image size must be 1..32768");
    if (!proj->rec || !aligned(proj->rec, 16)) return fail(MS_ERR_INVALID_ARG, "rec NULL or misaligned");
    if (!bins->gauss_idx || !bins->ranges || !bins->counts)
        return fail(MS_ERR_INVALID_ARG, "bins buffers NULL");
    if (proj->n < 1 || proj->n > INT32_MAX)
        return fail(MS_ERR_INVALID_ARG, "ms_proj_t n must be 1..2^31-1");
    const int tiles_x = (cam->width + 15) / 16, tiles_y = (cam->height + 15) / 16;
    const int64_t tiles = (int64_t)tiles_x * tiles_y;
    RasterLayout L;
    if (!raster_layout(tiles, bins->dup_capacity, L))
        return fail(MS_ERR_INVALID_ARG, "tiles or dup_capacity out of range");
    if (!ws || ws_bytes < L.total || !aligned(ws, 16))
        return fail(MS_ERR_INVALID_ARG, "raster workspace missing, too small or misaligned");
    cudaStream_t st = as_stream(stream);
    char *w = static_cast<char *>(ws);
    int rc;
    static bool attr_set = false;
    if (!attr_set) {
        if ((rc = cuda_check(cudaFuncSetAttribute(raster_kernel,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  2 * kBufBytes),
                             "raster smem attribute")))
            return rc;
        attr_set = true;
    }
    if ((rc = cuda_check(cudaMemsetAsync(w, 0, L.zero_bytes, st), "raster workspace memset")))
        return rc;
    RasterArgs a;
    a.ranges = bins->ranges;
    a.gidx = bins->gauss_idx;
    a.rec = reinterpret_cast<const float4 *>(proj->rec);
    a.n_rec = (uint32_t)proj->n;
    a.W = cam->width;
    a.H = cam->height;
    a.tiles_x = tiles_x;
    a.tiles = (int)tiles;
    a.bg0 = cam->bg[0];
    a.bg1 = cam->bg[1];
    a.bg2 = cam->bg[2];
    a.image = image;
    a.final_t = final_t;
    a.n_contrib = n_contrib;
    a.n_eval = n_eval;
    a.chunk_off = reinterpret_cast<uint32_t *>(w + L.chunk_off);
    a.ticket = reinterpret_cast<uint32_t *>(w + L.ticket);
    a.flags = reinterpret_cast<uint32_t *>(w + L.flags);
    a.state = reinterpret_cast<float4 *>(w + L.state);
    a.state2 = reinterpret_cast<uint2 *>(w + L.state2);
    a.err = reinterpret_cast<unsigned long long *>(bins->counts) + kCntStatus;
    chunk_offsets_kernel<<<1, 1024, 0, st>>>(bins->ranges, (int)tiles, a.chunk_off);
    raster_kernel<<<raster_grid(), kRasterThreads, 2 * kBufBytes, st>>>(a);
    return cuda_check(cudaGetLastError(), "raster launches");
}

// Front-to-back blending per 16x16 tile (Sec. 3.1; Eq. 3 with incremental
// transmittance T_k): a 256-thread CTA walks a segment of a tile's sorted
// list, one thread per pixel.
//
// Load balance: low resolutions put thousands of splats on a few tiles
// (Sec. 3.2, item 2), so one CTA per tile would leave most SMs idle.  Each
// tile's list is cut into segments of seg_len = max(kMinSegment, D /
// resident CTAs) entries; only tiles longer than a fair share of the work
// are split.
// A CTA walks its segment in sub-batches of kChunk records, double-buffered:
// the next sub-batch arrives in shared memory by per-record bulk copies
// (cp.async.bulk) on an mbarrier while the current one is blended.
//
// The blend stays exactly sequential across segments (decoupled look-back):
//   - a segment whose predecessor has published its inclusive prefix
//     starts from that per-pixel (C, T) and applies the termination rule
//     directly;
//   - otherwise it blends from T = 1 into a local aggregate (C_l, T_l),
//     publishes it, and folds forward from the nearest published prefix
//     over the aggregates after it to get its exact (C_in, T_in).  If no
//     termination can fall inside the segment (T_in T_l >= 1e-4, T being
//     monotone) the result is C_in + T_in C_l, T_in T_l; otherwise the pixel
//     terminates inside the segment: it is handed on as terminated at once,
//     and the segment is walked again from T_in to find the exact stopping
//     point.
// Each pixel is written by the segment it terminates in, or by its tile's
// last segment.  A segment after which every pixel has terminated marks
// the tile done; later segments of that tile stop as soon as they see the
// mark.  Every wait is bounded; a wait that gives
// up sets a status bit and the CTA carries on.
#include <cuda_runtime.h>

#include <atomic>
#include <stdint.h>

#include "common.cuh"
#include "f32x2.cuh"
#include "tma.cuh"
#include "raster_ws.cuh"
#include "raster_list.cuh"

namespace msgs {

constexpr int kRecBytes = 48;                // one raster record
constexpr int kBufBytes = kChunk * kRecBytes;  // staged records, as copied
constexpr int kPairs = kChunk / 2;
constexpr float kAlphaMax = 0.99f;
constexpr float kTStop = 1e-4f;
#ifndef MS_RASTER_WINDOW
#define MS_RASTER_WINDOW 16
#endif
// Segments of one tile walked at once: segment k starts when segment k - W
// has published its result (or the tile is done).  Pixels of low-resolution
// frames terminate long before the end of their tile's list, and every
// segment started past that point is wasted work.
constexpr uint32_t kWindow = MS_RASTER_WINDOW;
constexpr uint32_t kAgg = 1u;                // segment flag: local aggregate published
constexpr uint32_t kPre = 2u;                // segment flag: inclusive prefix published
// ms_raster (AUTO) launches both blend kernels for frames with at least as
// many tiles as SMs and fewer than kListBandSms times as many, and the list
// kernel takes the frame when its mean list length lies in kListMeanMin ..
// kListMeanMax.
constexpr int64_t kListBandSms = 4;
constexpr uint32_t kListMeanMin = 1024;
constexpr uint32_t kListMeanMax = 8192;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
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
    uint32_t *seg_off;    // [tiles + 1] exclusive prefix of segments per tile
    uint32_t *seg_len;    // [1] entries per segment (a multiple of kChunk)
    uint32_t *ticket;
    uint32_t *flags;      // [max_segs] 0, kAgg (local aggregate), kPre (prefix)
    uint32_t *tile_done;  // [tiles] every pixel terminated, image written
    float4 *agg;          // [max_segs][256] local (C0, C1, C2, T) from T = 1
    uint2 *agg2;          // [max_segs][256] (n_contrib, n_eval | term bit)
    float4 *pre;          // [max_segs][256] inclusive (C0, C1, C2, T)
    uint2 *pre2;          // [max_segs][256] (n_contrib, n_eval | term bit)
    const uint32_t *use_list;  // NULL, or nonzero when the list kernel blends this frame instead
    unsigned long long *err;
};

struct Seg {
    uint32_t t, k, nk, start, len;
};

__device__ __forceinline__ Seg seg_of(const RasterArgs &a, uint32_t c, uint32_t L) {
    int lo = 0, hi = a.tiles;  // seg_off[lo] <= c < seg_off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (a.seg_off[mid] <= c) lo = mid;
        else hi = mid;
    }
    Seg sg;
    sg.t = lo;
    sg.k = c - a.seg_off[lo];
    sg.nk = a.seg_off[lo + 1] - a.seg_off[lo];
    uint32_t s = a.ranges[2 * lo], e = a.ranges[2 * lo + 1];
    sg.start = s + sg.k * L;
    uint32_t stop = min(e, sg.start + L);
    sg.len = stop > sg.start ? stop - sg.start : 0;
    return sg;
}

// One block: D = sum of list lengths, segment length L = max(kChunk,
// ceil(D / resident) rounded up to kChunk), then the number of segments of
// every tile (at least one, so empty tiles still write the background),
// exclusive-scanned.  It also zeroes the n_zero16 16-byte words at zero (the
// tile kernel's ticket, segment flags and tile marks; none for the list
// kernel), which the raster launch after it reads.  With use_list, it
// writes there which blend kernel takes the frame: the list kernel when the
// mean list length D / tiles lies in list_mean_min .. list_mean_max, else
// the tile kernel.
__global__ void __launch_bounds__(1024)
segment_offsets_kernel(const uint32_t *__restrict__ ranges, int tiles, uint32_t resident,
                       uint32_t *__restrict__ off, uint32_t *__restrict__ seg_len,
                       uint4 *__restrict__ zero, uint32_t n_zero16,
                       uint32_t *__restrict__ use_list, uint32_t list_mean_min,
                       uint32_t list_mean_max) {
    __shared__ uint32_t s_warp[32];
    __shared__ unsigned long long s_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint32_t i = tid; i < n_zero16; i += 1024) zero[i] = make_uint4(0u, 0u, 0u, 0u);
    const int per = (tiles + 1023) / 1024;
    const int t0 = tid * per;
    if (tid == 0) s_total = 0;
    __syncthreads();
    unsigned long long d = 0;
    for (int t = t0; t < t0 + per && t < tiles; t++) d += ranges[2 * t + 1] - ranges[2 * t];
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0 && d) atomicAdd(&s_total, d);
    __syncthreads();
    unsigned long long share = (s_total + resident - 1) / (resident > 0 ? resident : 1);
    uint32_t L = (uint32_t)(((share + kChunk - 1) / kChunk) * kChunk);
    if (L < kMinSegment) L = kMinSegment;
    uint32_t sum = 0;
    for (int t = t0; t < t0 + per && t < tiles; t++) {
        uint32_t len = ranges[2 * t + 1] - ranges[2 * t];
        sum += len > 0 ? (len + L - 1) / L : 1u;
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
        run += len > 0 ? (len + L - 1) / L : 1u;
    }
    if (tid == 1023) {
        off[tiles] = run;
        seg_len[0] = L;
        if (use_list)
            use_list[0] = s_total >= (unsigned long long)list_mean_min * (unsigned long long)tiles &&
                          s_total <= (unsigned long long)list_mean_max * (unsigned long long)tiles;
    }
}

struct PixelState {
    float C0, C1, C2, T;
    uint32_t last, evals;
    bool term;
};

// One warp's share of a staged sub-batch: the records whose alpha >= 1/255
// level set can reach the warp's 8x4 pixel block, in list order, regrouped
// into pairs (2m, 2m+1) with each field of the two records side by side,
// so one packed FP32x2 instruction evaluates both records' power terms.
struct WarpPairs {
    float4 q0[kPairs];     // ux0 ux1 uy0 uy1
    float4 q1[kPairs];     // A0 A1 B0 B1
    float4 q2[kPairs];     // C0 C1 thr0 thr1
    float4 q3[kPairs];     // opacity0 opacity1 r0 r1
    float4 q4[kPairs];     // g0 g1 b0 b1
    uint16_t idx[kChunk];  // index of each record within the sub-batch
};
constexpr int kWarps = kRasterThreads / 32;
constexpr int kSmemBytes = 2 * kBufBytes + kWarps * (int)sizeof(WarpPairs);
// Half extents of a warp's block of pixel centres (8 x 4 pixels) plus a
// margin for FP32 rounding: the record's half extents bound the exact
// alpha >= 1/255 level set, and the rounding of that bound and of the
// distances is below 1e-4 px at the largest image coordinates.
#ifndef MS_CULL_MARGIN
#define MS_CULL_MARGIN 0.0625f
#endif
constexpr float kBlockHalfX = 3.5f + MS_CULL_MARGIN;
constexpr float kBlockHalfY = 1.5f + MS_CULL_MARGIN;

// Compact the records [0, cnt) of the staged sub-batch whose level-set box
// (centre +- (ex, ey)) can reach the warp's block of pixel centres
// (centre (cx, cy)) into the warp's pair buffer, keeping list order.  Any
// other record has alpha < 1/255 at every pixel of the block, so skipping
// it changes nothing.  An odd count is padded with a record that no pixel
// accepts (thr = +inf).  Returns the count (warp-uniform).
__device__ __forceinline__ uint32_t compact(const float4 *__restrict__ aos, uint32_t cnt,
                                            float cx, float cy, WarpPairs &wp) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t base = 0;
#pragma unroll
    for (int k = 0; k < kChunk / 32; k++) {
        const uint32_t i = (uint32_t)k * 32u + lane;
        bool rel = false;
        float4 r0, r2;
        if (i < cnt) {
            r0 = aos[3 * i];
            r2 = aos[3 * i + 2];
            rel = fabsf(r0.x - cx) <= r2.z + kBlockHalfX && fabsf(r0.y - cy) <= r2.w + kBlockHalfY;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, rel);
        if (rel) {
            const float4 r1 = aos[3 * i + 1];
            const uint32_t p = base + __popc(m & ((1u << lane) - 1u));
            const uint32_t q = p >> 1, h = p & 1u;
            float *q0 = reinterpret_cast<float *>(&wp.q0[q]);
            float *q1 = reinterpret_cast<float *>(&wp.q1[q]);
            float *q2 = reinterpret_cast<float *>(&wp.q2[q]);
            float *q3 = reinterpret_cast<float *>(&wp.q3[q]);
            float *q4 = reinterpret_cast<float *>(&wp.q4[q]);
            q0[h] = r0.x;
            q0[2 + h] = r0.y;
            q1[h] = r0.z;
            q1[2 + h] = r0.w;
            q2[h] = r1.x;
            q2[2 + h] = r2.y;
            q3[h] = r1.y;
            q3[2 + h] = r1.z;
            q4[h] = r1.w;
            q4[2 + h] = r2.x;
            wp.idx[p] = (uint16_t)i;
        }
        base += __popc(m);
    }
    if ((base & 1u) && lane == 0) {
        const uint32_t q = base >> 1;
        float *q0 = reinterpret_cast<float *>(&wp.q0[q]);
        float *q1 = reinterpret_cast<float *>(&wp.q1[q]);
        float *q2 = reinterpret_cast<float *>(&wp.q2[q]);
        float *q3 = reinterpret_cast<float *>(&wp.q3[q]);
        float *q4 = reinterpret_cast<float *>(&wp.q4[q]);
        q0[1] = q0[3] = q1[1] = q1[3] = q2[1] = 0.0f;
        q2[3] = __int_as_float(0x7f800000);
        q3[1] = q3[3] = q4[1] = q4[3] = 0.0f;
        wp.idx[base] = 0;
    }
    __syncwarp();
    return base;
}

// One record's contribution once it passed the alpha test: stop before a
// Gaussian that would bring T below 1e-4, else accumulate and advance T.
// Returns true when the pixel terminated.
__device__ __forceinline__ bool blend_one(float p, float opacity, float r, float g, float b,
                                          uint32_t pos, PixelState &s) {
    const float al = fminf(kAlphaMax, opacity * ex2_approx(p));
    const float Tn = fmaf(-al, s.T, s.T);
    if (Tn < kTStop) {
        s.term = true;
        s.evals = pos;
        return true;
    }
    const float w = al * s.T;
    s.C0 = fmaf(w, r, s.C0);
    s.C1 = fmaf(w, g, s.C1);
    s.C2 = fmaf(w, b, s.C2);
    s.T = Tn;
    s.last = pos;
    return false;
}

// Blend the warp's n compacted records of a sub-batch of cnt into s.  pos0
// is the list position of the sub-batch's first record.  power * log2(e)
// = A dx^2 + B dx dy + C dy^2 is evaluated for both records of a pair at
// once; a record is skipped when the power is positive or alpha would stay
// below 1/255 (power * log2(e) < thr).
__device__ __forceinline__ void blend_pairs(const WarpPairs &wp, uint32_t n, uint32_t cnt,
                                            uint32_t pos0, f32x2 fx2, f32x2 fy2, PixelState &s) {
    const uint32_t np = (n + 1) >> 1;
#pragma unroll 2
    for (uint32_t m = 0; m < np; m++) {
        const ulonglong2 v0 = *reinterpret_cast<const ulonglong2 *>(&wp.q0[m]);
        const ulonglong2 v1 = *reinterpret_cast<const ulonglong2 *>(&wp.q1[m]);
        const ulonglong2 v2 = *reinterpret_cast<const ulonglong2 *>(&wp.q2[m]);
        const f32x2 dx = sub2(fx2, v0.x), dy = sub2(fy2, v0.y);
        const f32x2 u = fma2(v1.y, dy, mul2(v1.x, dx));
        const f32x2 pw = fma2(mul2(v2.x, dy), dy, mul2(dx, u));
        float p0, p1, t0, t1;
        unpack2(pw, p0, p1);
        unpack2(v2.y, t0, t1);
        const bool h0 = p0 <= 0.0f && p0 >= t0;
        const bool h1 = p1 <= 0.0f && p1 >= t1;
        if (!(h0 || h1)) continue;
        const float4 w3 = wp.q3[m], w4 = wp.q4[m];
        const uint32_t ix = *reinterpret_cast<const uint32_t *>(&wp.idx[2 * m]);
        if (h0 && blend_one(p0, w3.x, w3.z, w4.x, w4.z, pos0 + (ix & 0xffffu) + 1, s)) return;
        if (h1 && blend_one(p1, w3.y, w3.w, w4.y, w4.w, pos0 + (ix >> 16) + 1, s)) return;
    }
    s.evals = pos0 + cnt;
}

// Thread 0 arms the buffer's mbarrier with the sub-batch's byte count and
// every thread issues the bulk copies of its gathered records.  The phase
// cannot complete before the arming arrival, so no barrier is needed
// between the two; the caller guarantees that every warp is done reading
// the buffer.
__device__ __forceinline__ void issue_batch(const RasterArgs &a, uint32_t first, uint32_t cnt,
                                            float4 *buf, uint64_t *bar) {
    MS_DCHECK(cnt <= (uint32_t)kChunk, a.err);
    if (threadIdx.x == 0) mbar_expect_tx(bar, cnt * kRecBytes);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (uint32_t i = threadIdx.x; i < cnt; i += kRasterThreads) {
        uint32_t g = a.gidx[first + i];
        MS_DCHECK(g < a.n_rec, a.err);
        if (g >= a.n_rec) g = 0;  // unreachable unless binning reported an error
        bulk_copy_g2s(buf + 3 * i, a.rec + 3 * (size_t)g, kRecBytes, bar);
    }
}

__device__ __forceinline__ bool wait_batch(const RasterArgs &a, uint64_t *bar, uint32_t parity) {
    for (uint32_t spins = 0; spins < kSpinLimit; spins++)
        if (mbar_try_wait(bar, parity)) return true;
    atomicOr(a.err, (unsigned long long)kStatusTimeout);
    for (uint32_t spins = 0; spins < kSpinLimit; spins++)  // copies still in flight
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ PixelState load_state(const float4 *v, const uint2 *v2, uint32_t c) {
    float4 st = __ldcg(v + (size_t)c * kRasterThreads + threadIdx.x);
    uint2 st2 = __ldcg(v2 + (size_t)c * kRasterThreads + threadIdx.x);
    PixelState s = {st.x, st.y, st.z, st.w, st2.x, st2.y & ~kTermBit, (st2.y & kTermBit) != 0};
    return s;
}

__device__ __forceinline__ void store_state(float4 *v, uint2 *v2, uint32_t c,
                                            const PixelState &s) {
    v[(size_t)c * kRasterThreads + threadIdx.x] = make_float4(s.C0, s.C1, s.C2, s.T);
    v2[(size_t)c * kRasterThreads + threadIdx.x] =
        make_uint2(s.last, s.evals | (s.term ? kTermBit : 0u));
}

// The exact state after one more segment, from the state P before it and
// the segment's local result X (blended from T = 1).  A pixel terminates in
// the segment when X terminated locally or P.T X.T < 1e-4 (T is monotone);
// its colour then needs a re-walk, the fold only records the termination.
// Every segment folds with this one function in list order, so all of them
// reach bit-identical prefixes and the same termination decisions.
__device__ __forceinline__ PixelState fold(const PixelState &P, const PixelState &X) {
    if (P.term) return P;
    PixelState r = P;
    if (X.term || P.T * X.T < kTStop) {
        r.term = true;
        return r;
    }
    r.C0 = fmaf(P.T, X.C0, P.C0);
    r.C1 = fmaf(P.T, X.C1, P.C1);
    r.C2 = fmaf(P.T, X.C2, P.C2);
    r.T = P.T * X.T;
    r.last = X.last != 0 ? X.last : P.last;
    r.evals = X.evals;
    return r;
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p) {
    return *reinterpret_cast<const volatile uint32_t *>(p);
}

// Walk one segment in sub-batches through two staging buffers: while the
// warps compact and blend sub-batch j from one buffer, the bulk copies of
// sub-batch j + 1 land in the other.  One CTA barrier per sub-batch (the
// termination count) also guarantees that every warp has compacted
// sub-batch j before sub-batch j + 2 is copied over it.  In local mode
// (`exact` false) the walk stops as soon as the tile is marked done.  The
// CTA stops early once every pixel has terminated.  Returns kWalked,
// kAborted.  A copy wait that gives up sets the status word and ends the
// waiting warps' pixels; the walk stays in step across the CTA.
constexpr int kWalked = 0, kAborted = 1;
__device__ __forceinline__ int run_segment(const RasterArgs &a, const Seg &sg, uint32_t L,
                                            bool exact, bool inside, float fx, float fy,
                                            float cx, float cy, PixelState &s,
                                            float4 *aos, WarpPairs &wp, uint64_t *bar,
                                            uint32_t &par, uint32_t *s_abort) {
    const uint32_t pos0 = sg.k * L;
    if (sg.len == 0) return kWalked;
    const uint32_t nb = (sg.len + kChunk - 1) / kChunk;
    const f32x2 fx2 = pack2(fx, fx), fy2 = pack2(fy, fy);
    issue_batch(a, sg.start, min(sg.len, (uint32_t)kChunk), aos, &bar[0]);
    bool abort = false;
    for (uint32_t j = 0; j < nb; j++) {
        const uint32_t b = j & 1u, off = j * kChunk;
        const uint32_t cnt = min(sg.len - off, (uint32_t)kChunk);
        const bool ok = wait_batch(a, &bar[b], (par >> b) & 1u);
        par ^= 1u << b;
        const bool more = j + 1 < nb;
        if (more)
            issue_batch(a, sg.start + off + kChunk, min(sg.len - off - kChunk, (uint32_t)kChunk),
                        aos + (b ^ 1u) * 3 * kChunk, &bar[b ^ 1u]);
        // a copy wait that gave up has set the status word: the warp's pixels
        // stop here (their result is reported wrong), the walk goes on in
        // step with the other warps
        const bool wok = __all_sync(0xffffffffu, ok);
        if (!wok) s.term = true;
        // warps whose pixels have all terminated skip their share
        const bool wlive = wok && __any_sync(0xffffffffu, inside && !s.term);
        const uint32_t nw = wlive ? compact(aos + b * 3 * kChunk, cnt, cx, cy, wp) : 0u;
        if (wlive && inside && !s.term) blend_pairs(wp, nw, cnt, pos0 + off, fx2, fy2, s);
        // two slots: a warp may still be reading sub-batch j's value while
        // thread 0 writes sub-batch j + 1's (one barrier per sub-batch)
        if (threadIdx.x == 0) s_abort[b] = exact ? 0u : ld_volatile(a.tile_done + sg.t);
        const int done = __syncthreads_count(s.term || !inside);
        abort = s_abort[b] != 0;
        if (done == kRasterThreads || abort) {
            if (more) {  // drain the copies already issued
                wait_batch(a, &bar[b ^ 1u], (par >> (b ^ 1u)) & 1u);
                par ^= 1u << (b ^ 1u);
            }
            break;
        }
    }
    return abort ? kAborted : kWalked;
}

__global__ void __launch_bounds__(kRasterThreads, 4)  // 64 registers: 4 CTAs per SM
raster_kernel(RasterArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t s_next;
    __shared__ uint32_t s_flag;
    __shared__ uint32_t s_wait;
    __shared__ uint32_t s_abort[2];
    if (a.use_list && *a.use_list) return;  // the list kernel blends this frame
    float4 *aos = reinterpret_cast<float4 *>(smem);
    WarpPairs &wp = reinterpret_cast<WarpPairs *>(smem + 2 * kBufBytes)[threadIdx.x >> 5];
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const uint32_t total = a.seg_off[a.tiles];
    const uint32_t L = a.seg_len[0];
    uint32_t parity = 0u;  // phase parity of bar[0] (bit 0) and bar[1] (bit 1)
    for (;;) {
        __syncthreads();
        if (tid == 0) s_next = atomicAdd(a.ticket, 1u);
        __syncthreads();
        const uint32_t c = s_next;
        if (c >= total) break;
        const Seg sg = seg_of(a, c, L);
        if (sg.k >= kWindow) {
            // wait for the segment kWindow places earlier in this tile; it
            // holds an earlier ticket, so its CTA is running
            if (tid == 0) {
                uint32_t skip = 0, spins = 0;
                for (;;) {
                    if (ld_volatile(a.flags + c - kWindow) != 0) break;
                    if (ld_volatile(a.tile_done + sg.t)) {
                        skip = 1;
                        break;
                    }
                    if (++spins > kSpinLimit) {
                        atomicOr(a.err, (unsigned long long)kStatusTimeout);
                        break;
                    }
                    __nanosleep(64);
                }
                s_wait = skip;
            }
            __syncthreads();
            if (s_wait) continue;  // an earlier segment finished the tile
        }
        const uint32_t prev = c - 1;
        bool exact = sg.k == 0;
        if (!exact) {
            if (tid == 0)
                s_flag = ld_volatile(a.tile_done + sg.t) ? 3u : ld_acquire(a.flags + prev);
            __syncthreads();
            if (s_flag == 3u) continue;  // an earlier segment finished the tile
            exact = s_flag == kPre;
        }
        const int tx = sg.t % a.tiles_x, ty = sg.t / a.tiles_x;
        // each warp covers an 8x4 pixel block (2 x 4 blocks per tile): close
        // pixels accept and terminate alike, which keeps lanes converged
        const int wid = tid >> 5, lid = tid & 31;
        const int px = tx * 16 + (wid & 1) * 8 + (lid & 7);
        const int py = ty * 16 + (wid >> 1) * 4 + (lid >> 3);
        const bool inside = px < a.W && py < a.H;
        const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
        // centre of the warp's block of pixel centres
        const float cx = (float)(tx * 16 + (wid & 1) * 8) + 4.0f;
        const float cy = (float)(ty * 16 + (wid >> 1) * 4) + 2.0f;
        PixelState s = {0.0f, 0.0f, 0.0f, 1.0f, 0u, sg.k * L, false};
        bool was_term = false;  // terminated in an earlier segment (already written)
        if (sg.k > 0 && exact) {
            s = load_state(a.pre, a.pre2, prev);
            was_term = s.term;
        }
        // pass 0 walks the segment (exact from the predecessor's prefix, or
        // locally from T = 1); pass 1 re-walks it from the exact prefix for
        // the pixels that terminate inside it, after the prefix is published
        bool active = inside, skip = false, redone = false;
        const bool last_seg = sg.k + 1 == sg.nk;
        for (int pass = 0; pass < 2; pass++) {
            const int rc = run_segment(a, sg, L, exact || pass == 1, active, fx, fy, cx, cy, s,
                                       aos, wp, bar, parity, s_abort);
            if (rc == kAborted) {
                skip = true;  // an earlier segment finished the tile
                break;
            }
            if (pass == 1) break;
            bool redo = false;
            PixelState in = s;
            if (!exact) {
                // publish the local aggregate, then look back: the nearest
                // predecessor with a published prefix, and the aggregates
                // after it
                store_state(a.agg, a.agg2, c, s);
                __threadfence();
                __syncthreads();
                if (tid == 0) {
                    st_release(a.flags + c, kAgg);
                    // batched look-back over the flags of up to 16
                    // predecessors; the tile's first segment never publishes
                    // an aggregate, so the walk ends there at the latest
                    const uint32_t c0 = c - sg.k;
                    uint32_t j = prev, spins = 0, res = 0;
                    for (;;) {
                        uint32_t pre_mask = 0, agg_mask = 0;
#pragma unroll
                        for (int i = 0; i < 16; i++) {
                            const uint32_t f = (j >= c0 + i) ? ld_relaxed(a.flags + j - i) : 0u;
                            pre_mask |= (uint32_t)(f == kPre) << i;
                            agg_mask |= (uint32_t)(f == kAgg) << i;
                        }
                        // leading run of aggregates, then a prefix or a gap
                        const uint32_t run = __ffs(~agg_mask) - 1;
                        j -= run;
                        if (run < 16 && ((pre_mask >> run) & 1u)) {
                            fence_acquire();  // the states behind the flags seen
                            break;
                        }
                        if (run < 16) {
                            // j has published nothing yet
                            if (ld_volatile(a.tile_done + sg.t)) {
                                res = 1u;
                                break;
                            }
                            if (++spins > kSpinLimit) {
                                atomicOr(a.err, (unsigned long long)kStatusTimeout);
                                res = 1u;
                                break;
                            }
                            __nanosleep(32);
                        }
                    }
                    s_flag = res;
                    s_next = j;
                }
                __syncthreads();
                if (s_flag) {
                    skip = true;
                    break;
                }
                const uint32_t j = s_next;
                in = load_state(a.pre, a.pre2, j);
                // fold the aggregates after j, four loads in flight at a time;
                // stop once every pixel is known to have terminated before this
                // segment (the segments it terminated in write it)
                uint32_t i = j + 1;
                for (; i + 4 <= c; i += 4) {
                    PixelState x0 = load_state(a.agg, a.agg2, i);
                    PixelState x1 = load_state(a.agg, a.agg2, i + 1);
                    PixelState x2 = load_state(a.agg, a.agg2, i + 2);
                    PixelState x3 = load_state(a.agg, a.agg2, i + 3);
                    in = fold(fold(fold(fold(in, x0), x1), x2), x3);
                    if (__syncthreads_and(in.term || !inside)) {
                        i = c;
                        break;
                    }
                }
                for (; i < c; i++) in = fold(in, load_state(a.agg, a.agg2, i));
                if (in.term) {
                    s = in;
                    was_term = true;
                } else if (!s.term && in.T * s.T >= kTStop) {
                    s = fold(in, s);
                } else {
                    // the pixel terminates inside this segment: successors
                    // only need to know that; its exact result comes next
                    redo = inside;
                    s.term = true;
                }
            }
            // publish the inclusive prefix before any re-walk, so no
            // successor ever waits for one
            const bool all_done = __syncthreads_and(s.term || !inside);
            if (!last_seg) {
                if (!all_done) store_state(a.pre, a.pre2, c, s);
                __threadfence();
                __syncthreads();
                if (tid == 0) st_release(all_done ? a.tile_done + sg.t : a.flags + c,
                                         all_done ? 1u : kPre);
            }
            if (!__syncthreads_or(redo)) break;
            if (redo) s = in;
            active = redo;
            redone = redo;
        }
        if (skip) continue;
        // every pixel is written once: by the segment it terminates in, or
        // by the tile's last segment
        if (inside && !was_term && (s.term || last_seg || redone)) {
            const size_t p = (size_t)py * a.W + px, plane = (size_t)a.W * a.H;
            MS_DCHECK(p < plane, a.err);
            a.image[p] = fmaf(s.T, a.bg0, s.C0);
            a.image[plane + p] = fmaf(s.T, a.bg1, s.C1);
            a.image[2 * plane + p] = fmaf(s.T, a.bg2, s.C2);
            if (a.final_t) a.final_t[p] = s.T;
            if (a.n_contrib) a.n_contrib[p] = s.last;
            if (a.n_eval) a.n_eval[p] = s.evals;
        }
    }
}

static int raster_blocks_per_sm() {
    // the same for every device of the one architecture this library targets
    static std::atomic<int> blocks_per_sm{0};
    int b = blocks_per_sm.load(std::memory_order_relaxed);
    if (b == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, raster_kernel, kRasterThreads,
                                                          kSmemBytes) != cudaSuccess ||
            b < 1)
            b = 1;
        blocks_per_sm.store(b, std::memory_order_relaxed);
    }
    return b;
}

}  // namespace msgs

using namespace msgs;

extern "C" size_t ms_raster_workspace_bytes(int64_t tiles, int64_t dup_capacity) {
    RasterLayout L;
    if (!raster_layout(tiles, dup_capacity, L)) return 0;
    return L.total;
}

extern "C" int ms_raster_ex2(const ms_proj_t *proj, const ms_bins_t *bins,
                             const ms_camera_t *cam, float *image, float *final_t,
                             uint32_t *n_contrib, uint32_t *n_eval, void *ws, size_t ws_bytes,
                             int strategy, int32_t max_ctas_per_sm, void *stream) {
    if (strategy < MS_RASTER_AUTO || strategy > MS_RASTER_GROUP32)
        return fail(MS_ERR_INVALID_ARG, "unknown raster strategy");
    if (max_ctas_per_sm < 0) return fail(MS_ERR_INVALID_ARG, "max_ctas_per_sm must be >= 0");
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
    if ((rc = ensure_smem_attr(reinterpret_cast<const void *>(raster_kernel), kSmemBytes)))
        return rc;
    // the tile kernel's persistent CTAs: as many as fit, or at most
    // max_ctas_per_sm per SM so that other frames' kernels find room beside it
    const int per_sm = max_ctas_per_sm > 0 ? std::min(raster_blocks_per_sm(), (int)max_ctas_per_sm)
                                           : raster_blocks_per_sm();
    const int resident = (int)std::min<int64_t>((int64_t)per_sm * num_sms(), kMaxResident);
    // A frame with fewer tiles than SMs would leave SMs without a tile: the
    // tile kernel then splits every list into many segments, most of them
    // blended speculatively, and the list kernel is faster.  Up to
    // kListBandSms x SMs tiles (and no cap on the tile kernel's CTAs), the
    // frame's mean list length decides on the device (both kernels are
    // launched, the one not chosen returns at once): lists of
    // kListMeanMin .. kListMeanMax entries per tile (selective frames, whose
    // pixels walk deep into them) go to the list kernel; short ones, which
    // the tile kernel walks quickly, and long ones (all levels, whose
    // pixels end early in lists whose first kMaskPrefix entries the list
    // kernel's mask pass covers whole) to the tile kernel.  Measured on
    // GB300, 314x208 frames of the 1M-Gaussian scene: selective (3.5k
    // entries per tile) list 120 against tile 184 us; all levels (19k per
    // tile) tile 60 us against list 173; the 256x256 single-level frame (70
    // per tile) is faster on the tile kernel.
    // The group kernels are chosen only explicitly: the 8-lane one blends a
    // 314x208 frame alone faster than the tile kernel (176 against 200 us on
    // GB300) but costs more SM time, and the concurrent 8-frame sweep was
    // slower with it (1.236 against 1.222 ms).
    const int64_t sms = num_sms();
    const int group = strategy == MS_RASTER_GROUP8    ? 8
                      : strategy == MS_RASTER_GROUP16 ? 16
                      : strategy == MS_RASTER_GROUP32 ? 32
                                                      : 0;
    const bool auto_list = strategy == MS_RASTER_AUTO && tiles < sms;
    // a cap on the tile kernel's CTAs (frames blended side by side) keeps
    // the tile kernel: the list kernel cannot leave SMs to other frames; so
    // does a duplicate capacity below kListMeanMin entries per tile, which
    // rules the list kernel out before the lists are known
    const bool band = strategy == MS_RASTER_AUTO && !auto_list && max_ctas_per_sm == 0 &&
                      tiles < kListBandSms * sms &&
                      bins->dup_capacity >= (int64_t)kListMeanMin * tiles;
    const bool list = group > 0 || strategy == MS_RASTER_LIST || auto_list;
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
    a.seg_off = reinterpret_cast<uint32_t *>(w + L.seg_off);
    a.seg_len = reinterpret_cast<uint32_t *>(w + L.seg_len);
    a.ticket = reinterpret_cast<uint32_t *>(w + L.ticket);
    a.flags = reinterpret_cast<uint32_t *>(w + L.flags);
    a.tile_done = reinterpret_cast<uint32_t *>(w + L.tile_done);
    a.agg = reinterpret_cast<float4 *>(w + L.agg);
    a.agg2 = reinterpret_cast<uint2 *>(w + L.agg2);
    a.pre = reinterpret_cast<float4 *>(w + L.pre);
    a.pre2 = reinterpret_cast<uint2 *>(w + L.pre2);
    uint32_t *use_list = band ? reinterpret_cast<uint32_t *>(w + L.use_list) : nullptr;
    a.use_list = use_list;
    a.err = reinterpret_cast<unsigned long long *>(bins->counts) + kCntStatus;
    // the segmentation is the same for both kernels: the backward walks it
    // the tile kernel's ticket, flags and tile marks are zeroed by the first
    // kernel (the workspace and zero_bytes are 256-byte aligned)
    segment_offsets_kernel<<<1, 1024, 0, st>>>(bins->ranges, (int)tiles, (uint32_t)resident,
                                               a.seg_off, a.seg_len, reinterpret_cast<uint4 *>(w),
                                               list ? 0u : (uint32_t)(L.zero_bytes / 16),
                                               use_list, kListMeanMin, kListMeanMax);
    if (list || band) {
        ListArgs la;
        la.ranges = a.ranges;
        la.gidx = a.gidx;
        la.rec = a.rec;
        la.n_rec = a.n_rec;
        la.W = a.W;
        la.H = a.H;
        la.tiles_x = a.tiles_x;
        la.tiles = a.tiles;
        la.bg0 = a.bg0;
        la.bg1 = a.bg1;
        la.bg2 = a.bg2;
        la.image = a.image;
        la.final_t = a.final_t;
        la.n_contrib = a.n_contrib;
        la.n_eval = a.n_eval;
        la.seg_off = a.seg_off;
        la.seg_len = a.seg_len;
        la.pre = a.pre;
        la.rowmask = reinterpret_cast<uint32_t *>(w + L.rowmask);
        la.use_list = use_list;
        la.max_segs = (uint32_t)L.max_segs;
        la.err = a.err;
        if ((rc = cuda_check(cudaGetLastError(), "segment offsets launch"))) return rc;
        if (group > 0) return cuda_check(launch_raster_group(la, group, st), "raster group launch");
        if ((rc = cuda_check(launch_raster_list(la, st), "raster list launch"))) return rc;
        if (!band) return MS_OK;
    }
    raster_kernel<<<resident, kRasterThreads, kSmemBytes, st>>>(a);
    return cuda_check(cudaGetLastError(), "raster launches");
}

extern "C" int ms_raster_ex(const ms_proj_t *proj, const ms_bins_t *bins,
                            const ms_camera_t *cam, float *image, float *final_t,
                            uint32_t *n_contrib, uint32_t *n_eval, void *ws, size_t ws_bytes,
                            int strategy, void *stream) {
    return ms_raster_ex2(proj, bins, cam, image, final_t, n_contrib, n_eval, ws, ws_bytes,
                         strategy, 0, stream);
}

extern "C" int ms_raster(const ms_proj_t *proj, const ms_bins_t *bins, const ms_camera_t *cam,
                         float *image, float *final_t, uint32_t *n_contrib, uint32_t *n_eval,
                         void *ws, size_t ws_bytes, void *stream) {
    return ms_raster_ex(proj, bins, cam, image, final_t, n_contrib, n_eval, ws, ws_bytes,
                        MS_RASTER_AUTO, stream);
}

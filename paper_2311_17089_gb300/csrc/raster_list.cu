// Front-to-back blending with each pixel's list spread across the lanes of
// a warp (Sec. 3.1, Eq. 3 with incremental transmittance T_k).
//
// Coarse frames have few pixels and long tile lists (Sec. 3.2: at low
// resolution many splats fall on one tile).  One thread per pixel then
// leaves most of the GPU idle, and splitting the list across CTAs blends
// segments that the pixels never reach.  Here one warp blends one pixel,
// and a CTA the eight pixels of one half row of a tile:
//   - A first pass gives every entry of every tile list (its first
//     kMaskPrefix entries; past them the blend's own threads do it) a 32-bit
//     mask of the tile's half rows its alpha >= 1/255 level-set box (the
//     record's half extents) reaches.  Any entry whose bit is clear has
//     alpha below 1/255 at every pixel of that half row, so leaving it out
//     changes no result.
//     On coarse frames about a fifth of a tile's entries reach a given half
//     row, and a pixel that never terminates (an image edge with no surface
//     behind it) walks its whole list.
//   - The blend takes its tile's list in windows of kCullWin entries; the
//     masks and list indices of a window are read coalesced one window
//     ahead, and only the records of the entries reaching the CTA's half row
//     are copied (cp.async), packed in list order, while the window before
//     is blended.
//   - The packed entries are blended 32 per warp step: every lane evaluates
//     one Gaussian's alpha at the pixel centre with the tile kernel's FP32
//     operations (same power, same alpha >= 1/255 test, same 0.99 clamp),
//     and a warp-wide inclusive product scan of (1 - alpha) gives the
//     transmittance after every entry.
//   - The first accepted entry whose T falls below 1e-4 ends the pixel (it
//     is not blended); the entries before it add alpha_k T_{k-1} rgb_k into
//     per-lane partial colours, summed across the warp at the end.
// The result is the sequential blend up to FP32 rounding of the products
// (left-out entries have alpha = 0 and would multiply T by exactly 1).
// Nothing is speculative: a CTA walks its tile's list only until all of its
// pixels have terminated.  Windows never straddle a boundary of the frame's
// segmentation (segment_offsets_kernel): there a pixel still blending
// stores its (C, T) in the segment's prefix-state slot, which is where the
// backward starts each segment.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "raster_list.cuh"
#include "raster_ws.cuh"
#include "tma.cuh"

namespace msgs {
namespace {

constexpr float kListAlphaMax = 0.99f;
constexpr float kListTStop = 1e-4f;
constexpr uint32_t kFull = 0xffffffffu;

// List entries per window (kCullPerThread per thread) and the dynamic
// shared memory: two stages of up to kCullWin packed records, and each
// stage's list offsets within its window, and the per-warp counts.
constexpr int kCullPerThread = 2;
constexpr int kCullWin = 256 * kCullPerThread;
constexpr int kStageF4 = 3 * kCullWin;
constexpr int kPosOff = 2 * kStageF4 * 16;
constexpr int kCntOff = kPosOff + 2 * kCullWin * 2;
constexpr int kListSmem = kCntOff + kCullPerThread * kListPixelsPerCta * 4;
// Half extents of the row's pixel centres (8 x 1) plus the margin the tile
// kernel's per-warp culling uses for FP32 rounding: the record's half
// extents bound the exact alpha >= 1/255 level set, and the rounding of
// that bound and of the distances is below 1e-4 px at the largest image
// coordinates.
constexpr float kRowHalfX = 3.5f + 0.0625f;
constexpr float kRowHalfY = 0.0625f;

__device__ __forceinline__ float ex2_list(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Copy the record of Gaussian g (48 bytes) into a stage slot.
__device__ __forceinline__ void stage_copy(const ListArgs &a, float4 *dst, uint32_t g) {
    MS_DCHECK(g < a.n_rec, a.err);
    if (g >= a.n_rec) g = 0;  // unreachable unless binning reported an error
    const float4 *src = a.rec + 3 * (size_t)g;
    cp_async16(dst, src);
    cp_async16(dst + 1, src + 1);
    cp_async16(dst + 2, src + 2);
}

// End of the window that starts at p: kCullWin entries, cut at the next
// segment boundary (a multiple of L) and at the list's end.
__device__ __forceinline__ uint32_t window_end(uint32_t p, uint32_t L, uint32_t len) {
    return min(min(p + (uint32_t)kCullWin, (p / L + 1u) * L), len);
}

// Only the first kMaskPrefix entries of a tile's list get their mask from
// the mask pass: pixels seldom walk further (all-levels frames end within
// the first few percent of their long lists), and an entry the blend
// reaches beyond it has its mask formed by the blend's own thread.
constexpr uint32_t kMaskPrefix = 16384;

// Bit 2 r + h: the level-set box of the entry for Gaussian g, widened by
// the half extents of a half row, reaches the centre of the pixels (16 tx +
// 8 h + 0..7, 16 ty + r) of tile t = (tx, ty).  The FP32 expression is the
// one the blend assumes, the same for every half row.
__device__ __forceinline__ uint32_t row_mask_of(const ListArgs &a, uint32_t g, int t) {
    const int tx = t % a.tiles_x, ty = t / a.tiles_x;
    const float cx0 = (float)(tx * 16) + 4.0f, cx1 = (float)(tx * 16 + 8) + 4.0f;
    MS_DCHECK(g < a.n_rec, a.err);
    if (g >= a.n_rec) g = 0;  // unreachable unless binning reported an error
    // the centre (r0.xy) and the half extents (r2.zw)
    const float2 u = __ldg(reinterpret_cast<const float2 *>(a.rec + 3 * (size_t)g));
    const float2 x = __ldg(reinterpret_cast<const float2 *>(a.rec + 3 * (size_t)g + 2) + 1);
    const uint32_t h0 = fabsf(u.x - cx0) <= x.x + kRowHalfX;
    const uint32_t h1 = fabsf(u.x - cx1) <= x.x + kRowHalfX;
    uint32_t m = 0u;
#pragma unroll
    for (int r = 0; r < 16; r++) {
        const float cy = (float)(ty * 16 + r) + 0.5f;
        const uint32_t hit = fabsf(u.y - cy) <= x.y + kRowHalfY;
        m |= (hit & h0) << (2 * r) | (hit & h1) << (2 * r + 1);
    }
    return m;
}

// The half-row masks of the first kMaskPrefix entries of every tile list,
// one CTA per segment of the frame's segmentation (segment_offsets_kernel:
// tile t holds segments seg_off[t] .. seg_off[t + 1] - 1 of L entries
// each), so long lists are spread over many CTAs.  A frame the tile kernel
// blends (*a.use_list == 0) is skipped.
__global__ void __launch_bounds__(256) row_mask_kernel(ListArgs a) {
    const uint32_t c = blockIdx.x;
    if (a.use_list && *a.use_list == 0u) return;
    if (c >= a.seg_off[a.tiles]) return;
    int lo = 0, hi = a.tiles;  // seg_off[lo] <= c < seg_off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (a.seg_off[mid] <= c) lo = mid;
        else hi = mid;
    }
    const int t = lo;
    const uint32_t L = a.seg_len[0];
    const uint32_t beg = a.ranges[2 * t], end = a.ranges[2 * t + 1];
    const uint32_t s0 = beg + (c - a.seg_off[t]) * L;
    const uint32_t s1 = min(min(end, s0 + L), beg + kMaskPrefix);
    for (uint32_t e = s0 + threadIdx.x; e < s1; e += 256u)
        a.rowmask[e] = row_mask_of(a, __ldg(a.gidx + e), t);
}

// One pixel's blend state, held by every lane of its warp: T and the
// termination are warp-uniform, the colour sums and `last` per lane.
struct ListPixel {
    float T, c0, c1, c2;
    uint32_t last;   // per lane: 1 + position of the last entry it blended
    uint32_t evals;  // 1 + position of the entry that ended the pixel, or the list length
    bool live;
};

// Blend NQ warp steps of a stage's packed records i0 .. i0 + 32 NQ - 1
// (those below n) into the pixel at (fx, fy); the list position of packed
// record i is p0 + off[i].  Lanes past n load nothing.
template <int NQ>
__device__ __forceinline__ void blend_steps(const float4 *__restrict__ cur,
                                            const uint16_t *__restrict__ off, uint32_t i0,
                                            uint32_t n, uint32_t p0, float fx, float fy,
                                            uint32_t lane, ListPixel &s) {
    // phase 1: alpha, the lane-prefix product of (1 - alpha) and the whole
    // step's product, for every step (independent of T)
    float al[NQ], inc[NQ], tot[NQ], cr[NQ], cg[NQ], cb[NQ];
    uint32_t pos[NQ];
    uint32_t accm = 0u;
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        const uint32_t i = i0 + (uint32_t)q * 32u + lane;
        float4 r0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), r1 = r0, r2 = r0;
        uint32_t j = 0u;
        const bool valid = i < n;
        if (valid) {
            j = off[i];
            r0 = cur[3 * i];
            r1 = cur[3 * i + 1];
            r2 = cur[3 * i + 2];
        }
        // power * log2(e) = A dx^2 + B dx dy + C dy^2, in the tile kernel's
        // operation order
        const float dx = __fsub_rn(fx, r0.x), dy = __fsub_rn(fy, r0.y);
        const float u = __fmaf_rn(r0.w, dy, __fmul_rn(r0.z, dx));
        const float pw = __fmaf_rn(__fmul_rn(r1.x, dy), dy, __fmul_rn(dx, u));
        const bool acc = valid && pw <= 0.0f && pw >= r2.y;
        const float a1 = fminf(kListAlphaMax, __fmul_rn(r1.y, ex2_list(pw)));
        al[q] = acc ? a1 : 0.0f;
        accm |= (uint32_t)acc << q;
        cr[q] = r1.z;  // zero past n
        cg[q] = r1.w;
        cb[q] = r2.x;
        pos[q] = p0 + j + 1u;  // 1 + list position
    }
    // steps no lane accepts leave T and the colour unchanged
    if (!__any_sync(kFull, accm != 0u)) return;
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        float v = __fsub_rn(1.0f, al[q]);
#pragma unroll
        for (uint32_t o = 1; o < 32u; o <<= 1) {
            const float y = __shfl_up_sync(kFull, v, o);
            if (lane >= o) v = __fmul_rn(v, y);
        }
        inc[q] = v;
        tot[q] = __shfl_sync(kFull, v, 31);
    }
    // phase 2: T before each step, T after every entry, and the first step
    // with an accepted entry that would bring T below 1e-4 (T is monotone,
    // so later steps cannot end it sooner)
    float tin[NQ], ta[NQ];
    uint32_t tm[NQ];
    tin[0] = s.T;
#pragma unroll
    for (int q = 1; q < NQ; q++) tin[q] = __fmul_rn(tin[q - 1], tot[q - 1]);
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        ta[q] = __fmul_rn(tin[q], inc[q]);
        tm[q] = __ballot_sync(kFull, ((accm >> q) & 1u) && ta[q] < kListTStop);
    }
    int qt = NQ;
#pragma unroll
    for (int q = NQ - 1; q >= 0; q--)
        if (tm[q]) qt = q;
    uint32_t kt = 32u;
#pragma unroll
    for (int q = 0; q < NQ; q++)
        if (q == qt) kt = (uint32_t)__ffs(tm[q]) - 1u;
    // blend the entries before the end: alpha_k T_{k-1} rgb_k
    float tend = 0.0f;
    uint32_t pend = 0u;
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        if (q > qt) break;
        float tb = __shfl_up_sync(kFull, ta[q], 1);  // T before this lane's entry
        if (lane == 0) tb = tin[q];
        const bool bl = ((accm >> q) & 1u) && (q < qt || lane < kt);
        const float wgt = bl ? __fmul_rn(al[q], tb) : 0.0f;
        s.c0 = __fmaf_rn(wgt, cr[q], s.c0);
        s.c1 = __fmaf_rn(wgt, cg[q], s.c1);
        s.c2 = __fmaf_rn(wgt, cb[q], s.c2);
        if (bl) s.last = pos[q];
        if (q == qt) {
            tend = tb;
            pend = pos[q];
        }
    }
    if (qt < NQ) {
        s.T = __shfl_sync(kFull, tend, kt);  // T before the entry that ends the pixel
        s.evals = __shfl_sync(kFull, pend, kt);
        s.live = false;
    } else {
        s.T = __fmul_rn(tin[NQ - 1], tot[NQ - 1]);
    }
}

// The masks and list indices of window [p, q) for this thread's entries
// p + 256 k + threadIdx.x (a coalesced read); past the mask pass's prefix
// the thread forms the entry's mask itself.
__device__ __forceinline__ void load_window(const ListArgs &a, const uint32_t *__restrict__ gl,
                                            const uint32_t *__restrict__ ml, uint32_t p,
                                            uint32_t q, int t, uint32_t (&m)[kCullPerThread],
                                            uint32_t (&g)[kCullPerThread]) {
#pragma unroll
    for (int k = 0; k < kCullPerThread; k++) {
        const uint32_t e = p + (uint32_t)k * 256u + threadIdx.x;
        g[k] = e < q ? __ldg(gl + e) : 0u;
        m[k] = e >= q ? 0u : e < kMaskPrefix ? __ldg(ml + e) : row_mask_of(a, g[k], t);
    }
}

// Pack the entries of window [p, q) whose mask has bit b into a stage, in
// list order: their records by cp.async (one commit group), their offsets
// within the window into off.  The per-warp counts go through s_cnt; the
// barrier in between also counts the CTA's pixels still blending (`live`).
// Returns that count; n is the number of packed entries.
__device__ __forceinline__ int pack_window(const ListArgs &a, uint32_t b, uint32_t p, uint32_t q,
                                           const uint32_t (&m)[kCullPerThread],
                                           const uint32_t (&g)[kCullPerThread], float4 *stage,
                                           uint16_t *off, uint32_t *s_cnt, bool live,
                                           uint32_t &n) {
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    uint32_t bal[kCullPerThread];
#pragma unroll
    for (int k = 0; k < kCullPerThread; k++) {
        const uint32_t j = (uint32_t)k * 256u + threadIdx.x;
        bal[k] = __ballot_sync(kFull, p + j < q && ((m[k] >> b) & 1u));
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kCullPerThread; k++) s_cnt[k * 8 + w] = __popc(bal[k]);
    }
    const int nlive = __syncthreads_count(live);
    // window entry j = 256 k + 32 w + lane is slice 8 k + w; the slices'
    // counts, scanned
    uint32_t inc = lane < (uint32_t)(8 * kCullPerThread) ? s_cnt[lane] : 0u;
#pragma unroll
    for (uint32_t o = 1; o < 16u; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    n = __shfl_sync(kFull, inc, 8 * kCullPerThread - 1);
    if (nlive > 0) {
#pragma unroll
        for (int k = 0; k < kCullPerThread; k++) {
            const uint32_t base = __shfl_sync(kFull, inc, k * 8 + w) - __popc(bal[k]);
            if ((bal[k] >> lane) & 1u) {
                const uint32_t i = base + __popc(bal[k] & ((1u << lane) - 1u));
                stage_copy(a, &stage[3 * i], g[k]);
                off[i] = (uint16_t)((uint32_t)k * 256u + threadIdx.x);
            }
        }
    }
    cp_async_commit();
    return nlive;
}

// CTA b of tile t blends the pixels (8 (b & 1) + w, b >> 1) of the tile,
// w = 0..7 its warps, which is half row b of the tile's row mask.  Per
// window two CTA barriers: the packed records of the window have landed
// (and every warp is done with the stage the next window is packed into);
// the packing counts of the next window are in (with the count of pixels
// still blending).  The next window is packed and its records copied
// before this one is blended, and the masks and list indices of the window
// after it are loaded while this one is blended.
__global__ void __launch_bounds__(256, 4) raster_list_kernel(ListArgs a) {
    extern __shared__ __align__(16) unsigned char list_smem[];
    float4 *stage = reinterpret_cast<float4 *>(list_smem);
    uint16_t *soff = reinterpret_cast<uint16_t *>(list_smem + kPosOff);
    uint32_t *s_cnt = reinterpret_cast<uint32_t *>(list_smem + kCntOff);
    const uint32_t lane = threadIdx.x & 31u;
    const int w = threadIdx.x >> 5;
    const int t = blockIdx.x / kListCtasPerTile, b = blockIdx.x % kListCtasPerTile;
    if (t >= a.tiles) return;
    if (a.use_list && *a.use_list == 0u) return;  // the tile kernel blends this frame
    const int tx = t % a.tiles_x, ty = t / a.tiles_x;
    const int lx = (b & 1) * 8 + w, ly = b >> 1;
    const int px = tx * 16 + lx, py = ty * 16 + ly;
    if (tx * 16 + (b & 1) * 8 >= a.W || py >= a.H) return;  // no pixel of this CTA is inside
    const bool inside = px < a.W;
    const uint32_t beg = a.ranges[2 * t], end = a.ranges[2 * t + 1];
    const uint32_t len = end > beg ? end - beg : 0u;
    const uint32_t L = a.seg_len[0];
    const uint32_t seg0 = a.seg_off[t];
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    ListPixel px_state = {1.0f, 0.0f, 0.0f, 0.0f, 0u, len, inside};
    const uint32_t *gl = a.gidx + beg;
    const uint32_t *ml = a.rowmask + beg;
    // windows [p0, p1) (packed, being blended), [p1, p2) (packed next), [p2, p3)
    uint32_t p0 = 0u, p1 = window_end(0u, L, len), p2 = window_end(p1, L, len);
    uint32_t m[kCullPerThread], g[kCullPerThread];
    load_window(a, gl, ml, p0, p1, t, m, g);
    uint32_t n_cur = 0u, n_next = 0u;
    pack_window(a, (uint32_t)b, p0, p1, m, g, stage, soff, s_cnt, true, n_cur);
    load_window(a, gl, ml, p1, p2, t, m, g);
    for (uint32_t wi = 0;; wi++) {
        const uint32_t sb = wi & 1u;
        // this thread's copies of window wi have landed; after the barrier
        // every thread's have, and every warp is done with window wi - 1
        cp_async_wait<0>();
        __syncthreads();
        if (p0 >= p1) break;  // the list is walked to its end
        const uint32_t sn = sb ^ 1u;
        if (pack_window(a, (uint32_t)b, p1, p2, m, g, stage + sn * kStageF4, soff + sn * kCullWin,
                        s_cnt, px_state.live, n_next) == 0)
            break;  // every pixel has terminated
        const uint32_t p3 = window_end(p2, L, len);
        load_window(a, gl, ml, p2, p3, t, m, g);
        // blend the window's packed entries two warp steps of 32 at a time
        // (their product scans side by side; 3 or 4 at a time needed more
        // registers than four CTAs per SM leave and were slower)
        const float4 *cur = stage + sb * kStageF4;
        const uint16_t *off = soff + sb * kCullWin;
        for (uint32_t i0 = 0; px_state.live && i0 < n_cur; i0 += 64u) {
            if (n_cur - i0 > 32u) blend_steps<2>(cur, off, i0, n_cur, p0, fx, fy, lane, px_state);
            else blend_steps<1>(cur, off, i0, n_cur, p0, fx, fy, lane, px_state);
        }
        // a window ending on a segment boundary: the state after segment
        // p1 / L - 1, where the backward starts the next segment; the tile's
        // last segment stores none
        if (px_state.live && p1 < len && p1 % L == 0u) {
            const float s0 = warp_sum(px_state.c0), s1 = warp_sum(px_state.c1),
                        s2 = warp_sum(px_state.c2);
            if (lane == 0)
                a.pre[(size_t)(seg0 + p1 / L - 1u) * kRasterThreads + fwd_index(lx, ly)] =
                    make_float4(s0, s1, s2, px_state.T);
        }
        n_cur = n_next;
        p0 = p1;
        p1 = p2;
        p2 = p3;
    }
    cp_async_wait<0>();  // no copy outlives the CTA
    if (!inside) return;
    const float C0 = warp_sum(px_state.c0), C1 = warp_sum(px_state.c1),
                C2 = warp_sum(px_state.c2);
    const float T = px_state.T;
    // 1 + position of the last blended entry
    const uint32_t last = __reduce_max_sync(kFull, px_state.last);
    if (lane == 0) {
        const size_t p = (size_t)py * a.W + px, plane = (size_t)a.W * a.H;
        a.image[p] = fmaf(T, a.bg0, C0);
        a.image[plane + p] = fmaf(T, a.bg1, C1);
        a.image[2 * plane + p] = fmaf(T, a.bg2, C2);
        if (a.final_t) a.final_t[p] = T;
        if (a.n_contrib) a.n_contrib[p] = last;
        if (a.n_eval) a.n_eval[p] = px_state.evals;
    }
}

}  // namespace

cudaError_t launch_raster_list(const ListArgs &a, cudaStream_t st) {
    if (ensure_smem_attr(reinterpret_cast<const void *>(raster_list_kernel), kListSmem))
        return cudaErrorInvalidValue;
    row_mask_kernel<<<(unsigned)a.max_segs, 256, 0, st>>>(a);
    const int64_t grid = (int64_t)a.tiles * kListCtasPerTile;
    raster_list_kernel<<<(unsigned)grid, 256, kListSmem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace msgs

// Front-to-back blending with each pixel's list spread across the lanes of
// a warp (Sec. 3.1, Eq. 3 with incremental transmittance T_k).
//
// Coarse frames have few pixels and long tile lists (Sec. 3.2: at low
// resolution many splats fall on one tile).  One thread per pixel then
// leaves most of the GPU idle, and splitting the list across CTAs blends
// segments that the pixels never reach.  Here one warp blends one pixel:
// lane j takes entry g0 + j of the tile's list, so a warp step covers 32
// entries of that pixel's list at once.
//   - Every lane evaluates its Gaussian's alpha at the pixel centre with
//     the tile kernel's FP32 operations (same power, same alpha >= 1/255
//     test, same 0.99 clamp).
//   - A warp-wide inclusive product scan of (1 - alpha) gives the
//     transmittance after every entry: T_k = T_in prod_{j <= k}(1 - alpha_j).
//   - The first accepted entry whose T_k falls below 1e-4 ends the pixel
//     (it is not blended); the entries before it add alpha_k T_{k-1} rgb_k
//     into per-lane partial colours, summed across the warp at the end.
//   - A warp takes its entries in sub-batches of four such steps; one vote
//     per sub-batch skips the scans and the blend of a sub-batch in which
//     no lane accepts its entry (a pixel far down a list in a sparse
//     region sees many).
// The result is the sequential blend up to FP32 rounding of the products.
// Nothing is speculative: a CTA walks its tile's list only until all of its
// pixels have terminated.  At every boundary of the frame's segmentation
// (segment_offsets_kernel), a pixel still blending stores its (C, T) in the
// segment's prefix-state slot, which is where the backward starts each
// segment.
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

// CTA b of tile t blends the pixels (8 (b & 1) + w, b >> 1) of the tile,
// w = 0..7 its warps.  The CTA stages the tile's list in sub-batches of
// kListBatch records in a ring of kListStages shared-memory buffers: warps
// 0-3 copy each record of a sub-batch with cp.async, kListStages - 1
// sub-batches ahead of the one being blended, and load the list indices one
// sub-batch further ahead still, so a record costs one global round trip,
// hidden behind the blending of the sub-batches before it.  Each record is
// gathered once per CTA, not once per warp.  One barrier per sub-batch; a
// pixel that has terminated leaves its warp idle until every pixel of the
// CTA has.
constexpr int kListBatch = 128;
constexpr int kListSteps = kListBatch / 32;
constexpr int kListStages = 4;

// Copy the record of Gaussian g (48 bytes) into a stage slot.
__device__ __forceinline__ void stage_copy(const ListArgs &a, float4 *dst, uint32_t g) {
    MS_DCHECK(g < a.n_rec, a.err);
    if (g >= a.n_rec) g = 0;  // unreachable unless binning reported an error
    const float4 *src = a.rec + 3 * (size_t)g;
    cp_async16(dst, src);
    cp_async16(dst + 1, src + 1);
    cp_async16(dst + 2, src + 2);
}

// A slot past the list's end: a zero record (no colour; its alpha is
// masked by the position test).
__device__ __forceinline__ void stage_zero(float4 *dst) {
    const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    dst[0] = z;
    dst[1] = z;
    dst[2] = z;
}

__global__ void __launch_bounds__(256) raster_list_kernel(ListArgs a) {
    __shared__ float4 buf[kListStages][3 * kListBatch];
    const uint32_t lane = threadIdx.x & 31u;
    const int w = threadIdx.x >> 5;
    const int t = blockIdx.x / kListCtasPerTile, b = blockIdx.x % kListCtasPerTile;
    if (t >= a.tiles) return;
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
    float T = 1.0f, c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
    uint32_t last = 0u;  // per lane: 1 + position of the last entry it blended
    uint32_t evals = len;
    bool live = inside;
    const uint32_t *gl = a.gidx + beg;
    const bool loader = w < kListBatch / 32;
    const uint32_t slot = (uint32_t)w * 32u + lane;  // record of a sub-batch this thread gathers
    const uint32_t nsb = (len + kListBatch - 1) / kListBatch;
    // prologue: stages 0 .. kListStages - 2 in flight, indices of the next
    uint32_t gn = 0u;
    if (loader) {
#pragma unroll
        for (int s = 0; s < kListStages - 1; s++) {
            const uint32_t pos = (uint32_t)s * kListBatch + slot;
            if (pos < len) stage_copy(a, &buf[s][3 * slot], __ldg(gl + pos));
            else stage_zero(&buf[s][3 * slot]);
            cp_async_commit();
        }
        const uint32_t pos = (uint32_t)(kListStages - 1) * kListBatch + slot;
        if (pos < len) gn = __ldg(gl + pos);
    }
    for (uint32_t sb = 0;; sb++) {
        // this thread's copies of sub-batch sb have landed; after the barrier
        // every thread's have, and every warp is done with sub-batch sb - 1
        if (loader) cp_async_wait<kListStages - 2>();
        if (__syncthreads_count(live) == 0 || sb >= nsb) break;
        if (loader) {
            // sub-batch sb + stages - 1 into the stage sub-batch sb - 1 used;
            // a group is committed even when empty, so the counting holds
            const uint32_t nsb2 = sb + kListStages - 1;
            const uint32_t pos = nsb2 * kListBatch + slot;
            if (pos < len) stage_copy(a, &buf[nsb2 % kListStages][3 * slot], gn);
            else stage_zero(&buf[nsb2 % kListStages][3 * slot]);
            cp_async_commit();
            const uint32_t pos2 = pos + kListBatch;
            if (pos2 < len) gn = __ldg(gl + pos2);
        }
        const uint32_t bi = sb % kListStages, base = sb * kListBatch;
        if (live) {
            // phase 1: alpha, the lane-prefix product of (1 - alpha) and the
            // whole step's product, for every step of the sub-batch
            // (independent of T)
            const uint32_t nv = len - base;  // entries of the list in this sub-batch
            float al[kListSteps], inc[kListSteps], tot[kListSteps];
            float cr[kListSteps], cg[kListSteps], cb[kListSteps];
            uint32_t accm = 0u;
#pragma unroll
            for (int q = 0; q < kListSteps; q++) {
                const uint32_t i = (uint32_t)q * 32u + lane;
                const float4 r0 = buf[bi][3 * i], r1 = buf[bi][3 * i + 1], r2 = buf[bi][3 * i + 2];
                // power * log2(e) = A dx^2 + B dx dy + C dy^2, in the tile
                // kernel's operation order
                const float dx = __fsub_rn(fx, r0.x), dy = __fsub_rn(fy, r0.y);
                const float u = __fmaf_rn(r0.w, dy, __fmul_rn(r0.z, dx));
                const float pw = __fmaf_rn(__fmul_rn(r1.x, dy), dy, __fmul_rn(dx, u));
                const bool acc = i < nv && pw <= 0.0f && pw >= r2.y;
                const float a1 = fminf(kListAlphaMax, __fmul_rn(r1.y, ex2_list(pw)));
                al[q] = acc ? a1 : 0.0f;
                accm |= (uint32_t)acc << q;
                cr[q] = r1.z;  // slots past the list's end hold zeros
                cg[q] = r1.w;
                cb[q] = r2.x;
            }
            // a sub-batch no lane accepts (common for pixels far down a list
            // in a sparse region) leaves T and the colour unchanged
            if (__any_sync(kFull, accm != 0u)) {
#pragma unroll
                for (int q = 0; q < kListSteps; q++) {
                    float v = __fsub_rn(1.0f, al[q]);
#pragma unroll
                    for (uint32_t o = 1; o < 32u; o <<= 1) {
                        const float y = __shfl_up_sync(kFull, v, o);
                        if (lane >= o) v = __fmul_rn(v, y);
                    }
                    inc[q] = v;
                    tot[q] = __shfl_sync(kFull, v, 31);
                }
                // phase 2: T before each step, T after every entry, and the
                // first step with an accepted entry that would bring T below
                // 1e-4 (T is monotone, so later steps cannot end it sooner)
                float tin[kListSteps], ta[kListSteps];
                uint32_t tm[kListSteps];
                tin[0] = T;
#pragma unroll
                for (int q = 1; q < kListSteps; q++) tin[q] = __fmul_rn(tin[q - 1], tot[q - 1]);
#pragma unroll
                for (int q = 0; q < kListSteps; q++) {
                    ta[q] = __fmul_rn(tin[q], inc[q]);
                    tm[q] = __ballot_sync(kFull, ((accm >> q) & 1u) && ta[q] < kListTStop);
                }
                int qt = kListSteps;
#pragma unroll
                for (int q = kListSteps - 1; q >= 0; q--)
                    if (tm[q]) qt = q;
                uint32_t kt = 32u;
#pragma unroll
                for (int q = 0; q < kListSteps; q++)
                    if (q == qt) kt = (uint32_t)__ffs(tm[q]) - 1u;
                // blend the entries before the end: alpha_k T_{k-1} rgb_k
                float tend = 0.0f;
#pragma unroll
                for (int q = 0; q < kListSteps; q++) {
                    if (q > qt) break;
                    float tb = __shfl_up_sync(kFull, ta[q], 1);  // T before this lane's entry
                    if (lane == 0) tb = tin[q];
                    const bool bl = ((accm >> q) & 1u) && (q < qt || lane < kt);
                    const float wgt = bl ? __fmul_rn(al[q], tb) : 0.0f;
                    c0 = __fmaf_rn(wgt, cr[q], c0);
                    c1 = __fmaf_rn(wgt, cg[q], c1);
                    c2 = __fmaf_rn(wgt, cb[q], c2);
                    if (bl) last = base + (uint32_t)q * 32u + lane + 1u;
                    if (q == qt) tend = tb;
                }
                if (qt < kListSteps) {
                    T = __shfl_sync(kFull, tend, kt);  // T before the entry that ends the pixel
                    evals = base + (uint32_t)qt * 32u + kt + 1u;
                    live = false;
                } else {
                    T = __fmul_rn(tin[kListSteps - 1], tot[kListSteps - 1]);
                }
            }
            // segment boundaries fall on sub-batch ends (L is a multiple of
            // the sub-batch): the state after segment (base + batch) / L - 1,
            // where the backward starts the next segment; the tile's last
            // segment stores none
            const uint32_t next = base + kListBatch;
            if (live && next < len && next % L == 0u) {
                const float s0 = warp_sum(c0), s1 = warp_sum(c1), s2 = warp_sum(c2);
                if (lane == 0)
                    a.pre[(size_t)(seg0 + next / L - 1u) * kRasterThreads + fwd_index(lx, ly)] =
                        make_float4(s0, s1, s2, T);
            }
        }
    }
    if (loader) cp_async_wait<0>();  // no copy outlives the CTA
    if (!inside) return;
    const float C0 = warp_sum(c0), C1 = warp_sum(c1), C2 = warp_sum(c2);
    last = __reduce_max_sync(kFull, last);  // 1 + position of the last blended entry
    if (lane == 0) {
        const size_t p = (size_t)py * a.W + px, plane = (size_t)a.W * a.H;
        a.image[p] = fmaf(T, a.bg0, C0);
        a.image[plane + p] = fmaf(T, a.bg1, C1);
        a.image[2 * plane + p] = fmaf(T, a.bg2, C2);
        if (a.final_t) a.final_t[p] = T;
        if (a.n_contrib) a.n_contrib[p] = last;
        if (a.n_eval) a.n_eval[p] = evals;
    }
}

}  // namespace

cudaError_t launch_raster_list(const ListArgs &a, cudaStream_t st) {
    const int64_t grid = (int64_t)a.tiles * kListCtasPerTile;
    raster_list_kernel<<<(unsigned)grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace msgs

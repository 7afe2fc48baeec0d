// Front-to-back blending with each pixel's list spread over a group of G
// lanes (Sec. 3.1, Eq. 3 with incremental transmittance T_k): the list
// kernel for frames with few tiles and long lists (Sec. 3.2: at low
// resolution many splats fall on one tile, and each pixel's sequential sum
// grows).
//
// A warp holds 32 / G pixels side by side in a tile row, G lanes each.  A
// step covers the next G * 4 entries of the tile's list for every pixel of
// the warp: lane j of a group takes the 4 consecutive entries j*4 .. j*4+3
// of the step and, in list order,
//   - evaluates alpha_k at its pixel centre with the tile kernel's FP32
//     operations (same power, same alpha >= 1/255 test, same 0.99 clamp),
//   - forms its local transmittance P_k = prod_{i <= k} (1 - alpha_i) and
//     its local colour sum c = sum_k alpha_k P_{k-1} rgb_k (from T = 1);
// a product scan over the group's lanes gives the transmittance T_j in
// front of each lane, T_j = T prod_{i < j} P_i.  The first accepted entry
// whose T_j P_k falls below 1e-4 ends the pixel (it is not blended); the
// lanes before it add T_j c to their partial colours, the lane holding it
// re-sums its entries before that one, and the partial colours are summed
// over the group at the end.  One scan per 4 G entries (the lane-per-entry
// form needs one per G), and the G lanes of a pixel read G different
// records that every pixel of the warp shares, so a shared-memory load
// serves 32 / G pixels at once.
//
// All warps of a CTA walk one tile's list together: 256 records per
// sub-batch, one per thread, copied by cp.async into a ring of four
// stages (three sub-batches in flight), the list indices loaded two
// sub-batches further ahead.  The
// records of a step are laid out so that the G lanes of a group read
// consecutive 16-byte slots.  Nothing is blended speculatively beyond the
// end of a step: a CTA walks its tile's list only until all of its pixels
// have terminated.  At every boundary of the frame's segmentation
// (segment_offsets_kernel), a pixel still blending stores its (C, T) in the
// segment's prefix-state slot, where the backward starts the next segment.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "raster_list.cuh"
#include "raster_ws.cuh"
#include "tma.cuh"

namespace msgs {
namespace {

constexpr float kGAlphaMax = 0.99f;
constexpr float kGTStop = 1e-4f;
constexpr uint32_t kGFull = 0xffffffffu;
constexpr int kGM = 4;          // consecutive entries per lane per step
constexpr int kGBatch = 256;    // records per staged sub-batch, one per thread
constexpr int kGStages = 4;     // ring depth
constexpr int kGIdxAhead = 2;   // sub-batches of list indices held beyond the ring

__device__ __forceinline__ float ex2_group(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int G>
struct GroupShape {
    static constexpr int kPixPerWarp = 32 / G;
    static constexpr int kPixPerCta = 8 * kPixPerWarp;
    static constexpr int kCtasPerTile = 256 / kPixPerCta;
    static constexpr int kStep = G * kGM;  // list entries per step
    static constexpr int kSteps = kGBatch / kStep;
};

// Slot of sub-batch entry e: entry j*4 + k of a step goes to k * G + j, so
// the lanes of a group reading their k-th entries touch consecutive slots.
template <int G>
__device__ __forceinline__ uint32_t group_slot(uint32_t e) {
    constexpr uint32_t S = GroupShape<G>::kStep;
    const uint32_t s = e / S, r = e % S;
    return s * S + (r % kGM) * G + r / kGM;
}

template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kGFull, v, o, G);
    return v;
}

// alpha of one staged record at pixel centre (fx, fy): power * log2(e) =
// A dx^2 + B dx dy + C dy^2 in the tile kernel's operation order, accepted
// when 0 >= power >= thr (slots past the list's end hold thr = +inf and are
// never accepted), clamped to 0.99; 0 when not accepted.
__device__ __forceinline__ float entry_alpha(const float4 r0, const float4 r1, float thr,
                                             float fx, float fy, bool live, bool &ok) {
    const float dx = __fsub_rn(fx, r0.x), dy = __fsub_rn(fy, r0.y);
    const float u = __fmaf_rn(r0.w, dy, __fmul_rn(r0.z, dx));
    const float pw = __fmaf_rn(__fmul_rn(r1.x, dy), dy, __fmul_rn(dx, u));
    ok = live && pw <= 0.0f && pw >= thr;
    return ok ? fminf(kGAlphaMax, __fmul_rn(r1.y, ex2_group(pw))) : 0.0f;
}

template <int G>
__global__ void __launch_bounds__(256, 4) raster_group_kernel(ListArgs a) {
    using S = GroupShape<G>;
    // three planes per stage: (ux, uy, A, B), (C, opacity, r, g), (b, thr, ex, ey)
    __shared__ float4 buf[kGStages][3][kGBatch];
    const uint32_t lane = threadIdx.x & 31u;
    const int w = threadIdx.x >> 5;
    const uint32_t j = lane % G;                 // lane within the pixel's group
    const uint32_t gbase = lane - j;             // first lane of the group
    const uint32_t gmask = (G == 32) ? kGFull : (((1u << G) - 1u) << gbase);
    const int t = blockIdx.x / S::kCtasPerTile, b = blockIdx.x % S::kCtasPerTile;
    if (t >= a.tiles) return;
    const int tx = t % a.tiles_x, ty = t / a.tiles_x;
    const int p0 = b * S::kPixPerCta;            // first tile pixel of the CTA
    // the CTA's first pixel has its smallest x and y (it holds part of one
    // row, or whole rows): if that one is outside the image, all are
    if (tx * 16 + (p0 & 15) >= a.W || ty * 16 + (p0 >> 4) >= a.H) return;
    const int p = p0 + w * S::kPixPerWarp + (int)(lane / G);
    const int lx = p & 15, ly = p >> 4;
    const int px = tx * 16 + lx, py = ty * 16 + ly;
    const bool inside = px < a.W && py < a.H;
    const uint32_t beg = a.ranges[2 * t], end = a.ranges[2 * t + 1];
    const uint32_t len = end > beg ? end - beg : 0u;
    const uint32_t L = a.seg_len[0];
    const uint32_t seg0 = a.seg_off[t];
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    float T = 1.0f;                       // group-uniform
    float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;  // this lane's part of the pixel colour
    uint32_t last = 0u;                   // 1 + position of the last entry this lane blended
    uint32_t evals = len;
    bool live = inside;                   // group-uniform
    const uint32_t *gl = a.gidx + beg;
    const uint32_t nsb = (len + kGBatch - 1) / kGBatch;
    const uint32_t my_slot = group_slot<G>(threadIdx.x);
    uint32_t nextb = L;  // the next segment boundary (a multiple of L)

    auto stage = [&](int s, uint32_t sb, uint32_t g) {
        const uint32_t pos = sb * kGBatch + threadIdx.x;
        if (pos < len) {
            MS_DCHECK(g < a.n_rec, a.err);
            if (g >= a.n_rec) g = 0;  // unreachable unless binning reported an error
            const float4 *src = a.rec + 3 * (size_t)g;
            cp_async16(&buf[s][0][my_slot], src);
            cp_async16(&buf[s][1][my_slot], src + 1);
            cp_async16(&buf[s][2][my_slot], src + 2);
        } else {
            // past the list's end: no colour, and a threshold no power reaches
            const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            buf[s][0][my_slot] = z;
            buf[s][1][my_slot] = z;
            buf[s][2][my_slot] = make_float4(0.0f, __int_as_float(0x7f800000), 0.0f, 0.0f);
        }
    };
    // prologue: sub-batches 0 .. kGStages - 2 in flight, and the indices of
    // the kGIdxAhead sub-batches after them in registers
#pragma unroll
    for (int s = 0; s < kGStages - 1; s++) {
        const uint32_t pos = (uint32_t)s * kGBatch + threadIdx.x;
        stage(s, (uint32_t)s, pos < len ? __ldg(gl + pos) : 0u);
        cp_async_commit();
    }
    uint32_t gn[kGIdxAhead];
#pragma unroll
    for (int i = 0; i < kGIdxAhead; i++) {
        const uint32_t pos = (uint32_t)(kGStages - 1 + i) * kGBatch + threadIdx.x;
        gn[i] = pos < len ? __ldg(gl + pos) : 0u;
    }
    for (uint32_t sb = 0;; sb++) {
        // this thread's copies of sub-batch sb have landed; after the barrier
        // every thread's have, and every warp is done with sub-batch sb - 1
        cp_async_wait<kGStages - 2>();
        if (__syncthreads_count(live) == 0 || sb >= nsb) break;
        {
            // sub-batch sb + stages - 1 into the stage sub-batch sb - 1 used;
            // a group is committed even when empty, so the counting holds
            const uint32_t nb = sb + kGStages - 1;
            stage((int)(nb % kGStages), nb, gn[0]);
            cp_async_commit();
#pragma unroll
            for (int i = 0; i + 1 < kGIdxAhead; i++) gn[i] = gn[i + 1];
            const uint32_t pos2 = (nb + kGIdxAhead) * kGBatch + threadIdx.x;
            gn[kGIdxAhead - 1] = pos2 < len ? __ldg(gl + pos2) : 0u;
        }
        const int bi = (int)(sb % kGStages);
        if (!__any_sync(kGFull, live)) continue;
#pragma unroll 1
        for (int st = 0; st < S::kSteps; st++) {
            const uint32_t base = sb * kGBatch + (uint32_t)st * S::kStep;  // warp-uniform
            if (base >= len) break;
            // local pass over this lane's 4 entries (from T = 1)
            float P[kGM];
            float lr = 0.0f, lg = 0.0f, lb = 0.0f, Pc = 1.0f;
            uint32_t acc = 0u;
#pragma unroll
            for (int k = 0; k < kGM; k++) {
                const uint32_t slot = (uint32_t)st * S::kStep + (uint32_t)k * G + j;
                const float4 r1 = buf[bi][1][slot];
                const float4 r2 = buf[bi][2][slot];
                bool ok;
                const float a1 = entry_alpha(buf[bi][0][slot], r1, r2.y, fx, fy, live, ok);
                const float wgt = __fmul_rn(a1, Pc);
                lr = __fmaf_rn(wgt, r1.z, lr);
                lg = __fmaf_rn(wgt, r1.w, lg);
                lb = __fmaf_rn(wgt, r2.x, lb);
                Pc = __fmaf_rn(-a1, Pc, Pc);
                P[k] = Pc;
                acc |= (uint32_t)ok << k;
            }
            // a step no lane of the warp accepts an entry in leaves T and the
            // colour unchanged
            if (__any_sync(kGFull, acc != 0u)) {
                // transmittance in front of this lane: T times the product of
                // the group's earlier lanes' local transmittances
                float inc = Pc;
#pragma unroll
                for (int o = 1; o < G; o <<= 1) {
                    const float y = __shfl_up_sync(kGFull, inc, o, G);
                    if (j >= (uint32_t)o) inc = __fmul_rn(inc, y);
                }
                float ex = __shfl_up_sync(kGFull, inc, 1, G);
                if (j == 0) ex = 1.0f;
                const float tot = __shfl_sync(kGFull, inc, G - 1, G);
                const float Tl = __fmul_rn(T, ex);
                // the first accepted entry of this lane that would bring T
                // below 1e-4 (T is monotone along the lane)
                uint32_t tk = kGM;
#pragma unroll
                for (int k = kGM - 1; k >= 0; k--)
                    if (((acc >> k) & 1u) && __fmul_rn(Tl, P[k]) < kGTStop) tk = (uint32_t)k;
                const uint32_t gt = (__ballot_sync(kGFull, tk < kGM) & gmask) >> gbase;
                const uint32_t js = gt ? (uint32_t)__ffs(gt) - 1u : (uint32_t)G;
                if (j < js) {
                    c0 = __fmaf_rn(Tl, lr, c0);
                    c1 = __fmaf_rn(Tl, lg, c1);
                    c2 = __fmaf_rn(Tl, lb, c2);
                    if (acc) last = base + j * kGM + (31u - (uint32_t)__clz(acc)) + 1u;
                } else if (j == js) {
                    // the entries before the one that ends the pixel, with
                    // alpha formed again by the same operations
                    float pr = 0.0f, pg = 0.0f, pb = 0.0f;
#pragma unroll
                    for (int k = 0; k < kGM; k++) {
                        if ((uint32_t)k < tk) {
                            const uint32_t slot = (uint32_t)st * S::kStep + (uint32_t)k * G + j;
                            const float4 r1 = buf[bi][1][slot];
                            bool ok;
                            const float a1 = entry_alpha(buf[bi][0][slot], r1,
                                                         buf[bi][2][slot].y, fx, fy, true, ok);
                            const float wgt = __fmul_rn(a1, k ? P[k - 1] : 1.0f);
                            pr = __fmaf_rn(wgt, r1.z, pr);
                            pg = __fmaf_rn(wgt, r1.w, pg);
                            pb = __fmaf_rn(wgt, buf[bi][2][slot].x, pb);
                        }
                    }
                    c0 = __fmaf_rn(Tl, pr, c0);
                    c1 = __fmaf_rn(Tl, pg, c1);
                    c2 = __fmaf_rn(Tl, pb, c2);
                    const uint32_t am = acc & ((1u << tk) - 1u);
                    if (am) last = base + j * kGM + (31u - (uint32_t)__clz(am)) + 1u;
                }
                // T before the entry that ends the pixel (lane js), else
                // after the whole step
                float tend = Tl;
#pragma unroll
                for (int k = 0; k < kGM; k++)
                    if ((uint32_t)k + 1u == tk) tend = __fmul_rn(Tl, P[k]);
                const uint32_t src = gbase + (js < (uint32_t)G ? js : 0u);
                const float te = __shfl_sync(kGFull, tend, src);
                const uint32_t tks = __shfl_sync(kGFull, tk, src);
                if (live) {
                    if (js < (uint32_t)G) {
                        T = te;
                        evals = base + js * kGM + tks + 1u;
                        live = false;
                    } else {
                        T = __fmul_rn(T, tot);
                    }
                }
            }
            // segment boundaries fall on step ends (L is a multiple of 128,
            // a step at most 128 entries): the state after segment
            // next / L - 1, where the backward starts the next segment; the
            // tile's last segment stores none
            const uint32_t next = base + S::kStep;
            if (next == nextb) {
                nextb += L;
                if (next < len) {
                    const float s0 = group_sum<G>(c0), s1 = group_sum<G>(c1);
                    const float s2 = group_sum<G>(c2);
                    if (live && j == 0)
                        a.pre[(size_t)(seg0 + next / L - 1u) * kRasterThreads +
                              fwd_index(lx, ly)] = make_float4(s0, s1, s2, T);
                }
            }
            if (!__any_sync(kGFull, live)) break;
        }
    }
    cp_async_wait<0>();  // no copy outlives the CTA
    const float C0 = group_sum<G>(c0), C1 = group_sum<G>(c1), C2 = group_sum<G>(c2);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) last = max(last, __shfl_xor_sync(kGFull, last, o, G));
    if (inside && j == 0) {
        const size_t pp = (size_t)py * a.W + px, plane = (size_t)a.W * a.H;
        a.image[pp] = fmaf(T, a.bg0, C0);
        a.image[plane + pp] = fmaf(T, a.bg1, C1);
        a.image[2 * plane + pp] = fmaf(T, a.bg2, C2);
        if (a.final_t) a.final_t[pp] = T;
        if (a.n_contrib) a.n_contrib[pp] = last;
        if (a.n_eval) a.n_eval[pp] = evals;
    }
}

template <int G>
cudaError_t launch_group(const ListArgs &a, cudaStream_t st) {
    const int64_t grid = (int64_t)a.tiles * GroupShape<G>::kCtasPerTile;
    raster_group_kernel<G><<<(unsigned)grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_raster_group(const ListArgs &a, int group, cudaStream_t st) {
    switch (group) {
        case 8: return launch_group<8>(a, st);
        case 16: return launch_group<16>(a, st);
        case 32: return launch_group<32>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace msgs

// Gradient of the rendered image with respect to the scene parameters
// (the back-propagation a multi-scale training step runs, Sec. 4.1
// "Multi-Scale Training").
//
// raster_bwd_kernel: the forward cut every tile's list into segments and
// left, for each segment, the exact per-pixel state (C, T) after it.  The
// backward therefore treats segments independently: a CTA takes a segment
// by ticket, starts each pixel from the state the forward reached before
// it, and walks the segment front to back up to the pixel's last
// contributor, recomputing each alpha with exactly the forward's FP32
// operations (so the same Gaussians contribute).  With F_k the colour
// accumulated up to and including Gaussian k and C the final pixel colour,
// the colour behind k is R_k = C - F_k, and
//   dC/dalpha_k = T_k c_k - R_k / (1 - alpha_k),  dC/dc_k = alpha_k T_k.
// alpha = sigma e^power (below the 0.99 clamp) gives dsigma and dpower, and
// power = -(a dx^2 + c dy^2)/2 - b dx dy gives the centre and conic
// gradients.  Per record, a warp reduce-scatters its 32 pixels' nine values
// (12 shuffles; nine lanes end up owning one full sum each), the owners add
// them to shared memory, and the CTA adds each record's sums to the
// per-Gaussian 2D gradient with one atomic per value.
//
// project_bwd_kernel: per Gaussian, the chain rule from (centre, conic,
// opacity, colour) through V' = V + 0.3 I, V = J W Sigma W^T J^T, the
// Jacobian, Sigma = R diag(e^s)^2 R^T, the normalised quaternion and the
// SH colour (basis derivatives in closed form, projected on the sphere).
#include <cuda_runtime.h>

#include <atomic>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "f32x2.cuh"
#include "raster_ws.cuh"

namespace msgs {

constexpr int kBwdThreads = 128;  // two pixels per thread
constexpr int kBwdBatch = 256;
constexpr int kG2 = 9;  // dux, duy, da, db, dc, dsigma, dr, dg, db
constexpr float kInvConicA = -1.3862943611198906f;  // 1 / (-log2(e)/2)
constexpr float kInvConicB = -0.6931471805599453f;  // 1 / (-log2(e))

__device__ __forceinline__ float ex2_approx_b(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr int kMaxViews = MS_MAX_BWD_VIEWS;  // views one batched backward call takes

struct ViewB {                // one view's inputs to raster_bwd_kernel
    const uint32_t *ranges;
    const uint32_t *gidx;
    const float4 *rec;
    uint32_t n_rec;
    int W, H, tiles_x, tiles;
    const float *image;       // [3][H][W] as the forward wrote it
    const float *dl;          // [3][H][W]
    const uint32_t *n_contrib;
    const uint32_t *seg_off;  // the forward's segmentation
    const uint32_t *seg_len;
    const float4 *pre;        // [max_segs][256] state after each segment
    float *g2;                // [n][kG2] this view's 2D gradients
};

struct BwdArgs {
    ViewB v[kMaxViews];
    int n_views;
    uint32_t *ticket;
};

// Sum of v[q] over the 32 lanes of a warp, reduce-scattered: lane l returns
// the full sum of value q(l) = l < 4 ? l / 2 : l / 4 + 1 when it is an
// owner (l < 4 ? l even : l % 4 == 0), a partial sum otherwise.  Halving
// the set of values a lane carries at every step costs 5 + 3 + 2 + 1 + 1
// shuffles instead of 9 x 5.
__device__ __forceinline__ float reduce_scatter9(const float v[kG2], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    // xor 16: lanes 0-15 keep values 0-4, lanes 16-31 values 5-8
    float a[5];
#pragma unroll
    for (int k = 0; k < 5; k++) {
        const float hi = k < 4 ? v[5 + k] : 0.0f;
        const float keep = b4 ? hi : v[k], send = b4 ? v[k] : hi;
        a[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    // xor 8: {0,1,2 | 3,4} and {5,6 | 7,8}
    float b[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float hi = b4 ? (k + 2 < 5 ? a[k + 2] : 0.0f) : (k + 3 < 5 ? a[k + 3] : 0.0f);
        const float keep = b3 ? hi : a[k], send = b3 ? a[k] : hi;
        b[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    // xor 4: {0,1 | 2}, {3 | 4}, {5 | 6}, {7 | 8}
    const bool g3 = !b4 && !b3;
    float c[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const float hi = g3 ? (k + 2 < 3 ? b[k + 2] : 0.0f) : b[k + 1];
        const float keep = b2 ? hi : b[k], send = b2 ? b[k] : hi;
        c[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    // xor 2: {0 | 1}; every other group holds one value
    const bool two = g3 && !b2;
    const float keep = (two && b1) ? c[1] : c[0];
    const float send = two ? (b1 ? c[0] : c[1]) : c[0];
    const float d = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    return d + __shfl_xor_sync(0xffffffffu, d, 1);
}

// Two pixels of one thread, (x, y) and (x, y + 4): the same dx for every
// record, so their arithmetic runs as packed FP32x2 pairs.
struct PixPair {
    f32x2 T, F0, F1, F2, C0, C1, C2, d0, d1, d2;
    uint32_t cntA, cntB;  // entries of the segment each pixel blended through
};

__global__ void __launch_bounds__(kBwdThreads, 8)  // 64 registers: 8 CTAs per SM
raster_bwd_kernel(const __grid_constant__ BwdArgs args) {
    __shared__ float4 s_r0[kBwdBatch], s_r1[kBwdBatch];
    __shared__ float4 s_r2[kBwdBatch];             // b, thr, ex, ey
    __shared__ uint32_t s_idx[kBwdBatch];
    __shared__ uint16_t s_list[kBwdThreads / 32][kBwdBatch];  // per warp: records in reach
    __shared__ float s_acc[kBwdBatch][kG2 + 1];  // [kG2] marks a record some pixel took
    __shared__ uint32_t s_c, s_cnt;
    __shared__ uint32_t s_first[kMaxViews + 1];   // first ticket of each view's segments
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool owner = lane < 4 ? (lane & 1) == 0 : (lane & 3) == 0;
    const int q_own = lane < 4 ? lane >> 1 : (lane >> 2) + 1;
    // this thread's pixels within a tile: warp w covers the 8x8 block
    // ((w & 1) * 8, (w >> 1) * 8), lane l the pixels (l & 7, l >> 3) and
    // (l & 7, (l >> 3) + 4) of it
    const int lx = (wid & 1) * 8 + (lane & 7);
    const int lyA = (wid >> 1) * 8 + (lane >> 3), lyB = lyA + 4;
    const int fA = fwd_index(lx, lyA), fB = fwd_index(lx, lyB);
    for (int i = tid; i < kBwdBatch * (kG2 + 1); i += kBwdThreads) (&s_acc[0][0])[i] = 0.0f;
    if (tid == 0) {
        uint32_t run = 0;
        for (int k = 0; k < args.n_views; k++) {
            s_first[k] = run;
            run += args.v[k].seg_off[args.v[k].tiles];
        }
        s_first[args.n_views] = run;
    }
    __syncthreads();
    const uint32_t total = s_first[args.n_views];
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            s_c = atomicAdd(args.ticket, 1u);
            s_cnt = 0;
        }
        __syncthreads();
        const uint32_t cg = s_c;
        if (cg >= total) break;
        // the view whose segments this ticket falls in
        int view = 0;
        while (view + 1 < args.n_views && cg >= s_first[view + 1]) view++;
        const ViewB &a = args.v[view];
        const uint32_t c = cg - s_first[view];
        const uint32_t L = a.seg_len[0];
        // the segment: tile t, index k within the tile, list entries [start, start + len)
        int lo = 0, hi = a.tiles;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.seg_off[mid] <= c) lo = mid;
            else hi = mid;
        }
        const int t = lo;
        const uint32_t k = c - a.seg_off[t];
        const uint32_t tbeg = a.ranges[2 * t], tend = a.ranges[2 * t + 1];
        const uint32_t pos0 = k * L;  // tile-relative position of the first entry
        const uint32_t start = tbeg + pos0;
        const uint32_t len = tend > start ? min(tend - start, L) : 0u;
        const int tx = t % a.tiles_x, ty = t / a.tiles_x;
        const int px = tx * 16 + lx;
        PixPair pp;
        float st[2][10];  // per pixel: T, F0..2, C0..2, d0..2
        uint32_t cnt[2] = {0u, 0u};
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int py = ty * 16 + (h ? lyB : lyA);
            st[h][0] = 1.0f;
#pragma unroll
            for (int q = 1; q < 10; q++) st[h][q] = 0.0f;
            if (px < a.W && py < a.H && len > 0) {
                const size_t p = (size_t)py * a.W + px, plane = (size_t)a.W * a.H;
                const uint32_t nc = a.n_contrib[p];
                if (nc > pos0) {
                    cnt[h] = min(nc - pos0, len);
                    if (k > 0) {
                        const float4 s4 =
                            __ldcg(a.pre + (size_t)(c - 1) * kRasterThreads + (h ? fB : fA));
                        st[h][0] = s4.w;
                        st[h][1] = s4.x;
                        st[h][2] = s4.y;
                        st[h][3] = s4.z;
                    }
                    st[h][4] = a.image[p];
                    st[h][5] = a.image[plane + p];
                    st[h][6] = a.image[2 * plane + p];
                    st[h][7] = a.dl[p];
                    st[h][8] = a.dl[plane + p];
                    st[h][9] = a.dl[2 * plane + p];
                }
            }
        }
        pp.T = pack2(st[0][0], st[1][0]);
        pp.F0 = pack2(st[0][1], st[1][1]);
        pp.F1 = pack2(st[0][2], st[1][2]);
        pp.F2 = pack2(st[0][3], st[1][3]);
        pp.C0 = pack2(st[0][4], st[1][4]);
        pp.C1 = pack2(st[0][5], st[1][5]);
        pp.C2 = pack2(st[0][6], st[1][6]);
        pp.d0 = pack2(st[0][7], st[1][7]);
        pp.d1 = pack2(st[0][8], st[1][8]);
        pp.d2 = pack2(st[0][9], st[1][9]);
        pp.cntA = cnt[0];
        pp.cntB = cnt[1];
        const float fx = (float)px + 0.5f;
        const f32x2 fy2 = pack2((float)(ty * 16 + lyA) + 0.5f, (float)(ty * 16 + lyB) + 0.5f);
        // centre of the warp's 8x8 block of pixel centres
        const float bcx = (float)(tx * 16 + (wid & 1) * 8) + 4.0f;
        const float bcy = (float)(ty * 16 + (wid >> 1) * 8) + 4.0f;
        const uint32_t wcnt = __reduce_max_sync(0xffffffffu, max(pp.cntA, pp.cntB));
        if (lane == 0 && wcnt) atomicMax(&s_cnt, wcnt);
        __syncthreads();
        const uint32_t cnt_seg = s_cnt;
        for (uint32_t off = 0; off < cnt_seg; off += kBwdBatch) {
            const uint32_t nb = min(cnt_seg - off, (uint32_t)kBwdBatch);
            for (uint32_t r = tid; r < nb; r += kBwdThreads) {
                uint32_t g = a.gidx[start + off + r];
                if (g >= a.n_rec) g = 0;  // unreachable unless binning reported an error
                s_idx[r] = g;
                s_r0[r] = a.rec[3 * (size_t)g];
                s_r1[r] = a.rec[3 * (size_t)g + 1];
                s_r2[r] = a.rec[3 * (size_t)g + 2];
            }
            __syncthreads();
            const uint32_t jn = wcnt > off ? min(wcnt - off, nb) : 0u;  // warp-uniform
            // the records whose level-set box reaches the warp's
            // 8x8 block of pixel centres, in list order; any other record has
            // alpha < 1/255 at all of the warp's pixels
            uint32_t nl = 0;
            for (uint32_t j0 = 0; j0 < jn; j0 += 32) {
                const uint32_t j = j0 + lane;
                bool rel = false;
                if (j < jn) {
                    const float4 r0 = s_r0[j], r2 = s_r2[j];
                    // half extents of the 8x8 block of pixel centres, plus
                    // 1/16 px for the FP32 rounding of the level-set box
                    rel = fabsf(r0.x - bcx) <= r2.z + 3.5625f && fabsf(r0.y - bcy) <= r2.w + 3.5625f;
                }
                const uint32_t m = __ballot_sync(0xffffffffu, rel);
                if (rel) s_list[wid][nl + __popc(m & ((1u << lane) - 1u))] = (uint16_t)j;
                nl += __popc(m);
            }
            __syncwarp();
            for (uint32_t li = 0; li < nl; li++) {
                const uint32_t j = s_list[wid][li];
                const float4 r0 = s_r0[j], r1 = s_r1[j];
                const float4 r2 = s_r2[j];
                // the forward's exact FP32 operations, for both pixels
                const float dx = __fsub_rn(fx, r0.x);
                const f32x2 dy = sub2(fy2, splat2(r0.y));
                const f32x2 u = fma2(splat2(r0.w), dy, splat2(__fmul_rn(r0.z, dx)));
                const f32x2 pw = fma2(mul2(splat2(r1.x), dy), dy, mul2(splat2(dx), u));
                float pA, pB;
                unpack2(pw, pA, pB);
                const bool accA = off + j < pp.cntA && pA <= 0.0f && pA >= r2.y;
                const bool accB = off + j < pp.cntB && pB <= 0.0f && pB >= r2.y;
                if (!__any_sync(0xffffffffu, accA || accB)) continue;
                // alpha of accepted pixels, 0 for the others (no effect on
                // T, F or any gradient); gradients through alpha only below
                // the 0.99 clamp
                const float eA = ex2_approx_b(accA ? pA : -256.0f);
                const float eB = ex2_approx_b(accB ? pB : -256.0f);
                const float GA = r1.y * eA, GB = r1.y * eB;
                const float alA = accA ? fminf(0.99f, GA) : 0.0f;
                const float alB = accB ? fminf(0.99f, GB) : 0.0f;
                const f32x2 al = pack2(alA, alB);
                const f32x2 mg = pack2(accA && GA < 0.99f ? 1.0f : 0.0f,
                                       accB && GB < 0.99f ? 1.0f : 0.0f);
                const f32x2 e = pack2(eA, eB);
                const f32x2 w = mul2(al, pp.T);
                const f32x2 cr = splat2(r1.z), cg2 = splat2(r1.w), cb2 = splat2(r2.x);
                pp.F0 = fma2(w, cr, pp.F0);
                pp.F1 = fma2(w, cg2, pp.F1);
                pp.F2 = fma2(w, cb2, pp.F2);
                const f32x2 om = sub2(splat2(1.0f), al);
                const f32x2 iom = pack2(__fdividef(1.0f, 1.0f - alA), __fdividef(1.0f, 1.0f - alB));
                // dC/dalpha = T c - (C - F) / (1 - alpha), summed over channels with dL/dC
                const f32x2 t0 = fma2(sub2(pp.C0, pp.F0), mul2(splat2(-1.0f), iom),
                                      mul2(pp.T, cr));
                const f32x2 t1 = fma2(sub2(pp.C1, pp.F1), mul2(splat2(-1.0f), iom),
                                      mul2(pp.T, cg2));
                const f32x2 t2 = fma2(sub2(pp.C2, pp.F2), mul2(splat2(-1.0f), iom),
                                      mul2(pp.T, cb2));
                const f32x2 dal = fma2(pp.d2, t2, fma2(pp.d1, t1, mul2(pp.d0, t0)));
                pp.T = mul2(pp.T, om);
                const f32x2 hd = mul2(mul2(dal, mg), e);     // dL/dsigma terms
                const f32x2 dpow = mul2(mul2(dal, mg), al);  // dL/dpower terms
                const float ca = r0.z * kInvConicA, cb = r0.w * kInvConicB, cc = r1.x * kInvConicA;
                const f32x2 gx = fma2(splat2(cb), dy, splat2(ca * dx));
                const f32x2 gy = fma2(splat2(cc), dy, splat2(cb * dx));
                float v[kG2], lo2, hi2;
                unpack2(mul2(dpow, gx), lo2, hi2);
                v[0] = lo2 + hi2;
                unpack2(mul2(dpow, gy), lo2, hi2);
                v[1] = lo2 + hi2;
                unpack2(dpow, lo2, hi2);
                v[2] = (lo2 + hi2) * (-0.5f * dx * dx);
                unpack2(mul2(dpow, dy), lo2, hi2);
                v[3] = -dx * (lo2 + hi2);
                unpack2(mul2(mul2(dpow, dy), dy), lo2, hi2);
                v[4] = -0.5f * (lo2 + hi2);
                unpack2(hd, lo2, hi2);
                v[5] = lo2 + hi2;
                unpack2(mul2(w, pp.d0), lo2, hi2);
                v[6] = lo2 + hi2;
                unpack2(mul2(w, pp.d1), lo2, hi2);
                v[7] = lo2 + hi2;
                unpack2(mul2(w, pp.d2), lo2, hi2);
                v[8] = lo2 + hi2;
                const float sum = reduce_scatter9(v, lane);
                if (owner) {
                    atomicAdd(&s_acc[j][q_own], sum);
                    if (lane == 0) s_acc[j][kG2] = 1.0f;
                }
            }
            __syncthreads();
            for (uint32_t r = tid; r < nb; r += kBwdThreads) {
                if (s_acc[r][kG2] == 0.0f) continue;
                float *dst = a.g2 + (size_t)s_idx[r] * kG2;
#pragma unroll
                for (int q = 0; q < kG2; q++) {
                    if (s_acc[r][q] != 0.0f) atomicAdd(dst + q, s_acc[r][q]);
                    s_acc[r][q] = 0.0f;
                }
                s_acc[r][kG2] = 0.0f;
            }
            __syncthreads();
        }
    }
}

struct SceneB {
    int64_t n;
    int sh_degree;
    const float *mean, *quat, *color, *scale;
};

struct CamB {
    float W[9], t[3], campos[3];
    float fx, fy, width, height;
};

// d/d(x, y, z) of the real SH basis polynomials (degree <= 3), k = l^2 + l + m
template <int DEG>
__device__ __forceinline__ void sh_grad(float x, float y, float z, const float *coef,
                                        const float dr[3], float g[3]) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    float Dx[K], Dy[K], Dz[K];
    Dx[0] = Dy[0] = Dz[0] = 0.0f;
    if constexpr (DEG >= 1) {
        const float c1 = 0.4886025119029199f;
        Dx[1] = 0; Dy[1] = c1; Dz[1] = 0;
        Dx[2] = 0; Dy[2] = 0; Dz[2] = c1;
        Dx[3] = c1; Dy[3] = 0; Dz[3] = 0;
    }
    if constexpr (DEG >= 2) {
        const float k4 = 1.0925484305920792f, k6 = 0.31539156525252005f,
                    k8 = 0.5462742152960396f;
        Dx[4] = k4 * y; Dy[4] = k4 * x; Dz[4] = 0;
        Dx[5] = 0; Dy[5] = k4 * z; Dz[5] = k4 * y;
        Dx[6] = -2 * k6 * x; Dy[6] = -2 * k6 * y; Dz[6] = 4 * k6 * z;
        Dx[7] = k4 * z; Dy[7] = 0; Dz[7] = k4 * x;
        Dx[8] = 2 * k8 * x; Dy[8] = -2 * k8 * y; Dz[8] = 0;
    }
    if constexpr (DEG >= 3) {
        const float k9 = 0.5900435899266435f, k10 = 2.890611442640554f,
                    k11 = 0.4570457994644658f, k12 = 0.3731763325901154f,
                    k14 = 1.445305721320277f;
        const float xx = x * x, yy = y * y, zz = z * z;
        Dx[9] = 6 * k9 * x * y; Dy[9] = 3 * k9 * (xx - yy); Dz[9] = 0;
        Dx[10] = k10 * y * z; Dy[10] = k10 * x * z; Dz[10] = k10 * x * y;
        Dx[11] = -2 * k11 * x * y; Dy[11] = k11 * (4 * zz - xx - 3 * yy); Dz[11] = 8 * k11 * y * z;
        Dx[12] = -6 * k12 * x * z; Dy[12] = -6 * k12 * y * z; Dz[12] = k12 * (6 * zz - 3 * xx - 3 * yy);
        Dx[13] = k11 * (4 * zz - 3 * xx - yy); Dy[13] = -2 * k11 * x * y; Dz[13] = 8 * k11 * x * z;
        Dx[14] = 2 * k14 * x * z; Dy[14] = -2 * k14 * y * z; Dz[14] = k14 * (xx - yy);
        Dx[15] = 3 * k9 * (xx - yy); Dy[15] = -6 * k9 * x * y; Dz[15] = 0;
    }
    g[0] = g[1] = g[2] = 0.0f;
#pragma unroll
    for (int k = 1; k < K; k++) {
        const float s = dr[0] * coef[3 * k] + dr[1] * coef[3 * k + 1] + dr[2] * coef[3 * k + 2];
        g[0] = fmaf(s, Dx[k], g[0]);
        g[1] = fmaf(s, Dy[k], g[1]);
        g[2] = fmaf(s, Dz[k], g[2]);
    }
}

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y) {
    Y[0] = 0.28209479177387814f;
    if constexpr (DEG >= 1) {
        Y[1] = 0.4886025119029199f * y;
        Y[2] = 0.4886025119029199f * z;
        Y[3] = 0.4886025119029199f * x;
    }
    if constexpr (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = 1.0925484305920792f * x * y;
        Y[5] = 1.0925484305920792f * y * z;
        Y[6] = 0.31539156525252005f * (2.0f * zz - xx - yy);
        Y[7] = 1.0925484305920792f * x * z;
        Y[8] = 0.5462742152960396f * (xx - yy);
        if constexpr (DEG >= 3) {
            Y[9] = 0.5900435899266435f * y * (3.0f * xx - yy);
            Y[10] = 2.890611442640554f * x * y * z;
            Y[11] = 0.4570457994644658f * y * (4.0f * zz - xx - yy);
            Y[12] = 0.3731763325901154f * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
            Y[13] = 0.4570457994644658f * x * (4.0f * zz - xx - yy);
            Y[14] = 1.445305721320277f * z * (xx - yy);
            Y[15] = 0.5900435899266435f * x * (xx - 3.0f * yy);
        }
    }
}

// Store or accumulate one gradient entry.
__device__ __forceinline__ void put(float *p, float v, bool acc) { *p = acc ? *p + v : v; }

// Colour backward: SH coefficient gradients and the view-direction term of
// the mean gradient.  Returns the latter in dmu.
template <int DEG>
__device__ __forceinline__ void color_bwd(int64_t i, const SceneB &sc, const CamB &cam,
                                          const float *g2, const float *coef, float *dcol,
                                          float dmu[3]) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    float dx = sc.mean[3 * i] - cam.campos[0], dy = sc.mean[3 * i + 1] - cam.campos[1],
          dz = sc.mean[3 * i + 2] - cam.campos[2];
    const float r = sqrtf(dx * dx + dy * dy + dz * dz), ir = 1.0f / r;
    const float x = dx * ir, y = dy * ir, z = dz * ir;
    float Y[K];
    sh_basis<DEG>(x, y, z, Y);
    float pre[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int k = 0; k < K; k++) {
        pre[0] = fmaf(coef[3 * k], Y[k], pre[0]);
        pre[1] = fmaf(coef[3 * k + 1], Y[k], pre[1]);
        pre[2] = fmaf(coef[3 * k + 2], Y[k], pre[2]);
    }
    float dr[3];
    for (int c = 0; c < 3; c++) dr[c] = pre[c] > 0.0f ? g2[6 + c] : 0.0f;
#pragma unroll
    for (int k = 0; k < K; k++) {
        dcol[3 * k] += dr[0] * Y[k];
        dcol[3 * k + 1] += dr[1] * Y[k];
        dcol[3 * k + 2] += dr[2] * Y[k];
    }
    dmu[0] = dmu[1] = dmu[2] = 0.0f;
    if constexpr (DEG >= 1) {
        float gd[3];
        sh_grad<DEG>(x, y, z, coef, dr, gd);
        // project on the sphere's tangent plane, then through d / |d|
        const float dd = gd[0] * x + gd[1] * y + gd[2] * z;
        dmu[0] = (gd[0] - x * dd) * ir;
        dmu[1] = (gd[1] - y * dd) * ir;
        dmu[2] = (gd[2] - z * dd) * ir;
    }
}

struct GradsK {
    float *dmean, *dlog_scale, *dquat, *dopacity, *dcolor;
    bool acc;  // add to the outputs instead of overwriting them
};


// One view's chain rule for Gaussian i, from its 2D gradient g2: adds the
// geometry gradients to dm, dls, dqo and dop and the colour gradient to
// dcol (the Gaussian's row, as is coef).
template <int DEG>
__device__ __forceinline__ void view_chain(const SceneB &sc, const CamB &cam, const float *g2,
                                           int64_t i, float dm[3], float dls[3], float dqo[4],
                                           float &dop, const float *coef, float *dcol) {
    const float *W = cam.W;
    const float m0 = sc.mean[3 * i], m1 = sc.mean[3 * i + 1], m2 = sc.mean[3 * i + 2];
    const float tx = W[0] * m0 + W[1] * m1 + W[2] * m2 + cam.t[0];
    const float ty = W[3] * m0 + W[4] * m1 + W[5] * m2 + cam.t[1];
    const float tz = W[6] * m0 + W[7] * m1 + W[8] * m2 + cam.t[2];
    const float4 q4 = reinterpret_cast<const float4 *>(sc.quat)[i];
    const float qn = sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float iq = 1.0f / qn;
    const float w = q4.x * iq, x = q4.y * iq, y = q4.z * iq, z = q4.w * iq;
    float R[9];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
    const float se[3] = {sc.scale[3 * i], sc.scale[3 * i + 1], sc.scale[3 * i + 2]};
    float M[9], Sg[9];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) M[3 * r + c] = R[3 * r + c] * se[c];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++)
            Sg[3 * r + c] = M[3 * r] * M[3 * c] + M[3 * r + 1] * M[3 * c + 1] +
                            M[3 * r + 2] * M[3 * c + 2];
    const float limx = 1.3f * (0.5f * cam.width / cam.fx);
    const float limy = 1.3f * (0.5f * cam.height / cam.fy);
    const float xr = tx / tz, yr = ty / tz;
    const bool clx = fabsf(xr) > limx, cly = fabsf(yr) > limy;
    const float xc = fminf(limx, fmaxf(-limx, xr)), yc = fminf(limy, fmaxf(-limy, yr));
    const float J00 = cam.fx / tz, J02 = -cam.fx * xc / tz;
    const float J11 = cam.fy / tz, J12 = -cam.fy * yc / tz;
    float T[6];
    for (int c = 0; c < 3; c++) {
        T[c] = J00 * W[c] + J02 * W[6 + c];
        T[3 + c] = J11 * W[3 + c] + J12 * W[6 + c];
    }
    // V' and its inverse (the conic)
    float TS[6];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++)
            TS[3 * r + c] = T[3 * r] * Sg[c] + T[3 * r + 1] * Sg[3 + c] + T[3 * r + 2] * Sg[6 + c];
    const float va = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2] + 0.3f;
    const float vb = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
    const float vc = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5] + 0.3f;
    const float idet = 1.0f / (va * vc - vb * vb);
    const float Qa = vc * idet, Qb = -vb * idet, Qc = va * idet;
    float dt0 = 0.0f, dt1 = 0.0f, dt2 = 0.0f;
    // centre
    dt0 += g2[0] * cam.fx / tz;
    dt2 += -g2[0] * cam.fx * tx / (tz * tz);
    dt1 += g2[1] * cam.fy / tz;
    dt2 += -g2[1] * cam.fy * ty / (tz * tz);
    // G_V = -Q G_Q Q with G_Q = [[ga, gb/2], [gb/2, gc]]
    const float ga = g2[2], gb = 0.5f * g2[3], gc = g2[4];
    const float A00 = Qa * ga + Qb * gb, A01 = Qa * gb + Qb * gc;
    const float A10 = Qb * ga + Qc * gb, A11 = Qb * gb + Qc * gc;
    const float GV0 = -(A00 * Qa + A01 * Qb), GV1 = -(A00 * Qb + A01 * Qc),
                GV2 = -(A10 * Qb + A11 * Qc);
    const float GVm[4] = {GV0, GV1, GV1, GV2};
    // G_Sigma = T^T G_V T ; G_T = 2 G_V T Sigma
    float GS[9];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            float v = 0.0f;
            for (int p = 0; p < 2; p++)
                for (int q = 0; q < 2; q++) v += T[3 * p + r] * GVm[2 * p + q] * T[3 * q + c];
            GS[3 * r + c] = v;
        }
    float GT[6];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++)
            GT[3 * r + c] = 2.0f * (GVm[2 * r] * TS[c] + GVm[2 * r + 1] * TS[3 + c]);
    // G_J = G_T W^T
    float GJ[6];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++)
            GJ[3 * r + c] = GT[3 * r] * W[3 * c] + GT[3 * r + 1] * W[3 * c + 1] +
                            GT[3 * r + 2] * W[3 * c + 2];
    const float itz2 = 1.0f / (tz * tz);
    dt2 += GJ[0] * (-cam.fx * itz2) + GJ[4] * (-cam.fy * itz2) + GJ[2] * (cam.fx * xc * itz2) +
           GJ[5] * (cam.fy * yc * itz2);
    const float dxc = GJ[2] * (-cam.fx / tz), dyc = GJ[5] * (-cam.fy / tz);
    if (!clx) {
        dt0 += dxc / tz;
        dt2 += -dxc * tx * itz2;
    }
    if (!cly) {
        dt1 += dyc / tz;
        dt2 += -dyc * ty * itz2;
    }
    float dmu[3] = {0.0f, 0.0f, 0.0f};
    if constexpr (DEG >= 0) {
        color_bwd<DEG>(i, sc, cam, g2, coef, dcol, dmu);
    } else {  // plain RGB
        dcol[0] += g2[6];
        dcol[1] += g2[7];
        dcol[2] += g2[8];
    }
    for (int c = 0; c < 3; c++) dm[c] += W[c] * dt0 + W[3 + c] * dt1 + W[6 + c] * dt2 + dmu[c];
    // Sigma = M M^T: G_M = 2 G_Sigma M;  M = R diag(se)
    float GM[9];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++)
            GM[3 * r + c] = 2.0f * (GS[3 * r] * M[c] + GS[3 * r + 1] * M[3 + c] +
                                    GS[3 * r + 2] * M[6 + c]);
    float GR[9];
    for (int c = 0; c < 3; c++) {
        float gs = 0.0f;
        for (int r = 0; r < 3; r++) {
            gs += R[3 * r + c] * GM[3 * r + c];
            GR[3 * r + c] = GM[3 * r + c] * se[c];
        }
        dls[c] += gs * se[c];
    }
    float dq[4];
    dq[0] = GR[1] * (-2 * z) + GR[2] * (2 * y) + GR[3] * (2 * z) + GR[5] * (-2 * x) +
            GR[6] * (-2 * y) + GR[7] * (2 * x);
    dq[1] = GR[1] * (2 * y) + GR[2] * (2 * z) + GR[3] * (2 * y) + GR[4] * (-4 * x) +
            GR[5] * (-2 * w) + GR[6] * (2 * z) + GR[7] * (2 * w) + GR[8] * (-4 * x);
    dq[2] = GR[0] * (-4 * y) + GR[1] * (2 * x) + GR[2] * (2 * w) + GR[3] * (2 * x) +
            GR[5] * (2 * z) + GR[6] * (-2 * w) + GR[7] * (2 * z) + GR[8] * (-4 * y);
    dq[3] = GR[0] * (-4 * z) + GR[1] * (-2 * w) + GR[2] * (2 * x) + GR[3] * (2 * w) +
            GR[4] * (-4 * z) + GR[5] * (2 * y) + GR[6] * (2 * x) + GR[7] * (2 * y);
    const float dot = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
    dqo[0] += (dq[0] - w * dot) * iq;
    dqo[1] += (dq[1] - x * dot) * iq;
    dqo[2] += (dq[2] - y * dot) * iq;
    dqo[3] += (dq[3] - z * dot) * iq;
    dop += g2[5];
}

struct ProjBwdArgs {
    SceneB sc;
    CamB cam[kMaxViews];
    const float *g2[kMaxViews];  // [n][kG2] per view
    int n_views;
    GradsK out;
};

constexpr int kProjBwdWarps = 4;

// Colour coefficients per Gaussian and the padded (odd) row stride of their
// shared-memory copies, so that lanes reading their own rows hit distinct
// banks.
template <int DEG>
struct ColorRows {
    static constexpr int K = DEG < 0 ? 1 : (DEG + 1) * (DEG + 1);
    static constexpr int RS = 3 * K;
    static constexpr int STRIDE = RS | 1;
    static constexpr int WARP_FLOATS = 2 * 32 * STRIDE;  // coefficient and gradient rows
};

// A streaming pass over the scene, 32 consecutive Gaussians per warp: the
// warp stages their colour rows (and, when accumulating, the previous colour
// gradients) in shared memory with coalesced loads, each lane applies the
// chain rule of every view that blended its Gaussian, and the warp writes
// the colour gradient rows back coalesced.  Every output of every Gaussian
// is written (zero where no view blended it) unless accumulating.
template <int DEG>
__global__ void __launch_bounds__(kProjBwdWarps * 32)
project_bwd_kernel(const __grid_constant__ ProjBwdArgs p) {
    using CR = ColorRows<DEG>;
    extern __shared__ float s_rows[];
    __shared__ CamB s_cam[kMaxViews];  // lanes on different views read them at once
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < p.n_views; k += blockDim.x) s_cam[k] = p.cam[k];
    __syncthreads();
    float *s_coef = s_rows + wid * CR::WARP_FLOATS;
    float *s_dcol = s_coef + 32 * CR::STRIDE;
    const bool acc = p.out.acc;
    const int64_t n = p.sc.n;
    const int64_t warps = (int64_t)gridDim.x * kProjBwdWarps;
    for (int64_t i0 = ((int64_t)blockIdx.x * kProjBwdWarps + wid) * 32; i0 < n; i0 += warps * 32) {
        const int64_t i = i0 + lane;
        const int rows = (int)min((int64_t)32, n - i0);
        uint32_t vmask = 0;  // views that blended this lane's Gaussian
        if (i < n) {
            for (int k = 0; k < p.n_views; k++) {
                const float *g2 = p.g2[k] + i * kG2;
                bool any = false;
#pragma unroll
                for (int q = 0; q < kG2; q++) any |= g2[q] != 0.0f;
                vmask |= (uint32_t)any << k;
            }
        }
        const bool warp_any = __any_sync(0xffffffffu, vmask != 0);
        if (!warp_any && acc) continue;
        const float *gcol = p.sc.color + i0 * CR::RS;
        float *gdc = p.out.dcolor + i0 * CR::RS;
        if (warp_any) {
            for (int e = lane; e < rows * CR::RS; e += 32) {
                const int r = e / CR::RS, col = e - r * CR::RS;
                s_coef[r * CR::STRIDE + col] = gcol[e];
                s_dcol[r * CR::STRIDE + col] = acc ? gdc[e] : 0.0f;
            }
        }
        __syncwarp();
        float dm[3] = {0.0f, 0.0f, 0.0f}, dls[3] = {0.0f, 0.0f, 0.0f};
        float dq[4] = {0.0f, 0.0f, 0.0f, 0.0f}, dop = 0.0f;
        // each lane walks its own views in ascending order (the order of the
        // sums is the same for every lane), so a round is idle only for lanes
        // with fewer views, not for every view another lane needs
        uint32_t m = vmask;
        while (__any_sync(0xffffffffu, m != 0u)) {
            if (m) {
                const int k = __ffs(m) - 1;
                m &= m - 1u;
                view_chain<DEG>(p.sc, s_cam[k], p.g2[k] + i * kG2, i, dm, dls, dq, dop,
                                s_coef + lane * CR::STRIDE, s_dcol + lane * CR::STRIDE);
            }
        }
        __syncwarp();
        for (int e = lane; e < rows * CR::RS; e += 32) {
            const int r = e / CR::RS;
            gdc[e] = warp_any ? s_dcol[r * CR::STRIDE + e - r * CR::RS] : 0.0f;
        }
        __syncwarp();
        if (i < n && (vmask != 0 || !acc)) {
            for (int c = 0; c < 3; c++) {
                put(p.out.dmean + 3 * i + c, dm[c], acc);
                put(p.out.dlog_scale + 3 * i + c, dls[c], acc);
            }
            for (int c = 0; c < 4; c++) put(p.out.dquat + 4 * i + c, dq[c], acc);
            put(p.out.dopacity + i, dop, acc);
        }
    }
}

template <int DEG>
static int launch_project_bwd(const ProjBwdArgs &pb, cudaStream_t st) {
    using CR = ColorRows<DEG>;
    const int smem = kProjBwdWarps * CR::WARP_FLOATS * (int)sizeof(float);
    int rc = ensure_smem_attr(reinterpret_cast<const void *>(project_bwd_kernel<DEG>), smem);
    if (rc) return rc;
    const int64_t warps = ceil_div(pb.sc.n, 32);
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>(ceil_div(warps, kProjBwdWarps), (int64_t)num_sms() * 16));
    project_bwd_kernel<DEG><<<grid, kProjBwdWarps * 32, smem, st>>>(pb);
    return MS_OK;
}

constexpr int kL1Threads = 256;

__global__ void __launch_bounds__(kL1Threads)
l1_loss_grad_kernel(const float4 *__restrict__ img, const float4 *__restrict__ tgt, int64_t n4,
                    const float *__restrict__ img1, const float *__restrict__ tgt1, int64_t tail,
                    float weight, float4 *__restrict__ dl, float *__restrict__ dl1,
                    float *loss_sum) {
    float acc = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)kL1Threads + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * kL1Threads) {
        const float4 a = img[i], b = tgt[i];
        const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
        acc += fabsf(d0) + fabsf(d1) + fabsf(d2) + fabsf(d3);
        dl[i] = make_float4(copysignf(d0 != 0.0f ? weight : 0.0f, d0),
                            copysignf(d1 != 0.0f ? weight : 0.0f, d1),
                            copysignf(d2 != 0.0f ? weight : 0.0f, d2),
                            copysignf(d3 != 0.0f ? weight : 0.0f, d3));
    }
    if (blockIdx.x == 0 && threadIdx.x < tail) {
        const float d = img1[threadIdx.x] - tgt1[threadIdx.x];
        acc += fabsf(d);
        dl1[threadIdx.x] = copysignf(d != 0.0f ? weight : 0.0f, d);
    }
    if (!loss_sum) return;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float s_part[kL1Threads / 32];
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int k = 0; k < kL1Threads / 32; k++) t += s_part[k];
        atomicAdd(loss_sum, t * weight);
    }
}

}  // namespace msgs

using namespace msgs;

extern "C" int ms_l1_loss_grad(const float *image, const float *target, int64_t count,
                               float weight, float *dl_dimage, float *loss_sum, void *stream) {
    if (count < 0) return fail(MS_ERR_INVALID_ARG, "count must be >= 0");
    if (count == 0) return MS_OK;
    if (!image || !target || !dl_dimage) return fail(MS_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned(image, 16) || !aligned(target, 16) || !aligned(dl_dimage, 16))
        return fail(MS_ERR_INVALID_ARG, "image, target and dl_dimage must be 16-byte aligned");
    if (loss_sum && !aligned(loss_sum, 4)) return fail(MS_ERR_INVALID_ARG, "loss_sum misaligned");
    const int64_t n4 = count / 4, tail = count - 4 * n4;
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>(ceil_div(n4, kL1Threads), (int64_t)num_sms() * 8));
    l1_loss_grad_kernel<<<grid, kL1Threads, 0, as_stream(stream)>>>(
        reinterpret_cast<const float4 *>(image), reinterpret_cast<const float4 *>(target), n4,
        image + 4 * n4, target + 4 * n4, tail, weight, reinterpret_cast<float4 *>(dl_dimage),
        dl_dimage + 4 * n4, loss_sum);
    return cuda_check(cudaGetLastError(), "l1 loss launch");
}

extern "C" size_t ms_raster_bwd_views_workspace_bytes(int64_t n, int32_t n_views) {
    if (n < 0 || n > INT32_MAX || n_views < 1 || n_views > MS_MAX_BWD_VIEWS) return 0;
    return al256(4) + (size_t)n_views * al256((size_t)(n > 0 ? n : 1) * kG2 * sizeof(float));
}

extern "C" size_t ms_raster_bwd_workspace_bytes(int64_t n) {
    return ms_raster_bwd_views_workspace_bytes(n, 1);
}

static int raster_bwd_blocks_per_sm() {
    static std::atomic<int> v{0};
    int b = v.load(std::memory_order_relaxed);
    if (b == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, raster_bwd_kernel, kBwdThreads, 0) !=
                cudaSuccess ||
            b < 1)
            b = 1;
        v.store(b, std::memory_order_relaxed);
    }
    return b;
}

extern "C" int ms_raster_bwd_views(const ms_scene_t *scene, const ms_bwd_view_t *views,
                                   int32_t n_views, const ms_grads_t *grads, uint32_t flags,
                                   void *ws, size_t ws_bytes, void *stream) {
    if (!scene || !views || !grads) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    if (n_views < 1 || n_views > MS_MAX_BWD_VIEWS)
        return fail(MS_ERR_INVALID_ARG, "n_views must be 1..MS_MAX_BWD_VIEWS");
    if (scene->n < 0 || scene->n > INT32_MAX) return fail(MS_ERR_INVALID_ARG, "scene n out of range");
    if (scene->n > 0 && (!grads->dmean || !grads->dlog_scale || !grads->dquat ||
                         !grads->dopacity || !grads->dcolor))
        return fail(MS_ERR_INVALID_ARG, "ms_grads_t has a NULL buffer");
    if (scene->n > 0 && (!scene->mean || !scene->quat || !scene->scale || !scene->color))
        return fail(MS_ERR_INVALID_ARG, "scene mean/quat/scale/color is NULL");
    if (scene->sh_degree < -1 || scene->sh_degree > 3)
        return fail(MS_ERR_INVALID_ARG, "sh_degree must be in -1..3");
    if (flags & ~(MS_BWD_ACCUMULATE | MS_BWD_RASTER_PASS | MS_BWD_PROJECT_PASS))
        return fail(MS_ERR_INVALID_ARG, "unknown flags");
    const bool accumulate = (flags & MS_BWD_ACCUMULATE) != 0;
    const uint32_t passes = flags & (MS_BWD_RASTER_PASS | MS_BWD_PROJECT_PASS);
    const bool raster_pass = passes == 0 || (passes & MS_BWD_RASTER_PASS);
    const bool project_pass = passes == 0 || (passes & MS_BWD_PROJECT_PASS);
    const size_t need = ms_raster_bwd_views_workspace_bytes(scene->n, n_views);
    if (!ws || ws_bytes < need || !aligned(ws, 16))
        return fail(MS_ERR_INVALID_ARG, "backward workspace missing, too small or misaligned");
    char *w = static_cast<char *>(ws);
    const size_t g2_bytes = al256((size_t)(scene->n > 0 ? scene->n : 1) * kG2 * sizeof(float));
    BwdArgs a;
    ProjBwdArgs pb;
    a.n_views = n_views;
    a.ticket = reinterpret_cast<uint32_t *>(w);
    pb.n_views = n_views;
    for (int k = 0; k < n_views; k++) {
        const ms_bwd_view_t &v = views[k];
        const ms_camera_t *cam = &v.cam;
        if (!v.proj || !v.bins) return fail(MS_ERR_INVALID_ARG, "view proj or bins is NULL");
        if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
            return fail(MS_ERR_INVALID_ARG, "image size must be 1..32768");
        if (!v.dl_dimage || !v.image || !v.n_contrib)
            return fail(MS_ERR_INVALID_ARG, "image, n_contrib and dl_dimage are required");
        if (v.proj->n < scene->n || !v.proj->rec)
            return fail(MS_ERR_INVALID_ARG, "ms_proj_t too small");
        if (!v.bins->gauss_idx || !v.bins->ranges)
            return fail(MS_ERR_INVALID_ARG, "bins buffers NULL");
        const int tiles_x = (cam->width + 15) / 16, tiles_y = (cam->height + 15) / 16;
        RasterLayout RL;
        if (!raster_layout((int64_t)tiles_x * tiles_y, v.bins->dup_capacity, RL))
            return fail(MS_ERR_INVALID_ARG, "tiles or dup_capacity out of range");
        if (!v.raster_ws || v.raster_ws_bytes < RL.total || !aligned(v.raster_ws, 16))
            return fail(MS_ERR_INVALID_ARG, "forward raster workspace missing or too small");
        const char *rw = static_cast<const char *>(v.raster_ws);
        ViewB &b = a.v[k];
        b.ranges = v.bins->ranges;
        b.gidx = v.bins->gauss_idx;
        b.rec = reinterpret_cast<const float4 *>(v.proj->rec);
        b.n_rec = (uint32_t)v.proj->n;
        b.W = cam->width;
        b.H = cam->height;
        b.tiles_x = tiles_x;
        b.tiles = tiles_x * tiles_y;
        b.image = v.image;
        b.dl = v.dl_dimage;
        b.n_contrib = v.n_contrib;
        b.seg_off = reinterpret_cast<const uint32_t *>(rw + RL.seg_off);
        b.seg_len = reinterpret_cast<const uint32_t *>(rw + RL.seg_len);
        b.pre = reinterpret_cast<const float4 *>(rw + RL.pre);
        b.g2 = reinterpret_cast<float *>(w + al256(4) + (size_t)k * g2_bytes);
        CamB &cb = pb.cam[k];
        for (int q = 0; q < 9; q++) cb.W[q] = cam->R[q];
        for (int q = 0; q < 3; q++) {
            cb.t[q] = cam->t[q];
            cb.campos[q] = cam->campos[q];
        }
        cb.fx = cam->fx;
        cb.fy = cam->fy;
        cb.width = (float)cam->width;
        cb.height = (float)cam->height;
        pb.g2[k] = b.g2;
    }
    cudaStream_t st = as_stream(stream);
    const int64_t n = scene->n;
    int rc;
    if (raster_pass) {
        if ((rc = cuda_check(cudaMemsetAsync(ws, 0, need, st), "bwd workspace memset")))
            return rc;
        raster_bwd_kernel<<<raster_bwd_blocks_per_sm() * num_sms(), kBwdThreads, 0, st>>>(a);
    }
    if (n > 0 && project_pass) {
        pb.sc.n = n;
        pb.sc.sh_degree = scene->sh_degree;
        pb.sc.mean = scene->mean;
        pb.sc.quat = scene->quat;
        pb.sc.color = scene->color;
        pb.sc.scale = scene->scale;
        pb.out = {grads->dmean, grads->dlog_scale, grads->dquat, grads->dopacity, grads->dcolor,
                  accumulate};
        switch (scene->sh_degree) {
        case 0: rc = launch_project_bwd<0>(pb, st); break;
        case 1: rc = launch_project_bwd<1>(pb, st); break;
        case 2: rc = launch_project_bwd<2>(pb, st); break;
        case 3: rc = launch_project_bwd<3>(pb, st); break;
        default: rc = launch_project_bwd<-1>(pb, st);
        }
        if (rc) return rc;
    }
    return cuda_check(cudaGetLastError(), "backward launches");
}

extern "C" int ms_raster_bwd(const ms_scene_t *scene, const ms_camera_t *cam,
                             const ms_proj_t *proj, const ms_bins_t *bins, const float *image,
                             const uint32_t *n_contrib, const void *raster_ws,
                             size_t raster_ws_bytes, const float *dl_dimage,
                             const ms_grads_t *grads, uint32_t flags, void *ws, size_t ws_bytes,
                             void *stream) {
    if (!cam) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    ms_bwd_view_t v;
    v.cam = *cam;
    v.proj = proj;
    v.bins = bins;
    v.image = image;
    v.n_contrib = n_contrib;
    v.raster_ws = raster_ws;
    v.raster_ws_bytes = raster_ws_bytes;
    v.dl_dimage = dl_dimage;
    return ms_raster_bwd_views(scene, &v, 1, grads, flags, ws, ws_bytes, stream);
}

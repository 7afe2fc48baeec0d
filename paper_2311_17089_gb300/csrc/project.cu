// Per-Gaussian kernels: scene activations, splat + coverage + selection
// (the K1 "project" stage), stand-alone selection and UpdateRange.
//
// The footprint below performs the operations of the FP32 footprint
// definition in a fixed order with single-rounding intrinsics, so masks,
// coverage, depth keys and tile rectangles are reproducible bit-for-bit.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cstring>

#include "common.cuh"
#include "footprint.cuh"
#include "tma.cuh"

namespace msgs {

// Eq. 6 (S_rel^max = 1.5, S_rel^min = 0.5, S_T = 2 px) with the level
// exemptions of Sec. 4.1: the finest level is never dropped as too large,
// the coarsest never as too small.
__device__ __forceinline__ bool select_pred(float S, int level, int n_levels,
                                            float smax, float smin, int mode) {
    if (mode == MS_ALL_LEVELS) return true;
    bool small_ok = (fdv(S, smin) >= 0.5f) || (S >= 2.0f);
    if (mode == MS_FILTER_SMALL) return small_ok;
    bool large_ok = (level == 1) || (fdv(S, smax) <= 1.5f);
    return large_ok && ((level == n_levels) || small_ok);
}

// Real SH basis to degree 3 (orthonormal, k = l^2 + l + m), colour =
// max(0, sum_k f_k Y_k + 0.5) per channel; coef is [K][3].
template <int DEG>
__device__ __forceinline__ float3 sh_color(const float *__restrict__ coef, float dx,
                                           float dy, float dz) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    float c[3 * K];
    if constexpr ((3 * K) % 4 == 0) {
        const float4 *src = reinterpret_cast<const float4 *>(coef);
#pragma unroll
        for (int k = 0; k < (3 * K) / 4; k++) {
            float4 v = __ldg(src + k);
            c[4 * k] = v.x;
            c[4 * k + 1] = v.y;
            c[4 * k + 2] = v.z;
            c[4 * k + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 3 * K; k++) c[k] = __ldg(coef + k);
    }
    float r = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    float x = dx * r, y = dy * r, z = dz * r;
    float Y[K];
    Y[0] = 0.28209479177387814f;
    if constexpr (DEG >= 1) {
        Y[1] = 0.4886025119029199f * y;
        Y[2] = 0.4886025119029199f * z;
        Y[3] = 0.4886025119029199f * x;
    }
    if constexpr (DEG >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
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
    float3 out = make_float3(0.5f, 0.5f, 0.5f);
#pragma unroll
    for (int k = 0; k < K; k++) {
        out.x = fmaf(c[3 * k + 0], Y[k], out.x);
        out.y = fmaf(c[3 * k + 1], Y[k], out.y);
        out.z = fmaf(c[3 * k + 2], Y[k], out.z);
    }
    out.x = fmaxf(out.x, 0.0f);
    out.y = fmaxf(out.y, 0.0f);
    out.z = fmaxf(out.z, 0.0f);
    return out;
}

__device__ __forceinline__ float3 gaussian_color(const float *__restrict__ color, int deg,
                                                 int64_t i, float dx, float dy, float dz) {
    switch (deg) {
    case 0: return sh_color<0>(color + i * 3, dx, dy, dz);
    case 1: return sh_color<1>(color + i * 12, dx, dy, dz);
    case 2: return sh_color<2>(color + i * 27, dx, dy, dz);
    case 3: return sh_color<3>(color + i * 48, dx, dy, dz);
    default:
        return make_float3(__ldg(color + 3 * i), __ldg(color + 3 * i + 1), __ldg(color + 3 * i + 2));
    }
}

// ------------------------------------------------------------- kernels

// ---------------------------------------------------------------- prepare
//
// scale = exp(log_scale) and lnop = ln(255 opacity), each the float nearest
// to the exact value (the definition rounds an FP64 evaluation to FP32).
// FP64 runs at a small fraction of the FP32 rate on this GPU, so both are
// evaluated in float-float arithmetic (an unevaluated sum of two floats,
// about 46 correct bits): range reduction by ln 2, a 1/32 (exp) or 1/64
// (ln) table step, then a Taylor series of the remainder.  The result is
// rounded to float; when the float-float value lies within its error bound
// of a rounding midpoint, an FP64 evaluation decides (a few values in 10^5).

struct ff {
    float h, l;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ff ff_fast(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {  // accurate sum
    ff s = ff_two_sum(a.h, b.h);
    const ff t = ff_two_sum(a.l, b.l);
    s = ff_fast(s.h, __fadd_rn(s.l, t.h));
    return ff_fast(s.h, __fadd_rn(s.l, t.l));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return ff_fast(p, e);
}
__device__ __forceinline__ ff ff_mulf(ff a, float b) {
    const float p = __fmul_rn(a.h, b);
    return ff_fast(p, __fmaf_rn(a.l, b, __fmaf_rn(a.h, b, -p)));
}

// v.h is the float nearest to v.h + v.l + d for every |d| <= err.
__device__ __forceinline__ bool ff_rounds_to_hi(ff v, float err) {
    const float ah = fabsf(v.h);
    const float up = __fsub_rn(__int_as_float(__float_as_int(ah) + 1), ah);
    const float dn = __fsub_rn(ah, __int_as_float(__float_as_int(ah) - 1));
    const float l = v.h < 0.0f ? -v.l : v.l;
    return l < __fsub_rn(__fmul_rn(0.5f, up), err) && l > __fsub_rn(err, __fmul_rn(0.5f, dn));
}

// ln 2 = kLn2A + kLn2B + kLn2C (kLn2A has 12 significant bits, so k kLn2A
// is exact for |k| < 2^12); 1/6, 1/24, 1/3 as float-float
constexpr float kLn2A = 0x1.62ep-1f, kLn2B = 0x1.0bfbe8p-15f, kLn2C = 0x1.cf79acp-40f;
constexpr float kR6h = 0x1.555556p-3f, kR6l = -0x1.555556p-28f;
constexpr float kR24h = 0x1.555556p-5f, kR24l = -0x1.555556p-30f;
constexpr float kR3h = 0x1.555556p-2f, kR3l = -0x1.555556p-27f;
constexpr float kFFErr = 0x1p-42f;  // relative error bound of the float-float results
constexpr int kExpTab = 25;         // exp(j/32), j = -12 .. 12
constexpr int kLnTab = 49;          // ln(3/4 + j/64), j = 0 .. 48

__device__ __forceinline__ float exp_rn(float x, const ff *texp) {
    if (!(fabsf(x) < 80.0f)) return (float)exp((double)x);
    const float k = rintf(__fmul_rn(x, 1.44269504f));  // |k| <= 116
    ff r = ff_two_sum(x, -__fmul_rn(k, kLn2A));
    const ff kb = ff_two_prod(k, kLn2B);
    r = ff_add(r, {-kb.h, -kb.l});
    r = ff_add(r, {-__fmul_rn(k, kLn2C), 0.0f});
    const float j = rintf(__fmul_rn(r.h, 32.0f));     // |j| <= 12
    r = ff_add(r, {-__fmul_rn(j, 0.03125f), 0.0f});   // |r| <= 1/64
    // exp(r) = 1 + r(1 + r(1/2 + r(1/6 + r(1/24 + r q)))), q the float tail
    const float q = __fmaf_rn(r.h, __fmaf_rn(r.h, 1.0f / 5040.0f, 1.0f / 720.0f), 1.0f / 120.0f);
    ff p = ff_add({kR24h, kR24l}, ff_mulf(r, q));
    p = ff_add({kR6h, kR6l}, ff_mul(r, p));
    p = ff_add({0.5f, 0.0f}, ff_mul(r, p));
    p = ff_add({1.0f, 0.0f}, ff_mul(r, p));
    p = ff_add({1.0f, 0.0f}, ff_mul(r, p));
    ff e = ff_mul(texp[(int)j + 12], p);
    const int ki = (int)k;
    e.h = ldexpf(e.h, ki);
    e.l = ldexpf(e.l, ki);
    if (ff_rounds_to_hi(e, __fmul_rn(kFFErr, fabsf(e.h)))) return e.h;
    return (float)exp((double)x);
}

__device__ __forceinline__ float lnop_rn(float sigma, const ff *tln) {
    if (!(sigma > 1e-30f) || !(sigma < 1e30f)) return (float)log(255.0 * (double)sigma);
    const ff y = ff_two_prod(255.0f, sigma);  // exact
    // y = 2^ex m, m in [3/4, 3/2)
    const int bits = __float_as_int(y.h);
    int ex = ((bits >> 23) & 0xff) - 127;
    float m = __int_as_float((bits & 0x007fffff) | 0x3f800000);
    if (m >= 1.5f) {
        m = __fmul_rn(m, 0.5f);
        ex += 1;
    }
    const float ml = ldexpf(y.l, -ex);
    const float j = rintf(__fmul_rn(__fsub_rn(m, 0.75f), 64.0f));  // 0 .. 48
    const float c = __fmaf_rn(j, 0.015625f, 0.75f);                // exact
    // t = (m + ml - c) / c, |t| <= 1/96
    const ff num = ff_two_sum(__fsub_rn(m, c), ml);
    const float t0 = __fdiv_rn(num.h, c);
    const float rem = __fadd_rn(__fmaf_rn(-t0, c, num.h), num.l);
    const ff t = ff_fast(t0, __fdiv_rn(rem, c));
    // ln(1 + t) = t (1 + t(-1/2 + t(1/3 + t(-1/4 + t q)))), q the float tail
    const float q = __fmaf_rn(t.h, __fmaf_rn(t.h, __fmaf_rn(t.h, -0.125f, 1.0f / 7.0f), -1.0f / 6.0f), 0.2f);
    ff p = ff_add({-0.25f, 0.0f}, ff_mulf(t, q));
    p = ff_add({kR3h, kR3l}, ff_mul(t, p));
    p = ff_add({-0.5f, 0.0f}, ff_mul(t, p));
    p = ff_add({1.0f, 0.0f}, ff_mul(t, p));
    const ff lg = ff_mul(t, p);
    const float exf = (float)ex;
    const ff eb = ff_two_prod(exf, kLn2B);
    ff a = ff_add({__fmul_rn(exf, kLn2A), 0.0f}, eb);
    a = ff_add(a, {__fmul_rn(exf, kLn2C), 0.0f});
    const ff tl = tln[(int)j];
    const ff sum = ff_add(ff_add(a, tl), lg);
    const float err = __fmul_rn(kFFErr, __fadd_rn(__fadd_rn(fabsf(a.h), fabsf(tl.h)), fabsf(lg.h)));
    if (ff_rounds_to_hi(sum, err)) return sum.h;
    return (float)log(255.0 * (double)sigma);
}

__global__ void __launch_bounds__(256)
prepare_kernel(int64_t n, const float *__restrict__ log_scale, const float *__restrict__ opacity,
               float *__restrict__ scale, float *__restrict__ lnop) {
    __shared__ ff s_exp[kExpTab], s_ln[kLnTab];
    const int t = threadIdx.x;
    if (t < kExpTab) {
        const double v = exp((double)(t - 12) / 32.0);
        const float h = (float)v;
        s_exp[t] = {h, (float)(v - (double)h)};
    } else if (t >= 64 && t < 64 + kLnTab) {
        const double v = log(0.75 + (double)(t - 64) / 64.0);
        const float h = (float)v;
        s_ln[t - 64] = {h, (float)(v - (double)h)};
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + t; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < 3; k++) scale[3 * i + k] = exp_rn(log_scale[3 * i + k], s_exp);
        lnop[i] = lnop_rn(opacity[i], s_ln);
    }
}

constexpr int kProjThreads = 256;
constexpr int kProjBlocksPerSM = 4;  // 64 registers: the footprint fits without spills
constexpr float kConicA = -0.72134752044448170f;   // -log2(e) / 2
constexpr float kConicB = -1.4426950408889634f;    // -log2(e)
constexpr float kLog2e = 1.4426950408889634f;

// The per-Gaussian geometry and opacity of one chunk of kProjThreads
// Gaussians, staged in shared memory by bulk copies (8 arrays, 14,592
// bytes).  Opacity is staged with the geometry (one coalesced read for
// every Gaussian) rather than gathered per listed Gaussian, a 4-byte read
// that costs a whole DRAM sector.
struct ProjStage {
    float mean[3 * kProjThreads];
    float scale[3 * kProjThreads];
    float4 quat[kProjThreads];
    float lnop[kProjThreads];
    float smax[kProjThreads];
    float smin[kProjThreads];
    float opacity[kProjThreads];
    uint8_t level[kProjThreads];
};
constexpr uint32_t kProjStageBytes = (3 + 3 + 4 + 4) * 4 * kProjThreads + kProjThreads;
static_assert(sizeof(ProjStage) == kProjStageBytes, "stage layout");

// Threads 0..7 of warp 0 issue the bulk copies of chunk c (every array
// offset is a multiple of 256 elements, so 16-byte aligned when the arrays
// are).
__device__ __forceinline__ void issue_chunk(const SceneK &sc, int64_t c, ProjStage &st,
                                            uint64_t *bar) {
    if (threadIdx.x >= 8) return;
    const int64_t i0 = c * kProjThreads;
    if (threadIdx.x == 0) mbar_expect_tx(bar, kProjStageBytes);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    switch (threadIdx.x) {
    case 0: bulk_copy_g2s(st.mean, sc.mean + 3 * i0, 12 * kProjThreads, bar); break;
    case 1: bulk_copy_g2s(st.scale, sc.scale + 3 * i0, 12 * kProjThreads, bar); break;
    case 2: bulk_copy_g2s(st.quat, sc.quat + 4 * i0, 16 * kProjThreads, bar); break;
    case 3: bulk_copy_g2s(st.lnop, sc.lnop + i0, 4 * kProjThreads, bar); break;
    case 4: bulk_copy_g2s(st.smax, sc.s_max + i0, 4 * kProjThreads, bar); break;
    case 5: bulk_copy_g2s(st.smin, sc.s_min + i0, 4 * kProjThreads, bar); break;
    case 6: bulk_copy_g2s(st.opacity, sc.opacity + i0, 4 * kProjThreads, bar); break;
    default: bulk_copy_g2s(st.level, sc.level + i0, kProjThreads, bar); break;
    }
}

// The outputs of one view (the buffers of its ms_proj_t).
struct ProjOut {
    float4 *rec;
    uint2 *rect;
    uint32_t *n_tiles, *depth;
    float *cover;
    uint32_t *mask, *stats;
};

// The cameras and outputs of one launch.  color_src[v] is the first view
// whose camera centre equals view v's (bitwise), so views that share a
// centre share the SH colour of a Gaussian listed in both.
template <int MAXV>
struct ProjViews {
    int n_views;
    int update_level[MAXV];  // level whose coverage range the view updates (0: none)
    // the union of the views in union_mask (all with one pose, so one depth
    // per Gaussian, taken in view union_first): per Gaussian the mask of
    // those views that list it (bit v: view v), and stats with the union's
    // count and depth-digit histograms; NULL: not formed
    uint32_t *union_flags, *union_stats;
    uint32_t union_mask;
    int union_first;
    float *smax_out, *smin_out;  // the scene's ranges, written when a view updates
    int color_src[MAXV];
    float fx2[MAXV], fy2[MAXV];  // squared focal lengths (the coverage bound)
    CamK cam[MAXV];
    ProjOut out[MAXV];
};

// Depth-digit histograms in shared memory hold two 16-bit counts per word
// (digits 2k and 2k + 1 of word k).  A CTA adds at most one count per pass
// and view for each Gaussian, so flushing them to global memory at least
// every kHistFlushChunks chunks keeps every count below 2^16.
constexpr int kHistFlushChunks = 255;
static_assert(kHistFlushChunks * kProjThreads < 65536, "16-bit digit counts");

// Histogram slots in shared memory: one per view, and for MAXV > 1 one
// more (slot MAXV) for the union of the views.
template <int MAXV>
__host__ __device__ constexpr int hist_slots() { return MAXV == 1 ? 1 : MAXV + 1; }

template <int MAXV>
__device__ __forceinline__ void flush_hist(uint32_t (*s_hist)[4][128], const ProjViews<MAXV> &pv) {
    const int nv = MAXV == 1 ? 1 : pv.n_views;
    const int slots = nv + (MAXV > 1 && pv.union_stats ? 1 : 0);
    for (int k = threadIdx.x; k < slots * 512; k += blockDim.x) {
        const int v = k >> 9, w = k & 511;
        const int slot = v < nv ? v : MAXV;
        uint32_t &word = (&s_hist[slot][0][0])[w];
        const uint32_t x = word;
        if (x) {
            const int pass = w >> 7, d = (w & 127) * 2;
            uint32_t *g = (v < nv ? pv.out[v].stats : pv.union_stats) + kStatHist + 256 * pass + d;
            if (x & 0xffffu) atomicAdd(g, x & 0xffffu);
            if (x >> 16) atomicAdd(g + 1, x >> 16);
            word = 0;
        }
    }
}

// K1: one thread per Gaussian, chunks of kProjThreads Gaussians per CTA
// (grid-stride).  While a chunk is processed, the geometry of the CTA's
// next chunk streams into the other stage buffer (full chunks of 16-byte
// aligned arrays; the ragged last chunk, or unaligned arrays, read global
// memory directly).  The 3D covariance of a Gaussian is formed once; then,
// view by view, its footprint, selection and (for listed Gaussians) record
// are written to that view's outputs, with the survivor count, the
// duplicate count and the four depth-digit histograms that the binning
// stage's radix sort needs.
// CTAs per SM: one view fits 64 registers; the view loop keeps the
// Gaussian's geometry and covariance live across views and gets 80.
template <int MAXV>
constexpr int proj_blocks_per_sm() { return MAXV == 1 ? kProjBlocksPerSM : 3; }

template <int MAXV>
__global__ void __launch_bounds__(kProjThreads, proj_blocks_per_sm<MAXV>())
project_kernel(SceneK sc, const __grid_constant__ ProjViews<MAXV> pv, int mode, bool staged_ok) {
    __shared__ uint32_t s_hist[hist_slots<MAXV>()][4][128];
    __shared__ uint32_t s_surv[MAXV + 1];
    __shared__ unsigned long long s_dup[MAXV];
    __shared__ __align__(128) ProjStage s_st[2];
    __shared__ __align__(8) uint64_t s_bar[2];
    for (int i = threadIdx.x; i < hist_slots<MAXV>() * 512; i += blockDim.x)
        (&s_hist[0][0][0])[i] = 0;
    if (threadIdx.x <= MAXV) s_surv[threadIdx.x] = 0;
    if (threadIdx.x < MAXV) s_dup[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int nv = MAXV == 1 ? 1 : pv.n_views;
    const int64_t nchunks = (sc.n + kProjThreads - 1) / kProjThreads;
    auto full = [&](int64_t c) { return staged_ok && (c + 1) * kProjThreads <= sc.n; };
    if ((int64_t)blockIdx.x < nchunks && full(blockIdx.x)) issue_chunk(sc, blockIdx.x, s_st[0], &s_bar[0]);
    uint32_t par = 0;
    int it = 0;
    // all threads of a warp iterate together so warp ballots stay full
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x, it++) {
        const int b = it & 1;
        const int64_t cn = c + gridDim.x;
        if (cn < nchunks && full(cn)) issue_chunk(sc, cn, s_st[b ^ 1], &s_bar[b ^ 1]);
        bool staged = full(c);
        if (staged) {
            bool ok = false;
            for (uint32_t spins = 0; spins < kSpinLimit && !ok; spins++)
                ok = mbar_try_wait(&s_bar[b], (par >> b) & 1u);
            par ^= 1u << b;
            if (!ok) {  // copies still out: this chunk reads global memory
                staged = false;
                for (int v = 0; v < pv.n_views; v++)
                    atomicOr(pv.out[v].stats + kStatStatus, (uint32_t)kStatusTimeout);
            }
        }
        const ProjStage &st = s_st[b];
        const int64_t base = c * kProjThreads;
        const int t = threadIdx.x;
        const int64_t i = base + t;
        const bool in = i < sc.n;
        float m[3] = {0.0f, 0.0f, 0.0f}, S6[6], lnop_i = 0.0f, smax_i = 0.0f, smin_i = 0.0f;
        float op = 0.0f;
        int level_i = 0;
        bool cov_ok = false;
        if (in) {
            float sv[3];
            float4 q;
            if (staged) {
                m[0] = st.mean[3 * t];
                m[1] = st.mean[3 * t + 1];
                m[2] = st.mean[3 * t + 2];
                sv[0] = st.scale[3 * t];
                sv[1] = st.scale[3 * t + 1];
                sv[2] = st.scale[3 * t + 2];
                q = st.quat[t];
                lnop_i = st.lnop[t];
                smax_i = st.smax[t];
                smin_i = st.smin[t];
                op = st.opacity[t];
                level_i = st.level[t];
            } else {
                m[0] = sc.mean[3 * i];
                m[1] = sc.mean[3 * i + 1];
                m[2] = sc.mean[3 * i + 2];
                sv[0] = sc.scale[3 * i];
                sv[1] = sc.scale[3 * i + 1];
                sv[2] = sc.scale[3 * i + 2];
                q = reinterpret_cast<const float4 *>(sc.quat)[i];
                lnop_i = sc.lnop[i];
                smax_i = sc.s_max[i];
                smin_i = sc.s_min[i];
                op = sc.opacity[i];
                level_i = sc.level[i];
            }
            cov_ok = cov3d(sv, q, S6);
        }
        float3 col = make_float3(0.0f, 0.0f, 0.0f);
        int col_src = -1;  // view whose camera centre col was evaluated towards
        bool range_dirty = false;
        uint32_t umask = 0u;      // the union's views that list it
        uint32_t depth0 = 0u;     // depth key in the pose the union's views share
        for (int v = 0; v < nv; v++) {
            const CamK &cam = pv.cam[v];
            const ProjOut &o = pv.out[v];
            bool sel = false, listed = false;
            uint32_t ntiles = 0;
            if (in) {
                Foot f;
                footprint_cov(m, S6, cov_ok, lnop_i, cam, f);
                if (f.valid) sel = select_pred(f.S, level_i, sc.n_levels, smax_i, smin_i, mode);
                // Alg. 2: a training render at the creation scale of level
                // l_r updates that level's ranges (Eq. 5) after its
                // selection used the ranges before the update; the next view
                // selects with the updated ones
                if (pv.update_level[v] == level_i && f.valid && f.ntiles > 0) {
                    smax_i = fmaxf(fm(0.95f, smax_i), f.S);
                    smin_i = fminf(fm(1.05f, smin_i), f.S);
                    range_dirty = true;
                }
                listed = sel && f.ntiles > 0;
                ntiles = listed ? f.ntiles : 0u;
                if (listed && ((pv.union_mask >> v) & 1u)) umask |= 1u << v;
                if (v == pv.union_first) depth0 = f.depth;
                o.n_tiles[i] = ntiles;
                // depth and rectangle of every Gaussian: coalesced writes
                // (per listed Gaussian alone they would be scattered 4- and
                // 8-byte writes, each a partial DRAM sector)
                o.depth[i] = f.depth;
                o.rect[i] = make_uint2((uint32_t)f.x0 | ((uint32_t)f.y0 << 16),
                                       (uint32_t)f.x1 | ((uint32_t)f.y1 << 16));
                if (o.cover) o.cover[i] = f.S;
                if (listed) {
                    const int src = pv.color_src[v];
                    if (src != col_src) {
                        col = gaussian_color(sc.color, sc.sh_degree, i, m[0] - cam.campos[0],
                                             m[1] - cam.campos[1], m[2] - cam.campos[2]);
                        col_src = src;
                    }
                    // conic pre-scaled so power * log2(e) = A dx^2 + B dx dy + C dy^2
                    o.rec[3 * i + 0] = make_float4(f.ux, f.uy, fm(kConicA, f.ca), fm(kConicB, f.cb));
                    o.rec[3 * i + 1] = make_float4(fm(kConicA, f.cc), op, col.x, col.y);
                    // alpha >= 1/255 <=> power * log2(e) >= -ln(255 sigma) log2(e)
                    o.rec[3 * i + 2] = make_float4(col.z, fm(-kLog2e, lnop_i), f.ex, f.ey);
                    uint32_t(*h)[128] = s_hist[MAXV == 1 ? 0 : v];
#pragma unroll
                    for (int p = 0; p < 4; p++) {
                        const uint32_t d = (f.depth >> (8 * p)) & 255u;
                        atomicAdd(&h[p][d >> 1], 1u << (16 * (d & 1u)));
                    }
                }
            }
            if (o.mask) {
                const uint32_t bits = __ballot_sync(0xffffffffu, in && sel);
                if ((threadIdx.x & 31) == 0 && in) o.mask[i >> 5] = bits;
            }
            // ntiles <= 2^22 per Gaussian, so a warp's sum fits 32 bits
            const uint32_t ws = __reduce_add_sync(0xffffffffu, listed ? 1u : 0u);
            const uint32_t wd = __reduce_add_sync(0xffffffffu, ntiles);
            if ((threadIdx.x & 31) == 0 && ws) {
                atomicAdd(&s_surv[MAXV == 1 ? 0 : v], ws);
                atomicAdd(&s_dup[MAXV == 1 ? 0 : v], (unsigned long long)wd);
            }
        }
        if (range_dirty) {
            pv.smax_out[i] = smax_i;
            pv.smin_out[i] = smin_i;
        }
        if (MAXV > 1 && pv.union_flags) {
            const bool any_listed = umask != 0u;
            if (in) pv.union_flags[i] = umask;
            if (any_listed) {
#pragma unroll
                for (int p = 0; p < 4; p++) {
                    const uint32_t d = (depth0 >> (8 * p)) & 255u;
                    atomicAdd(&s_hist[MAXV > 1 ? MAXV : 0][p][d >> 1], 1u << (16 * (d & 1u)));
                }
            }
            const uint32_t wu = __reduce_add_sync(0xffffffffu, any_listed ? 1u : 0u);
            if ((threadIdx.x & 31) == 0 && wu) atomicAdd(&s_surv[MAXV], wu);
        }
        __syncthreads();  // the buffer is refilled by the next iteration but one
        if ((it + 1) % kHistFlushChunks == 0) {
            flush_hist<MAXV>(s_hist, pv);
            __syncthreads();
        }
    }
    flush_hist<MAXV>(s_hist, pv);
    __syncthreads();
    if (threadIdx.x < nv) {
        const int v = threadIdx.x;
        uint32_t *stats = pv.out[v].stats;
        if (s_surv[v]) atomicAdd(&stats[kStatSurvivors], s_surv[v]);
        if (s_dup[v]) atomicAdd(reinterpret_cast<unsigned long long *>(stats + kStatDup), s_dup[v]);
    }
    if (MAXV > 1 && pv.union_stats && threadIdx.x == 0 && s_surv[MAXV])
        atomicAdd(&pv.union_stats[kStatSurvivors], s_surv[MAXV]);
}

// Position of the set bit of rank r (0-based, from the least significant)
// in m, which has more than r set bits.
__device__ __forceinline__ int nth_set_bit(uint32_t m, int r) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));
        if (r >= c) {
            r -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

// K1 for selective renders of one pose at several resolutions (every view
// with view 0's R, t and camera centre, no coverage output, no range
// update), leaving out the footprints that cannot be selected.  Per
// Gaussian the coverage bound (cover_bound) marks the views whose exact
// footprint is needed; the warp packs its (Gaussian, view) pairs that need
// one, 32 per round, each lane taking the pair's Gaussian (view-space
// point, covariance, colour) from the owner lane by shuffles and the
// camera and outputs from shared memory.  A pair left out holds n_tiles 0,
// the depth key and the empty rectangle (0, 0xffffffff); every other pair
// writes what project_kernel writes, so the lists, records, masks and stats
// are the same bit for bit.
template <int MAXV>
__global__ void __launch_bounds__(kProjThreads, 3)
project_pruned_kernel(SceneK sc, const __grid_constant__ ProjViews<MAXV> pv, bool staged_ok) {
    constexpr int kWarps = kProjThreads / 32;
    __shared__ uint32_t s_hist[MAXV + 1][4][128];
    __shared__ uint32_t s_surv[MAXV + 1];
    __shared__ unsigned long long s_dup[MAXV];
    __shared__ __align__(128) ProjStage s_st[2];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ CamK s_cam[MAXV];
    __shared__ ProjOut s_out[MAXV];
    __shared__ uint32_t s_bits[kProjThreads];  // per Gaussian: bit v selected, bit 8 + v listed
    __shared__ uint32_t s_vlanes[kWarps][MAXV];  // per warp and view: lanes needing the footprint
    __shared__ int s_voff[kWarps][MAXV];         // first pair of each view in the warp's packing
    for (int k = threadIdx.x; k < (MAXV + 1) * 512; k += blockDim.x) (&s_hist[0][0][0])[k] = 0;
    for (int k = threadIdx.x; k < (int)(MAXV * sizeof(CamK) / 4); k += blockDim.x)
        reinterpret_cast<uint32_t *>(s_cam)[k] = reinterpret_cast<const uint32_t *>(pv.cam)[k];
    if (threadIdx.x < MAXV) s_out[threadIdx.x] = pv.out[threadIdx.x];
    s_bits[threadIdx.x] = 0u;
    if (threadIdx.x <= MAXV) s_surv[threadIdx.x] = 0;
    if (threadIdx.x < MAXV) s_dup[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int nv = pv.n_views;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nchunks = (sc.n + kProjThreads - 1) / kProjThreads;
    auto full = [&](int64_t c) { return staged_ok && (c + 1) * kProjThreads <= sc.n; };
    if ((int64_t)blockIdx.x < nchunks && full(blockIdx.x)) issue_chunk(sc, blockIdx.x, s_st[0], &s_bar[0]);
    uint32_t par = 0;
    int it = 0;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x, it++) {
        const int b = it & 1;
        const int64_t cn = c + gridDim.x;
        if (cn < nchunks && full(cn)) issue_chunk(sc, cn, s_st[b ^ 1], &s_bar[b ^ 1]);
        bool staged = full(c);
        if (staged) {
            bool ok = false;
            for (uint32_t spins = 0; spins < kSpinLimit && !ok; spins++)
                ok = mbar_try_wait(&s_bar[b], (par >> b) & 1u);
            par ^= 1u << b;
            if (!ok) {  // copies still out: this chunk reads global memory
                staged = false;
                for (int v = 0; v < nv; v++)
                    atomicOr(pv.out[v].stats + kStatStatus, (uint32_t)kStatusTimeout);
            }
        }
        const ProjStage &st = s_st[b];
        const int64_t base = c * kProjThreads;
        const int t = threadIdx.x;
        const int64_t i = base + t;
        const bool in = i < sc.n;
        float m[3] = {0.0f, 0.0f, 0.0f}, S6[6], lnop_i = 0.0f, smax_i = 0.0f, smin_i = 0.0f;
        float op = 0.0f;
        int level_i = 0;
        bool cov_ok = false;
        if (in) {
            float sv[3];
            float4 q;
            if (staged) {
                m[0] = st.mean[3 * t];
                m[1] = st.mean[3 * t + 1];
                m[2] = st.mean[3 * t + 2];
                sv[0] = st.scale[3 * t];
                sv[1] = st.scale[3 * t + 1];
                sv[2] = st.scale[3 * t + 2];
                q = st.quat[t];
                lnop_i = st.lnop[t];
                smax_i = st.smax[t];
                smin_i = st.smin[t];
                op = st.opacity[t];
                level_i = st.level[t];
            } else {
                m[0] = sc.mean[3 * i];
                m[1] = sc.mean[3 * i + 1];
                m[2] = sc.mean[3 * i + 2];
                sv[0] = sc.scale[3 * i];
                sv[1] = sc.scale[3 * i + 1];
                sv[2] = sc.scale[3 * i + 2];
                q = reinterpret_cast<const float4 *>(sc.quat)[i];
                lnop_i = sc.lnop[i];
                smax_i = sc.s_max[i];
                smin_i = sc.s_min[i];
                op = sc.opacity[i];
                level_i = sc.level[i];
            }
            cov_ok = cov3d(sv, q, S6);
        } else {
#pragma unroll
            for (int k = 0; k < 6; k++) S6[k] = 0.0f;
        }
        // the views whose exact footprint is needed
        float tz, xr, yr;
        view_point(m, s_cam[0], tz, xr, yr);
        CoverBound cb;
        cover_bound(tz, xr, yr, S6, cov_ok, lnop_i, s_cam[0], cb);
        uint32_t need = 0u;
        if (in)
            for (int v = 0; v < nv; v++)
                if (!(cb.ok && surely_unselected(cb, pv.fx2[v], pv.fy2[v], s_cam[v], level_i,
                                                 sc.n_levels, smax_i, smin_i)))
                    need |= 1u << v;
        // the colour, evaluated once towards the centre every view shares,
        // for a Gaussian that some view may list
        float3 col = make_float3(0.0f, 0.0f, 0.0f);
        if (need)
            col = gaussian_color(sc.color, sc.sh_degree, i, m[0] - s_cam[0].campos[0],
                                 m[1] - s_cam[0].campos[1], m[2] - s_cam[0].campos[2]);
        const int lc = level_i | (cov_ok ? 0x100 : 0);
        // every pair's tile count, depth key and empty rectangle first, in
        // whole-warp stores (full DRAM sectors); the pairs that need a
        // footprint overwrite theirs below
        const uint32_t depth_key = __float_as_uint(tz);
        if (in)
            for (int v = 0; v < nv; v++) {
                const ProjOut &o = pv.out[v];
                o.n_tiles[i] = 0u;
                o.depth[i] = depth_key;
                o.rect[i] = make_uint2(0u, 0xffffffffu);
            }
        // pack the warp's (Gaussian, view) pairs, view by view
        int total = 0;
        for (int v = 0; v < nv; v++) {
            const uint32_t bl = __ballot_sync(0xffffffffu, (need >> v) & 1u);
            if (lane == 0) {
                s_vlanes[warp][v] = bl;
                s_voff[warp][v] = total;
            }
            total += __popc(bl);
        }
        __syncwarp();
        for (int k0 = 0; k0 < total; k0 += 32) {
            const int k = k0 + lane;
            const bool act = k < total;
            int v = 0;
            for (int u = 1; u < nv; u++)
                if (k >= s_voff[warp][u]) v = u;
            const int src = act ? nth_set_bit(s_vlanes[warp][v], k - s_voff[warp][v]) : lane;
            float ss[6];
#pragma unroll
            for (int j = 0; j < 6; j++) ss[j] = __shfl_sync(0xffffffffu, S6[j], src);
            const float ptz = __shfl_sync(0xffffffffu, tz, src);
            const float pxr = __shfl_sync(0xffffffffu, xr, src);
            const float pyr = __shfl_sync(0xffffffffu, yr, src);
            const float L = __shfl_sync(0xffffffffu, lnop_i, src);
            const float smx = __shfl_sync(0xffffffffu, smax_i, src);
            const float smn = __shfl_sync(0xffffffffu, smin_i, src);
            const float opv = __shfl_sync(0xffffffffu, op, src);
            const float cr = __shfl_sync(0xffffffffu, col.x, src);
            const float cg = __shfl_sync(0xffffffffu, col.y, src);
            const float cbl = __shfl_sync(0xffffffffu, col.z, src);
            const int plc = __shfl_sync(0xffffffffu, lc, src);
            bool listed = false;
            uint32_t nt = 0u;
            if (act) {
                const int lev = plc & 0xff;
                const bool cok = (plc & 0x100) != 0;
                const ProjOut &o = s_out[v];
                const int64_t gi = base + warp * 32 + src;
                Foot f;
                footprint_vp(ptz, pxr, pyr, ss, cok, L, s_cam[v], f);
                const bool sel = f.valid && select_pred(f.S, lev, sc.n_levels, smx, smn, MS_SELECTIVE);
                listed = sel && f.ntiles > 0;
                nt = listed ? f.ntiles : 0u;
                if (listed) {  // the rest keeps the prefilled values
                    o.n_tiles[gi] = nt;
                    o.rect[gi] = make_uint2((uint32_t)f.x0 | ((uint32_t)f.y0 << 16),
                                            (uint32_t)f.x1 | ((uint32_t)f.y1 << 16));
                    o.rec[3 * gi + 0] = make_float4(f.ux, f.uy, fm(kConicA, f.ca), fm(kConicB, f.cb));
                    o.rec[3 * gi + 1] = make_float4(fm(kConicA, f.cc), opv, cr, cg);
                    o.rec[3 * gi + 2] = make_float4(cbl, fm(-kLog2e, L), f.ex, f.ey);
#pragma unroll
                    for (int p = 0; p < 4; p++) {
                        const uint32_t d = (f.depth >> (8 * p)) & 255u;
                        atomicAdd(&s_hist[v][p][d >> 1], 1u << (16 * (d & 1u)));
                    }
                }
                const uint32_t fl = (sel ? 1u << v : 0u) | (listed ? 1u << (8 + v) : 0u);
                if (fl) atomicOr(&s_bits[warp * 32 + src], fl);
            }
            // survivor and duplicate counts of the round's views (its pairs
            // are in view order, so one contiguous range of views)
            const int vlo = __shfl_sync(0xffffffffu, v, 0);
            const int vhi = __shfl_sync(0xffffffffu, v, min(31, total - 1 - k0));
            for (int u = vlo; u <= vhi; u++) {
                const bool mine = act && v == u;
                const uint32_t ws = __reduce_add_sync(0xffffffffu, mine && listed ? 1u : 0u);
                const uint32_t wd = __reduce_add_sync(0xffffffffu, mine ? nt : 0u);
                if (lane == 0 && ws) {
                    atomicAdd(&s_surv[u], ws);
                    atomicAdd(&s_dup[u], (unsigned long long)wd);
                }
            }
        }
        __syncwarp();
        const uint32_t bits = s_bits[t];
        s_bits[t] = 0u;
        for (int v = 0; v < nv; v++) {
            const ProjOut &o = pv.out[v];
            if (o.mask) {
                const uint32_t mb = __ballot_sync(0xffffffffu, in && ((bits >> v) & 1u));
                if (lane == 0 && in) o.mask[i >> 5] = mb;
            }
        }
        if (pv.union_flags) {
            const uint32_t umask = (bits >> 8) & pv.union_mask;
            const bool any_listed = umask != 0u;
            if (in) pv.union_flags[i] = umask;
            if (any_listed) {
#pragma unroll
                for (int p = 0; p < 4; p++) {
                    const uint32_t d = (depth_key >> (8 * p)) & 255u;
                    atomicAdd(&s_hist[MAXV][p][d >> 1], 1u << (16 * (d & 1u)));
                }
            }
            const uint32_t wu = __reduce_add_sync(0xffffffffu, any_listed ? 1u : 0u);
            if (lane == 0 && wu) atomicAdd(&s_surv[MAXV], wu);
        }
        __syncthreads();  // the buffer is refilled by the next iteration but one
        if ((it + 1) % kHistFlushChunks == 0) {
            flush_hist<MAXV>(s_hist, pv);
            __syncthreads();
        }
    }
    flush_hist<MAXV>(s_hist, pv);
    __syncthreads();
    if (threadIdx.x < nv) {
        const int v = threadIdx.x;
        uint32_t *stats = pv.out[v].stats;
        if (s_surv[v]) atomicAdd(&stats[kStatSurvivors], s_surv[v]);
        if (s_dup[v]) atomicAdd(reinterpret_cast<unsigned long long *>(stats + kStatDup), s_dup[v]);
    }
    if (pv.union_stats && threadIdx.x == 0 && s_surv[MAXV])
        atomicAdd(&pv.union_stats[kStatSurvivors], s_surv[MAXV]);
}

__global__ void select_kernel(int64_t n, const float *__restrict__ cover,
                              const uint8_t *__restrict__ level, int n_levels,
                              const float *__restrict__ smax,
                              const float *__restrict__ smin, int mode,
                              uint32_t *__restrict__ mask) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        int64_t i = base + threadIdx.x;
        bool sel = false;
        if (i < n) {
            float S = cover[i];
            sel = (S >= 0.0f) && select_pred(S, level[i], n_levels, smax[i], smin[i], mode);
        }
        uint32_t bits = __ballot_sync(0xffffffffu, sel);
        if ((threadIdx.x & 31) == 0 && i < n) mask[i >> 5] = bits;
    }
}

// Eq. 5: S_max' = max(0.95 S_max, S), S_min' = min(1.05 S_min, S) for the
// Gaussians of level_r that are valid and touch the image.
__global__ void update_range_kernel(SceneK sc, CamK cam, int level_r,
                                    float *__restrict__ smax,
                                    float *__restrict__ smin) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sc.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (sc.level[i] != level_r) continue;
        float m[3] = {sc.mean[3 * i], sc.mean[3 * i + 1], sc.mean[3 * i + 2]};
        float s[3] = {sc.scale[3 * i], sc.scale[3 * i + 1], sc.scale[3 * i + 2]};
        float4 q = reinterpret_cast<const float4 *>(sc.quat)[i];
        Foot f;
        footprint(m, s, q, sc.lnop[i], cam, f);
        if (!f.valid || f.ntiles == 0) continue;
        smax[i] = fmaxf(fm(0.95f, smax[i]), f.S);
        smin[i] = fminf(fm(1.05f, smin[i]), f.S);
    }
}

}  // namespace msgs

using namespace msgs;

extern "C" int ms_scene_prepare(const ms_scene_t *scene, void *stream) {
    if (!scene) return fail(MS_ERR_INVALID_ARG, "scene is NULL");
    if (scene->n < 0 || scene->n > INT32_MAX) return fail(MS_ERR_INVALID_ARG, "scene n out of range");
    if (scene->n == 0) return MS_OK;
    if (!scene->log_scale || !scene->opacity || !scene->scale || !scene->lnop)
        return fail(MS_ERR_INVALID_ARG, "scene log_scale/opacity/scale/lnop is NULL");
    prepare_kernel<<<grid_for(scene->n, 256, 8), 256, 0, as_stream(stream)>>>(
        scene->n, scene->log_scale, scene->opacity, scene->scale, scene->lnop);
    return cuda_check(cudaGetLastError(), "prepare_kernel launch");
}

namespace msgs {
namespace {

int check_proj_out(const ms_scene_t *scene, const ms_proj_t *out) {
    if (!out || !out->rec || !out->rect || !out->n_tiles || !out->depth || !out->stats)
        return fail(MS_ERR_INVALID_ARG, "ms_proj_t has a NULL required buffer");
    if (out->n < scene->n) return fail(MS_ERR_INVALID_ARG, "ms_proj_t holds fewer Gaussians than the scene");
    if (!aligned(out->rec, 16) || !aligned(out->rect, 8) || !aligned(out->stats, 16))
        return fail(MS_ERR_INVALID_ARG, "rec must be 16-B, rect 8-B, stats 16-B aligned");
    return MS_OK;
}

template <int MAXV>
int launch_project(const ms_scene_t *scene, const ms_camera_t *cams, int nv, ms_mode_t mode,
                   const ms_proj_t *outs, const int32_t *update_levels, uint32_t *union_flags,
                   uint32_t *union_stats, uint32_t union_mask, cudaStream_t st) {
    ProjViews<MAXV> pv;
    pv.n_views = nv;
    pv.union_flags = union_flags;
    pv.union_stats = union_stats;
    pv.union_mask = union_mask;
    pv.union_first = 0;
    while (pv.union_first < nv - 1 && !((union_mask >> pv.union_first) & 1u)) pv.union_first++;
    pv.smax_out = scene->s_max;
    pv.smin_out = scene->s_min;
    for (int v = 0; v < MAXV; v++) {
        pv.update_level[v] = (update_levels && v < nv) ? update_levels[v] : 0;
        const int u = v < nv ? v : 0;
        pv.cam[v] = make_cam(cams[u]);
        const ms_proj_t &o = outs[u];
        pv.out[v] = ProjOut{reinterpret_cast<float4 *>(o.rec), reinterpret_cast<uint2 *>(o.rect),
                            o.n_tiles, o.depth, o.cover, o.mask, o.stats};
        pv.color_src[v] = v;
        for (int w = 0; w < v && v < nv; w++)
            if (std::memcmp(cams[w].campos, cams[v].campos, sizeof(cams[v].campos)) == 0) {
                pv.color_src[v] = w;
                break;
            }
    }
    // bulk staging needs every geometry array 16-byte aligned
    const bool staged_ok = aligned(scene->mean, 16) && aligned(scene->scale, 16) &&
                           aligned(scene->quat, 16) && aligned(scene->lnop, 16) &&
                           aligned(scene->s_max, 16) && aligned(scene->s_min, 16) &&
                           aligned(scene->opacity, 16) && aligned(scene->level, 16);
    // selective views of one pose without coverage output or range updates
    // leave out the footprints their coverage bound rules out
    bool prune = MAXV > 1 && nv >= 2 && mode == MS_SELECTIVE;
    for (int v = 0; v < nv && prune; v++)
        prune = !outs[v].cover && pv.update_level[v] == 0 && pv.color_src[v] == 0 &&
                std::memcmp(cams[v].R, cams[0].R, sizeof(cams[0].R)) == 0 &&
                std::memcmp(cams[v].t, cams[0].t, sizeof(cams[0].t)) == 0;
    for (int v = 0; v < MAXV; v++) {
        const ms_camera_t &c = cams[v < nv ? v : 0];
        pv.fx2[v] = (float)((double)c.fx * (double)c.fx);
        pv.fy2[v] = (float)((double)c.fy * (double)c.fy);
    }
    const int grid = grid_for(scene->n, kProjThreads, proj_blocks_per_sm<MAXV>());
    if constexpr (MAXV > 1) {
        if (prune) {
            project_pruned_kernel<MAXV><<<grid, kProjThreads, 0, st>>>(make_scene(*scene), pv,
                                                                      staged_ok);
            return cuda_check(cudaGetLastError(), "project_pruned_kernel launch");
        }
    }
    project_kernel<MAXV><<<grid, kProjThreads, 0, st>>>(make_scene(*scene), pv, (int)mode,
                                                       staged_ok);
    return cuda_check(cudaGetLastError(), "project_kernel launch");
}

}  // namespace
}  // namespace msgs

namespace msgs {
namespace {

int project_views(const ms_scene_t *scene, const ms_camera_t *cams, int32_t n_views,
                  ms_mode_t mode, const int32_t *update_levels, const ms_proj_t *outs,
                  uint32_t *union_flags, uint32_t *union_stats, uint32_t union_mask,
                  void *stream) {
    int rc = check_scene(scene, true);
    if (rc) return rc;
    if (n_views < 1 || n_views > MS_MAX_PROJ_VIEWS)
        return fail(MS_ERR_INVALID_ARG, "n_views must be 1..MS_MAX_PROJ_VIEWS");
    if (!cams || !outs) return fail(MS_ERR_INVALID_ARG, "cams/outs is NULL");
    if (mode != MS_SELECTIVE && mode != MS_ALL_LEVELS && mode != MS_FILTER_SMALL)
        return fail(MS_ERR_INVALID_ARG, "unknown mode");
    for (int v = 0; v < n_views; v++) {
        if ((rc = check_cam(&cams[v]))) return rc;
        if ((rc = check_proj_out(scene, &outs[v]))) return rc;
        if (update_levels && (update_levels[v] < 0 || update_levels[v] > scene->n_levels))
            return fail(MS_ERR_INVALID_ARG, "update_levels[v] must be 0..n_levels");
    }
    cudaStream_t st = as_stream(stream);
    for (int v = 0; v < n_views; v++)
        if ((rc = cuda_check(cudaMemsetAsync(outs[v].stats, 0, MS_STATS_WORDS * sizeof(uint32_t), st),
                             "stats memset")))
            return rc;
    if (union_stats &&
        (rc = cuda_check(cudaMemsetAsync(union_stats, 0, MS_STATS_WORDS * sizeof(uint32_t), st),
                         "union stats memset")))
        return rc;
    if (scene->n == 0) return MS_OK;
    if (n_views == 1 && !union_flags)
        return launch_project<1>(scene, cams, 1, mode, outs, update_levels, nullptr, nullptr, 0u,
                                 st);
    return launch_project<MS_MAX_PROJ_VIEWS>(scene, cams, n_views, mode, outs, update_levels,
                                             union_flags, union_stats, union_mask, st);
}

}  // namespace
}  // namespace msgs

extern "C" int ms_project_views_update(const ms_scene_t *scene, const ms_camera_t *cams,
                                       int32_t n_views, ms_mode_t mode,
                                       const int32_t *update_levels, const ms_proj_t *outs,
                                       void *stream) {
    return project_views(scene, cams, n_views, mode, update_levels, outs, nullptr, nullptr, 0u,
                         stream);
}

extern "C" int ms_project_views_union(const ms_scene_t *scene, const ms_camera_t *cams,
                                      int32_t n_views, ms_mode_t mode, const ms_proj_t *outs,
                                      uint32_t union_views, uint32_t *union_flags,
                                      uint32_t *union_stats, void *stream) {
    if (!union_flags || !union_stats || !aligned(union_stats, 16))
        return fail(MS_ERR_INVALID_ARG, "union_flags / union_stats NULL or stats misaligned");
    if (!cams || n_views < 1 || n_views > MS_MAX_PROJ_VIEWS)
        return fail(MS_ERR_INVALID_ARG, "cams is NULL or n_views not 1..MS_MAX_PROJ_VIEWS");
    if (union_views == 0 || (union_views >> n_views) != 0)
        return fail(MS_ERR_INVALID_ARG, "union_views must name 1 or more of the n_views views");
    int first = 0;
    while (!((union_views >> first) & 1u)) first++;
    for (int v = first + 1; v < n_views; v++)
        if (((union_views >> v) & 1u) &&
            (std::memcmp(cams[v].R, cams[first].R, sizeof(cams[0].R)) != 0 ||
             std::memcmp(cams[v].t, cams[first].t, sizeof(cams[0].t)) != 0))
            return fail(MS_ERR_INVALID_ARG,
                        "the union needs one pose: the R and t of its views equal, bitwise");
    return project_views(scene, cams, n_views, mode, nullptr, outs, union_flags, union_stats,
                         union_views, stream);
}

extern "C" int ms_project_views(const ms_scene_t *scene, const ms_camera_t *cams,
                                int32_t n_views, ms_mode_t mode, const ms_proj_t *outs,
                                void *stream) {
    return ms_project_views_update(scene, cams, n_views, mode, nullptr, outs, stream);
}

extern "C" int ms_project(const ms_scene_t *scene, const ms_camera_t *cam,
                          ms_mode_t mode, const ms_proj_t *out, void *stream) {
    return ms_project_views(scene, cam, 1, mode, out, stream);
}

extern "C" int ms_select(const ms_scene_t *scene, const float *cover, ms_mode_t mode,
                         uint32_t *mask, void *stream) {
    int rc = check_scene(scene, false);
    if (rc) return rc;
    if (mode != MS_SELECTIVE && mode != MS_ALL_LEVELS && mode != MS_FILTER_SMALL)
        return fail(MS_ERR_INVALID_ARG, "unknown mode");
    if (scene->n == 0) return MS_OK;
    if (!cover || !mask) return fail(MS_ERR_INVALID_ARG, "cover/mask is NULL");
    select_kernel<<<grid_for(scene->n, 256, 8), 256, 0, as_stream(stream)>>>(
        scene->n, cover, scene->level, scene->n_levels, scene->s_max, scene->s_min, (int)mode,
        mask);
    return cuda_check(cudaGetLastError(), "select_kernel launch");
}

extern "C" int ms_update_range(const ms_scene_t *scene, const ms_camera_t *cam,
                               int32_t level_r, void *stream) {
    int rc = check_scene(scene, true);
    if (rc) return rc;
    if ((rc = check_cam(cam))) return rc;
    if (scene->n == 0) return MS_OK;
    if (level_r < 1 || level_r > scene->n_levels)
        return fail(MS_ERR_INVALID_ARG, "level_r must be in 1..n_levels");
    update_range_kernel<<<grid_for(scene->n, 256, 8), 256, 0, as_stream(stream)>>>(
        make_scene(*scene), make_cam(*cam), level_r, scene->s_max, scene->s_min);
    return cuda_check(cudaGetLastError(), "update_range_kernel launch");
}

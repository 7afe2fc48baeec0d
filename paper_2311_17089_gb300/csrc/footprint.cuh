// The FP32 footprint of one Gaussian in one camera (the operations of the
// footprint definition in a fixed order with single-rounding intrinsics, so
// validity, coverage, depth keys and tile rectangles are reproducible
// bit-for-bit), and the scene/camera views the per-Gaussian kernels share.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

namespace msgs {

struct CamK {
    float W[9], t[3], campos[3];
    float fx, fy, cx, cy, near_plane;
    float limx, limy;  // 1.3 x the half field of view as view ratios
    int width, height, tiles_x, tiles_y;
};

inline CamK make_cam(const ms_camera_t &c) {
    CamK k;
    for (int i = 0; i < 9; i++) k.W[i] = c.R[i];
    for (int i = 0; i < 3; i++) {
        k.t[i] = c.t[i];
        k.campos[i] = c.campos[i];
    }
    k.fx = c.fx;
    k.fy = c.fy;
    k.cx = c.cx;
    k.cy = c.cy;
    k.near_plane = c.near_plane;
    // the Jacobian's clamp limits, once per camera: the same single-precision
    // operations, in the same order, as every Gaussian would perform (host
    // float arithmetic is IEEE single precision, and no product here can be
    // contracted into an FMA)
    const volatile float hw = 0.5f * (float)c.width, hh = 0.5f * (float)c.height;
    const volatile float qx = hw / c.fx, qy = hh / c.fy;
    k.limx = 1.3f * qx;
    k.limy = 1.3f * qy;
    k.width = c.width;
    k.height = c.height;
    k.tiles_x = (c.width + 15) / 16;
    k.tiles_y = (c.height + 15) / 16;
    return k;
}

struct Foot {
    bool valid;
    float S, ux, uy, ca, cb, cc, ex, ey;
    uint32_t depth;
    int x0, y0, x1, y1;
    uint32_t ntiles;
};

__device__ __forceinline__ bool fin(float v) { return isfinite(v); }

// The view-independent part of the footprint (Sec. 3.1): the 3D covariance
// Sigma = R S S^T R^T of the Gaussian, R from the normalised quaternion q,
// as its six distinct entries (xx, xy, xz, yy, yz, zz).  False when q has
// no finite positive norm (the Gaussian is then invalid in every view).
__device__ __forceinline__ bool cov3d(const float s[3], float4 q, float S6[6]) {
    float n2 = fa(fa(fa(fm(q.x, q.x), fm(q.y, q.y)), fm(q.z, q.z)), fm(q.w, q.w));
    if (!(n2 > 0.0f) || !fin(n2)) {
#pragma unroll
        for (int k = 0; k < 6; k++) S6[k] = 0.0f;
        return false;
    }
    float rn = fdv(1.0f, fsq(n2));
    float w = fm(q.x, rn), x = fm(q.y, rn), y = fm(q.z, rn), z = fm(q.w, rn);
    float xx = fm(x, x), yy = fm(y, y), zz = fm(z, z);
    float xy = fm(x, y), xz = fm(x, z), yz = fm(y, z);
    float wx = fm(w, x), wy = fm(w, y), wz = fm(w, z);
    float R[9];
    R[0] = fs(1.0f, fm(2.0f, fa(yy, zz)));
    R[1] = fm(2.0f, fs(xy, wz));
    R[2] = fm(2.0f, fa(xz, wy));
    R[3] = fm(2.0f, fa(xy, wz));
    R[4] = fs(1.0f, fm(2.0f, fa(xx, zz)));
    R[5] = fm(2.0f, fs(yz, wx));
    R[6] = fm(2.0f, fs(xz, wy));
    R[7] = fm(2.0f, fa(yz, wx));
    R[8] = fs(1.0f, fm(2.0f, fa(xx, yy)));
    float M[9];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int k = 0; k < 3; k++) M[3 * r + k] = fm(R[3 * r + k], s[k]);
    int j = 0;
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int k = r; k < 3; k++)
            S6[j++] = fa(fa(fm(M[3 * r], M[3 * k]), fm(M[3 * r + 1], M[3 * k + 1])),
                         fm(M[3 * r + 2], M[3 * k + 2]));
    return true;
}

// The view-space point of a mean in camera c: depth tz and the view ratios
// xr = tx / tz, yr = ty / tz (the first steps of the footprint; cameras of
// one pose give the same bits).
__device__ __forceinline__ void view_point(const float m[3], const CamK &c, float &tz, float &xr,
                                           float &yr) {
    const float *W = c.W;
    const float tx = fa(fa(fa(fm(W[0], m[0]), fm(W[1], m[1])), fm(W[2], m[2])), c.t[0]);
    const float ty = fa(fa(fa(fm(W[3], m[0]), fm(W[4], m[1])), fm(W[5], m[2])), c.t[1]);
    tz = fa(fa(fa(fm(W[6], m[0]), fm(W[7], m[1])), fm(W[8], m[2])), c.t[2]);
    xr = fdv(tx, tz);
    yr = fdv(ty, tz);
}

// FP32 footprint in one camera (Sec. 3.1 EWA splat, Eq. 4 dilation by
// 0.3 px^2, Sec. 4.1 pixel coverage, Sec. 3.1 16x16 tiles) from the
// view-space point (view_point), the 3D covariance of cov3d (cov_ok its
// result) and L = ln(255 sigma).
__device__ __forceinline__ void footprint_vp(float tz, float xr, float yr, const float S6[6],
                                             bool cov_ok, float L, const CamK &c, Foot &o) {
    o.valid = false;
    o.S = -1.0f;
    o.ntiles = 0;
    o.x0 = o.y0 = 0;
    o.x1 = o.y1 = -1;
    o.depth = __float_as_uint(tz);
    if (!(L > 0.0f) || !fin(L) || !(tz > c.near_plane) || !fin(tz) || !cov_ok) return;
    const float *W = c.W;
    const float S3[9] = {S6[0], S6[1], S6[2], S6[1], S6[3], S6[4], S6[2], S6[4], S6[5]};
    const float limx = c.limx, limy = c.limy;
    float xc = fminf(limx, fmaxf(-limx, xr));
    float yc = fminf(limy, fmaxf(-limy, yr));
    float J00 = fdv(c.fx, tz);
    float J02 = fdv(-fm(c.fx, xc), tz);
    float J11 = fdv(c.fy, tz);
    float J12 = fdv(-fm(c.fy, yc), tz);
    float T[6];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        T[k] = fa(fm(J00, W[k]), fm(J02, W[6 + k]));
        T[3 + k] = fa(fm(J11, W[3 + k]), fm(J12, W[6 + k]));
    }
    float U[6];
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
        for (int k = 0; k < 3; k++)
            U[3 * r + k] = fa(fa(fm(T[3 * r], S3[k]), fm(T[3 * r + 1], S3[3 + k])),
                              fm(T[3 * r + 2], S3[6 + k]));
    float V00 = fa(fa(fm(U[0], T[0]), fm(U[1], T[1])), fm(U[2], T[2]));
    float V01 = fa(fa(fm(U[0], T[3]), fm(U[1], T[4])), fm(U[2], T[5]));
    float V11 = fa(fa(fm(U[3], T[3]), fm(U[4], T[4])), fm(U[5], T[5]));
    float a = fa(V00, 0.3f), b = V01, cc = fa(V11, 0.3f);
    float detd = fs(fm(a, cc), fm(b, b));
    float ux = fa(fm(c.fx, xr), c.cx);
    float uy = fa(fm(c.fy, yr), c.cy);
    if (!fin(V00) || !fin(V01) || !fin(V11) || !(detd > 0.0f) || !fin(detd) ||
        !fin(ux) || !fin(uy))
        return;
    o.valid = true;
    float det = fs(fm(V00, V11), fm(V01, V01));
    float mx = fmaxf(V00, V11);
    float S = 0.0f;
    if (det > 0.0f && mx > 0.0f) S = fsq(fdv(fm(fm(8.0f, L), det), mx));
    o.S = S;
    o.ux = ux;
    o.uy = uy;
    o.ca = fdv(cc, detd);
    o.cb = fdv(-b, detd);
    o.cc = fdv(a, detd);
    float ex = fsq(fm(fm(2.0f, L), a));
    float ey = fsq(fm(fm(2.0f, L), cc));
    o.ex = ex;
    o.ey = ey;
    float x0 = floorf(fm(fs(ux, ex), 0.0625f)), x1 = floorf(fm(fa(ux, ex), 0.0625f));
    float y0 = floorf(fm(fs(uy, ey), 0.0625f)), y1 = floorf(fm(fa(uy, ey), 0.0625f));
    x0 = fmaxf(x0, 0.0f);
    y0 = fmaxf(y0, 0.0f);
    x1 = fminf(x1, (float)(c.tiles_x - 1));
    y1 = fminf(y1, (float)(c.tiles_y - 1));
    if (x0 <= x1 && y0 <= y1) {
        o.x0 = (int)x0;
        o.y0 = (int)y0;
        o.x1 = (int)x1;
        o.y1 = (int)y1;
        o.ntiles = (uint32_t)((o.x1 - o.x0 + 1) * (o.y1 - o.y0 + 1));
    }
}

// The footprint from the mean.
__device__ __forceinline__ void footprint_cov(const float m[3], const float S6[6], bool cov_ok,
                                              float L, const CamK &c, Foot &o) {
    float tz, xr, yr;
    view_point(m, c, tz, xr, yr);
    footprint_vp(tz, xr, yr, S6, cov_ok, L, c, o);
}

// The footprint of one Gaussian in one camera.
__device__ __forceinline__ void footprint(const float m[3], const float s[3], float4 q,
                                          float L, const CamK &c, Foot &o) {
    float S6[6];
    const bool ok = cov3d(s, q, S6);
    footprint_cov(m, S6, ok, L, c, o);
}

// A bound on the pixel coverage S of one Gaussian in every camera of one
// pose (R, t), without that camera's footprint.  The pose fixes the
// view-space mean (tx, ty, tz) and the view ratios (xr, yr); where the
// Jacobian's clamp leaves them unchanged, a camera with focal lengths
// (fx, fy) has J = diag(fx, fy) J1, J1 the Jacobian for unit focal
// lengths, so its undilated 2D covariance is V = diag(fx, fy) V1 diag(fx, fy)
// and S^2 = 8 L fx^2 fy^2 det V1 / max(fx^2 V1_xx, fy^2 V1_yy).
// Error bound (u = 2^-24): the FP32 chain J -> J W -> J W Sigma ->
// J W Sigma W^T J^T leaves each entry of V within 20u of the same product
// taken over absolute values (|J||W| |Sigma| |W|^T|J|^T = Va; 16u for the
// footprint's correctly rounded Jacobian, 20u for V1's, whose 1 / tz comes
// from the approximate reciprocal), so det V is within
// 50u (Va_xx Va_yy + Va_xy^2) and max(V_xx, V_yy) within
// 20u max(Va_xx / V_xx, Va_yy / V_yy) relative; with the last few roundings
// S^2 from the camera's own fixed-order footprint and S^2 from V1 below
// each lie within eps = u (50 P / det + 20 q + 8) of the exact value
// (P, q those ratios' terms, the same for every camera of the pose), so
// within 2 eps (1 + eps) of each other.  The bound is kept only where V1 is
// well conditioned (eps < 1e-3; P / det and q need only a few correct
// digits); mu2 = 1 + 4 eps + 1e-6 covers the rest of the rounding of the
// comparisons.
struct CoverBound {
    bool ok;           // the bound holds
    float tz, xr, yr;  // view-space depth and view ratios of the pose
    float s2_unit;     // 8 L det V1
    float v00, v11;    // diagonal of V1
    float mu2;         // margin on squared coverage
};

__device__ __forceinline__ void cover_bound(float tz, float xr, float yr, const float S6[6],
                                            bool cov_ok, float L, const CamK &c, CoverBound &b) {
    const float *W = c.W;
    b.ok = false;
    b.tz = tz;
    b.xr = xr;
    b.yr = yr;
    if (!cov_ok || !(L > 0.0f) || !fin(L) || !(tz > 0.0f) || !fin(tz) || !fin(xr) || !fin(yr))
        return;
    const float r = __fdividef(1.0f, tz);
    const float j2 = -xr * r, k2 = -yr * r;  // J1 = [[r, 0, j2], [0, r, k2]]
    float T0[3], T1[3], A0[3], A1[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        T0[k] = r * W[k] + j2 * W[6 + k];
        T1[k] = r * W[3 + k] + k2 * W[6 + k];
        A0[k] = fabsf(r * W[k]) + fabsf(j2 * W[6 + k]);
        A1[k] = fabsf(r * W[3 + k]) + fabsf(k2 * W[6 + k]);
    }
    const float S3[9] = {S6[0], S6[1], S6[2], S6[1], S6[3], S6[4], S6[2], S6[4], S6[5]};
    float U0[3], U1[3], B0[3], B1[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        U0[k] = T0[0] * S3[k] + T0[1] * S3[3 + k] + T0[2] * S3[6 + k];
        U1[k] = T1[0] * S3[k] + T1[1] * S3[3 + k] + T1[2] * S3[6 + k];
        B0[k] = A0[0] * fabsf(S3[k]) + A0[1] * fabsf(S3[3 + k]) + A0[2] * fabsf(S3[6 + k]);
        B1[k] = A1[0] * fabsf(S3[k]) + A1[1] * fabsf(S3[3 + k]) + A1[2] * fabsf(S3[6 + k]);
    }
    const float v00 = U0[0] * T0[0] + U0[1] * T0[1] + U0[2] * T0[2];
    const float v01 = U0[0] * T1[0] + U0[1] * T1[1] + U0[2] * T1[2];
    const float v11 = U1[0] * T1[0] + U1[1] * T1[1] + U1[2] * T1[2];
    const float a00 = B0[0] * A0[0] + B0[1] * A0[1] + B0[2] * A0[2];
    const float a01 = B0[0] * A1[0] + B0[1] * A1[1] + B0[2] * A1[2];
    const float a11 = B1[0] * A1[0] + B1[1] * A1[1] + B1[2] * A1[2];
    const float det = v00 * v11 - v01 * v01;
    if (!(det > 0.0f) || !(v00 > 0.0f) || !(v11 > 0.0f)) return;
    const float P = a00 * a11 + a01 * a01;
    const float q = fmaxf(__fdividef(a00, v00), __fdividef(a11, v11));
    const float eps = 5.9604645e-8f * (50.0f * __fdividef(P, det) + 20.0f * q + 8.0f);
    if (!(eps < 1e-3f)) return;  // also false for NaN and infinity
    b.s2_unit = 8.0f * L * det;
    b.v00 = v00;
    b.v11 = v11;
    b.mu2 = 1.0f + 4.0f * eps + 1e-6f;
    b.ok = fin(b.s2_unit) && b.s2_unit > 0.0f;
}

// True only if the camera (focal lengths squared fx2, fy2; the pose of the
// bound) is sure to reject the Gaussian in selective mode (Eq. 6 with the
// exemptions of Sec. 4.1): too large for a level above the finest, or too
// small for a level below the coarsest, by more than the bound's margin.
// False where the camera's clamp would change the view ratios.
__device__ __forceinline__ bool surely_unselected(const CoverBound &b, float fx2, float fy2,
                                                  const CamK &c, int level, int n_levels,
                                                  float smax, float smin) {
    if (!(fabsf(b.xr) <= c.limx) || !(fabsf(b.yr) <= c.limy)) return false;
    // S^2 = num / den, compared without dividing
    const float num = b.s2_unit * fx2 * fy2, den = fmaxf(fx2 * b.v00, fy2 * b.v11);
    if (!fin(num) || !(den > 0.0f) || !fin(den)) return false;
    const float lo = num * (2.0f - b.mu2), hi = num * b.mu2;
    if (level != 1 && smax > 0.0f && fin(smax) && lo > 2.25f * smax * smax * den) return true;
    if (level != n_levels && smin > 0.0f && fin(smin) && hi < 4.0f * den &&
        hi < 0.25f * smin * smin * den)
        return true;
    return false;
}

struct SceneK {
    int64_t n;
    int n_levels, sh_degree;
    const float *mean, *quat, *opacity, *color, *scale, *lnop;
    const uint8_t *level;
    const float *s_max, *s_min;
};

inline SceneK make_scene(const ms_scene_t &s) {
    SceneK k;
    k.n = s.n;
    k.n_levels = s.n_levels;
    k.sh_degree = s.sh_degree;
    k.mean = s.mean;
    k.quat = s.quat;
    k.opacity = s.opacity;
    k.color = s.color;
    k.scale = s.scale;
    k.lnop = s.lnop;
    k.level = s.level;
    k.s_max = s.s_max;
    k.s_min = s.s_min;
    return k;
}

// ------------------------------------------------------- argument checks

inline int check_scene(const ms_scene_t *s, bool need_prepared) {
    if (!s) return fail(MS_ERR_INVALID_ARG, "scene is NULL");
    if (s->n < 0 || s->n > INT32_MAX) return fail(MS_ERR_INVALID_ARG, "scene n out of range");
    if (s->n == 0) return MS_OK;
    if (!s->mean || !s->quat || !s->opacity || !s->level)
        return fail(MS_ERR_INVALID_ARG, "scene has a NULL array");
    if (!aligned(s->quat, 16)) return fail(MS_ERR_INVALID_ARG, "quat must be 16-byte aligned");
    if (s->n_levels < 1 || s->n_levels > 255)
        return fail(MS_ERR_INVALID_ARG, "n_levels must be in 1..255");
    if (s->sh_degree < -1 || s->sh_degree > 3)
        return fail(MS_ERR_INVALID_ARG, "sh_degree must be in -1..3");
    if (!s->color) return fail(MS_ERR_INVALID_ARG, "scene color is NULL");
    if (s->sh_degree >= 0 && !aligned(s->color, 16))
        return fail(MS_ERR_INVALID_ARG, "SH coefficients must be 16-byte aligned");
    if (!s->s_max || !s->s_min) return fail(MS_ERR_INVALID_ARG, "s_max/s_min is NULL");
    if (need_prepared && (!s->scale || !s->lnop))
        return fail(MS_ERR_INVALID_ARG, "scene scale/lnop is NULL (run ms_scene_prepare)");
    return MS_OK;
}

inline int check_cam(const ms_camera_t *c) {
    if (!c) return fail(MS_ERR_INVALID_ARG, "camera is NULL");
    if (c->width < 1 || c->height < 1 || c->width > 32768 || c->height > 32768)
        return fail(MS_ERR_INVALID_ARG, "image size must be 1..32768");
    if (!(c->near_plane > 0.0f)) return fail(MS_ERR_INVALID_ARG, "near_plane must be > 0");
    if (!(c->fx > 0.0f) || !(c->fy > 0.0f)) return fail(MS_ERR_INVALID_ARG, "focal length must be > 0");
    return MS_OK;
}

inline int grid_for(int64_t n, int threads, int per_sm) {
    int64_t g = ceil_div(n, threads);
    int64_t cap = (int64_t)num_sms() * per_sm;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace msgs

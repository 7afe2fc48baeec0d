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

// FP32 footprint in one camera (Sec. 3.1 EWA splat, Eq. 4 dilation by
// 0.3 px^2, Sec. 4.1 pixel coverage, Sec. 3.1 16x16 tiles) from the mean,
// the 3D covariance of cov3d (cov_ok its result) and L = ln(255 sigma).
__device__ __forceinline__ void footprint_cov(const float m[3], const float S6[6], bool cov_ok,
                                              float L, const CamK &c, Foot &o) {
    o.valid = false;
    o.S = -1.0f;
    o.ntiles = 0;
    o.x0 = o.y0 = 0;
    o.x1 = o.y1 = -1;
    const float *W = c.W;
    float tx = fa(fa(fa(fm(W[0], m[0]), fm(W[1], m[1])), fm(W[2], m[2])), c.t[0]);
    float ty = fa(fa(fa(fm(W[3], m[0]), fm(W[4], m[1])), fm(W[5], m[2])), c.t[1]);
    float tz = fa(fa(fa(fm(W[6], m[0]), fm(W[7], m[1])), fm(W[8], m[2])), c.t[2]);
    o.depth = __float_as_uint(tz);
    if (!(L > 0.0f) || !fin(L) || !(tz > c.near_plane) || !fin(tz) || !cov_ok) return;
    const float S3[9] = {S6[0], S6[1], S6[2], S6[1], S6[3], S6[4], S6[2], S6[4], S6[5]};
    const float limx = c.limx, limy = c.limy;
    float xr = fdv(tx, tz), yr = fdv(ty, tz);
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

// The footprint of one Gaussian in one camera.
__device__ __forceinline__ void footprint(const float m[3], const float s[3], float4 q,
                                          float L, const CamK &c, Foot &o) {
    float S6[6];
    const bool ok = cov3d(s, q, S6);
    footprint_cov(m, S6, ok, L, c, o);
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

/*
 * FP32 footprint of every Gaussian: EWA projection, pixel coverage,
 * selection and tile rectangle.  TEST INFRASTRUCTURE (see oracle.h).
 *
 * Every floating-point step is one IEEE-754 single-precision operation
 * in the order written (compiled with -ffp-contract=off, no fast-math),
 * so the results are exactly reproducible by any implementation that
 * performs the same operations in the same order.  That fixed order is
 * the contract that makes selection masks and tile lists bit-exact.
 *
 * What is computed, following the paper:
 *   - Sec. 3.1: each 3D Gaussian (centre mu, covariance V-hat) is splatted
 *     to a 2D Gaussian (mu^k, V^k) by the perspective transformation, i.e.
 *     the local affine (Jacobian) approximation of EWA splatting:
 *     V = J W Sigma W^T J^T with Sigma = R diag(s)^2 R^T.
 *   - Sec. 3.2, Eq. 4: the rasterised splat uses V + V^h, V^h a low-pass
 *     filter whose size the paper ties to the screen pixel; it gives no
 *     value, this oracle reads it as 0.3 px^2 on each diagonal entry.
 *   - Sec. 4.1 "Pixel Coverage": S is the smaller of the horizontal and
 *     vertical full widths of the splat at the level set
 *     sigma * G = sigma_T, sigma_T = 1/255, in pixels.  Along x through
 *     the centre, sigma exp(-A x^2 / 2) = sigma_T with A = (V^-1)_xx =
 *     V_yy / det V gives the half width sqrt(2 L / A), L = ln(sigma /
 *     sigma_T).  Taking the smaller full width:
 *         S = sqrt(8 L det(V) / max(V_xx, V_yy)).
 *     The coverage uses the undilated V (with V^h every splat would be at
 *     least 2 sqrt(2 ln 255 * 0.3) = 3.6 px wide and the S >= S_T clause of
 *     Eq. 6 could never fail).  For sigma = 1 this is the supplementary's
 *     1-D result S = 2 sqrt(ln N / a) along each axis.
 *   - Eq. 6 and the paragraph after it: selected iff
 *         (S / S_max <= 1.5) and (S / S_min >= 0.5 or S >= S_T = 2),
 *     except that the finest level skips the first clause and the
 *     coarsest level skips the second.
 *   - Sec. 3.1: the image is divided into 16x16 tiles; a Gaussian is binned
 *     to every tile its level-set bounding box {sigma G >= sigma_T}
 *     touches.  The box of the dilated ellipse d^T V'^-1 d <= 2 L has half
 *     widths sqrt(2 L V'_xx), sqrt(2 L V'_yy).
 *
 * Inputs `scale` = exp(log_scale) and `lnop` = ln(255 sigma) are the
 * view-independent activations made once per scene by or_prepare (FP64,
 * then rounded to FP32), so no transcendental function enters the
 * per-view footprint.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

void or_prepare(int64_t n, const float *log_scale, const float *opacity,
                float *scale, float *lnop)
{
    for (int64_t i = 0; i < n; i++) {
        for (int k = 0; k < 3; k++)
            scale[3 * i + k] = (float)exp((double)log_scale[3 * i + k]);
        /* L = ln(sigma / sigma_T), sigma_T = 1/255 */
        lnop[i] = (float)log(255.0 * (double)opacity[i]);
    }
}

static int finite3(float a, float b, float c)
{
    return isfinite(a) && isfinite(b) && isfinite(c);
}

static void footprint_one(const float *m, const float *s, const float *q,
                          float L, int level, float smax, float smin,
                          int n_levels, int mode, const or_camera *cam,
                          float limx, float limy, int tiles_x, int tiles_y,
                          or_fp *o)
{
    memset(o, 0, sizeof(*o));
    o->cover = -1.0f;
    o->rect[0] = 0; o->rect[1] = 0; o->rect[2] = -1; o->rect[3] = -1;

    const float *W = cam->R;
    /* view-space centre t = W mu + t_view, summed left to right */
    float tx = ((W[0] * m[0] + W[1] * m[1]) + W[2] * m[2]) + cam->t[0];
    float ty = ((W[3] * m[0] + W[4] * m[1]) + W[5] * m[2]) + cam->t[1];
    float tz = ((W[6] * m[0] + W[7] * m[1]) + W[8] * m[2]) + cam->t[2];
    o->depth = 0;
    memcpy(&o->depth, &tz, 4);

    /* normalised quaternion -> rotation matrix */
    float n2 = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
    if (!(L > 0.0f) || !isfinite(L) || !(tz > cam->near_plane) ||
        !isfinite(tz) || !(n2 > 0.0f) || !isfinite(n2))
        return;
    float rn = 1.0f / sqrtf(n2);
    float w = q[0] * rn, x = q[1] * rn, y = q[2] * rn, z = q[3] * rn;
    float xx = x * x, yy = y * y, zz = z * z;
    float xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    float R[9];
    R[0] = 1.0f - 2.0f * (yy + zz);
    R[1] = 2.0f * (xy - wz);
    R[2] = 2.0f * (xz + wy);
    R[3] = 2.0f * (xy + wz);
    R[4] = 1.0f - 2.0f * (xx + zz);
    R[5] = 2.0f * (yz - wx);
    R[6] = 2.0f * (xz - wy);
    R[7] = 2.0f * (yz + wx);
    R[8] = 1.0f - 2.0f * (xx + yy);

    /* M = R diag(s); Sigma = M M^T (symmetric, 6 entries) */
    float M[9];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++)
            M[3 * r + c] = R[3 * r + c] * s[c];
    float S3[9];
    for (int r = 0; r < 3; r++)
        for (int c = r; c < 3; c++) {
            float v = (M[3 * r + 0] * M[3 * c + 0] + M[3 * r + 1] * M[3 * c + 1])
                      + M[3 * r + 2] * M[3 * c + 2];
            S3[3 * r + c] = v;
            S3[3 * c + r] = v;
        }

    /* Jacobian of the perspective map at t, with the view direction
     * clamped to 1.3x the half field of view (guards splats far outside
     * the frustum; the unclamped ratio places the centre). */
    float xr = tx / tz, yr = ty / tz;
    float xc = fminf(limx, fmaxf(-limx, xr));
    float yc = fminf(limy, fmaxf(-limy, yr));
    float J00 = cam->fx / tz;
    float J02 = (-(cam->fx * xc)) / tz;
    float J11 = cam->fy / tz;
    float J12 = (-(cam->fy * yc)) / tz;

    /* T = J W (2x3) */
    float T[6];
    for (int c = 0; c < 3; c++) {
        T[c] = J00 * W[c] + J02 * W[6 + c];
        T[3 + c] = J11 * W[3 + c] + J12 * W[6 + c];
    }
    /* U = T Sigma (2x3), V = U T^T (2x2) */
    float U[6];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++)
            U[3 * r + c] = (T[3 * r + 0] * S3[c] + T[3 * r + 1] * S3[3 + c])
                           + T[3 * r + 2] * S3[6 + c];
    float V00 = (U[0] * T[0] + U[1] * T[1]) + U[2] * T[2];
    float V01 = (U[0] * T[3] + U[1] * T[4]) + U[2] * T[5];
    float V11 = (U[3] * T[3] + U[4] * T[4]) + U[5] * T[5];

    /* low-pass dilation V' = V + 0.3 I (Eq. 4) */
    float a = V00 + 0.3f, b = V01, c = V11 + 0.3f;
    float detd = a * c - b * b;
    float ux = cam->fx * xr + cam->cx;
    float uy = cam->fy * yr + cam->cy;
    if (!finite3(V00, V01, V11) || !(detd > 0.0f) || !isfinite(detd) ||
        !isfinite(ux) || !isfinite(uy))
        return;
    o->valid = 1;

    /* pixel coverage on the undilated V (Sec. 4.1) */
    float det = V00 * V11 - V01 * V01;
    float mx = fmaxf(V00, V11);
    float S = 0.0f;
    if (det > 0.0f && mx > 0.0f)
        S = sqrtf(((8.0f * L) * det) / mx);
    o->cover = S;

    o->ux = ux;
    o->uy = uy;
    o->conic[0] = c / detd;
    o->conic[1] = (-b) / detd;
    o->conic[2] = a / detd;

    /* level-set bounding box -> tile rectangle */
    float ex = sqrtf((2.0f * L) * a);
    float ey = sqrtf((2.0f * L) * c);
    float x0 = floorf((ux - ex) * 0.0625f), x1 = floorf((ux + ex) * 0.0625f);
    float y0 = floorf((uy - ey) * 0.0625f), y1 = floorf((uy + ey) * 0.0625f);
    x0 = fmaxf(x0, 0.0f);
    y0 = fmaxf(y0, 0.0f);
    x1 = fminf(x1, (float)(tiles_x - 1));
    y1 = fminf(y1, (float)(tiles_y - 1));
    if (x0 <= x1 && y0 <= y1) {
        o->rect[0] = (int32_t)x0; o->rect[1] = (int32_t)y0;
        o->rect[2] = (int32_t)x1; o->rect[3] = (int32_t)y1;
        o->ntiles = (uint32_t)((o->rect[2] - o->rect[0] + 1) *
                               (o->rect[3] - o->rect[1] + 1));
    }

    /* selection, Eq. 6 with S_rel^max = 1.5, S_rel^min = 0.5, S_T = 2 */
    int sel;
    if (mode == OR_ALL_LEVELS) {
        sel = 1;
    } else if (mode == OR_FILTER_SMALL) {
        sel = (S / smin >= 0.5f) || (S >= 2.0f);
    } else {
        int keep_large = (level == 1) || (S / smax <= 1.5f);
        int keep_small = (level == n_levels) || (S / smin >= 0.5f) ||
                         (S >= 2.0f);
        sel = keep_large && keep_small;
    }
    o->selected = (uint8_t)(sel ? 1 : 0);
}

void or_footprints32(int64_t n, const float *mean, const float *scale,
                     const float *quat, const float *lnop,
                     const uint8_t *level, const float *s_max,
                     const float *s_min, int32_t n_levels, int32_t mode,
                     const or_camera *cam, or_fp *out)
{
    float limx = 1.3f * ((0.5f * (float)cam->width) / cam->fx);
    float limy = 1.3f * ((0.5f * (float)cam->height) / cam->fy);
    int tiles_x = (cam->width + 15) / 16, tiles_y = (cam->height + 15) / 16;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        footprint_one(mean + 3 * i, scale + 3 * i, quat + 4 * i, lnop[i],
                      level[i], s_max[i], s_min[i], n_levels, mode, cam,
                      limx, limy, tiles_x, tiles_y, out + i);
}

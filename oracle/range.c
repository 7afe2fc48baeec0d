/*
 * UpdateRange (Eq. 5) and an FP64 coverage for pins.  TEST
 * INFRASTRUCTURE (see oracle.h).
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

/*
 * Eq. 5 / Alg. 2: when the render scale equals the scale at which a
 * Gaussian's level was created (level l is created for the 4^(l-1)
 * downsampled resolution, Sec. 4.1), its coverage range is updated with
 * the new coverage S:
 *     S_max' = max(0.95 S_max, S),   S_min' = min(1.05 S_min, S).
 * Only Gaussians of level `level_r` that are valid and touch the image
 * (non-empty tile rectangle) are updated; S is the FP32 footprint's.
 * Starting from S_max = 0, S_min = +inf the first update yields S itself.
 */
void or_update_range(int64_t n, const float *mean, const float *scale,
                     const float *quat, const float *lnop,
                     const uint8_t *level, int32_t n_levels,
                     int32_t level_r, const or_camera *cam, float *s_max,
                     float *s_min)
{
    or_fp *fp = malloc((size_t)(n > 0 ? n : 1) * sizeof(or_fp));
    or_footprints32(n, mean, scale, quat, lnop, level, s_max, s_min,
                    n_levels, OR_ALL_LEVELS, cam, fp);
    for (int64_t i = 0; i < n; i++) {
        if (level[i] != level_r || !fp[i].valid || fp[i].ntiles == 0)
            continue;
        float S = fp[i].cover;
        s_max[i] = fmaxf(0.95f * s_max[i], S);
        s_min[i] = fminf(1.05f * s_min[i], S);
    }
    free(fp);
}

/*
 * Pixel coverage in FP64 straight from the scene parameters (log-scale,
 * unnormalised quaternion, opacity): the same definition as the FP32
 * footprint (Sec. 4.1) without the fixed single-precision order, used to
 * bound the FP32 result.  cov2d receives the undilated V00, V01, V11.
 * Invalid Gaussians (behind the near plane, sigma <= 1/255) get -1.
 */
void or_coverage64(int64_t n, const float *mean, const float *log_scale,
                   const float *quat, const float *opacity,
                   const or_camera *cam, double *cover, double *ux,
                   double *uy, double *cov2d)
{
    double W[9];
    for (int k = 0; k < 9; k++)
        W[k] = cam->R[k];
    double fx = cam->fx, fy = cam->fy;
    double limx = 1.3 * (0.5 * cam->width / fx);
    double limy = 1.3 * (0.5 * cam->height / fy);
    for (int64_t i = 0; i < n; i++) {
        const float *m = mean + 3 * i, *q = quat + 4 * i;
        double t[3];
        for (int r = 0; r < 3; r++)
            t[r] = W[3 * r] * m[0] + W[3 * r + 1] * m[1] + W[3 * r + 2] * m[2]
                   + cam->t[r];
        double L = log(255.0 * (double)opacity[i]);
        cover[i] = -1.0;
        ux[i] = uy[i] = 0.0;
        cov2d[3 * i] = cov2d[3 * i + 1] = cov2d[3 * i + 2] = 0.0;
        if (!(L > 0.0) || !(t[2] > cam->near_plane))
            continue;
        double qn = sqrt((double)q[0] * q[0] + (double)q[1] * q[1] +
                         (double)q[2] * q[2] + (double)q[3] * q[3]);
        double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
        double R[9] = {
            1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
            2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
            2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
        double s2[3];
        for (int k = 0; k < 3; k++)
            s2[k] = exp(2.0 * (double)log_scale[3 * i + k]);
        double Sg[9];
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) {
                double v = 0.0;
                for (int k = 0; k < 3; k++)
                    v += R[3 * r + k] * s2[k] * R[3 * c + k];
                Sg[3 * r + c] = v;
            }
        double xr = t[0] / t[2], yr = t[1] / t[2];
        double xc = fmin(limx, fmax(-limx, xr)), yc = fmin(limy, fmax(-limy, yr));
        double J[6] = {fx / t[2], 0.0, -fx * xc / t[2],
                       0.0, fy / t[2], -fy * yc / t[2]};
        double T[6];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 3; c++) {
                double v = 0.0;
                for (int k = 0; k < 3; k++)
                    v += J[3 * r + k] * W[3 * k + c];
                T[3 * r + c] = v;
            }
        double V[4];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 2; c++) {
                double v = 0.0;
                for (int k = 0; k < 3; k++)
                    for (int l = 0; l < 3; l++)
                        v += T[3 * r + k] * Sg[3 * k + l] * T[3 * c + l];
                V[2 * r + c] = v;
            }
        double det = V[0] * V[3] - V[1] * V[2];
        double mx = fmax(V[0], V[3]);
        cover[i] = (det > 0.0 && mx > 0.0) ? sqrt(8.0 * L * det / mx) : 0.0;
        ux[i] = fx * xr + cam->cx;
        uy[i] = fy * yr + cam->cy;
        cov2d[3 * i] = V[0];
        cov2d[3 * i + 1] = V[1];
        cov2d[3 * i + 2] = V[3];
    }
}

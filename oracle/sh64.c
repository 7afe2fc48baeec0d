/*
 * View-dependent colour from spherical-harmonic coefficients, FP64.
 * TEST INFRASTRUCTURE (see oracle.h).
 *
 * The Gaussian's colour c_k (Sec. 3.1) is stored as spherical-harmonic
 * coefficients (supplementary, "Average Pooling and Enlargement").  The paper
 * does not give the basis; this oracle uses the real orthonormal basis
 *     Y_l0  = K_l0 P_l^0(cos t)
 *     Y_lm  = sqrt(2) K_lm P_l^m(cos t) cos(m p)      m > 0
 *     Y_l-m = sqrt(2) K_lm P_l^m(cos t) sin(m p)      m > 0
 *     K_lm  = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)
 * with P_l^m the associated Legendre functions without the Condon-Shortley
 * phase, coefficient k = l^2 + l + m, the direction from the camera centre
 * to the Gaussian's mean, and colour = max(0, sum_k f_k Y_k + 0.5) per
 * channel (the 3DGS convention).  The Legendre values come from the
 * standard three-term recurrence, evaluated generically for any degree.
 */
#include <math.h>
#include "oracle.h"

static double factorial(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; i++)
        f *= i;
    return f;
}

/* P_l^m(x), no Condon-Shortley phase, 0 <= m <= l */
static double legendre(int l, int m, double x)
{
    double s = sqrt(fmax(0.0, 1.0 - x * x));
    double pmm = 1.0;
    for (int i = 1; i <= m; i++)
        pmm *= (2.0 * i - 1.0) * s;
    if (l == m)
        return pmm;
    double pm1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1)
        return pm1;
    double p = 0.0;
    for (int ll = m + 2; ll <= l; ll++) {
        p = (x * (2.0 * ll - 1.0) * pm1 - (ll + m - 1.0) * pmm) / (ll - m);
        pmm = pm1;
        pm1 = p;
    }
    return p;
}

void or_sh_basis64(int32_t deg, const double dir[3], double *out)
{
    double r = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    double x = dir[0] / r, y = dir[1] / r, z = dir[2] / r;
    double phi = atan2(y, x);
    for (int l = 0; l <= deg; l++)
        for (int m = -l; m <= l; m++) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) *
                            factorial(l - am) / factorial(l + am));
            double P = legendre(l, am, z);
            double v;
            if (m == 0)
                v = K * P;
            else if (m > 0)
                v = sqrt(2.0) * K * P * cos(am * phi);
            else
                v = sqrt(2.0) * K * P * sin(am * phi);
            out[l * l + l + m] = v;
        }
}

void or_colors64(int64_t n, const float *mean, const float *color,
                 int32_t sh_degree, const or_camera *cam, double *rgb)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        if (sh_degree < 0) {
            for (int c = 0; c < 3; c++)
                rgb[3 * i + c] = (double)color[3 * i + c];
            continue;
        }
        int K = (sh_degree + 1) * (sh_degree + 1);
        double d[3], Y[64];
        for (int c = 0; c < 3; c++)
            d[c] = (double)mean[3 * i + c] - (double)cam->campos[c];
        or_sh_basis64(sh_degree, d, Y);
        for (int c = 0; c < 3; c++) {
            double v = 0.5;
            for (int k = 0; k < K; k++)
                v += (double)color[((int64_t)i * K + k) * 3 + c] * Y[k];
            rgb[3 * i + c] = v > 0.0 ? v : 0.0;
        }
    }
}

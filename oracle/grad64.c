/*
 * FP64 forward with an FP64 projection, and its analytic gradient.
 * TEST INFRASTRUCTURE (see oracle.h).
 *
 * The rendered image as a function of the scene parameters, for
 * differentiation (multi-scale training, Sec. 4.1 "Multi-Scale Training",
 * renders and back-propagates through it).  Tile membership and list order
 * are held fixed (they come from the FP32 footprint lists, as in a training
 * step); every value inside is FP64:
 *   t = W mu + t_view; q^ = q/|q|; R = R(q^); Sigma = R diag(e^s)^2 R^T;
 *   J = perspective Jacobian at t (view ratio clamped to 1.3x the half
 *   field of view); V = J W Sigma W^T J^T; V' = V + 0.3 I; Q = V'^-1;
 *   u = (fx tx/tz + cx, fy ty/tz + cy); colour from SH (sh64.c);
 *   power = -(1/2) d^T Q d with d = pixel - u; alpha = min(0.99, sigma e^power);
 *   front-to-back blend of Eq. 3 with the skip / stop rules of render64.c.
 *
 * The gradient replays every pixel's list backwards from its final
 * transmittance: with R_k the colour behind Gaussian k (including T_N bg),
 *   dC/dalpha_k = T_k c_k - R_k / (1 - alpha_k),   dC/dc_k = alpha_k T_k,
 * then alpha -> (sigma, power) -> (u, Q) -> (V', t) -> (mu, s, q), and the
 * colour -> (SH coefficients, view direction -> mu).  The derivative of the
 * SH basis with respect to the direction is taken by a central difference
 * of sh64.c's basis (step 1e-6; error ~1e-10), everything else is
 * closed-form.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define SIGMA_T (1.0 / 255.0)
#define T_STOP 1e-4
#define ALPHA_MAX 0.99

typedef struct {
    int valid;
    double t[3], qn, qh[4], R[9], se[3], M[9], Sig[9];
    double xr, yr, xc, yc;
    int clx, cly;  /* view ratio clamped (no gradient through it) */
    double J[6], T[6], V[3], Vd[3], Q[3], det;
    double u[2];
    double sigma;
    double dir[3], rdist;
    double pre[3], rgb[3];
} p64;

static void quat_rot(const double q[4], double R[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

static void project64(int64_t i, const float *mean, const float *log_scale,
                      const float *quat, const float *opacity, const float *color,
                      int sh_degree, const or_camera *cam, p64 *o)
{
    memset(o, 0, sizeof(*o));
    double W[9];
    for (int k = 0; k < 9; k++) W[k] = cam->R[k];
    for (int r = 0; r < 3; r++)
        o->t[r] = W[3 * r] * mean[3 * i] + W[3 * r + 1] * mean[3 * i + 1] +
                  W[3 * r + 2] * mean[3 * i + 2] + cam->t[r];
    double n2 = 0;
    for (int k = 0; k < 4; k++) n2 += (double)quat[4 * i + k] * quat[4 * i + k];
    if (!(o->t[2] > cam->near_plane) || !(n2 > 0)) return;
    o->qn = sqrt(n2);
    for (int k = 0; k < 4; k++) o->qh[k] = quat[4 * i + k] / o->qn;
    quat_rot(o->qh, o->R);
    for (int k = 0; k < 3; k++) o->se[k] = exp((double)log_scale[3 * i + k]);
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) o->M[3 * r + c] = o->R[3 * r + c] * o->se[c];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            double v = 0;
            for (int k = 0; k < 3; k++) v += o->M[3 * r + k] * o->M[3 * c + k];
            o->Sig[3 * r + c] = v;
        }
    double fx = cam->fx, fy = cam->fy, tz = o->t[2];
    double limx = 1.3 * (0.5 * cam->width / fx), limy = 1.3 * (0.5 * cam->height / fy);
    o->xr = o->t[0] / tz;
    o->yr = o->t[1] / tz;
    o->clx = fabs(o->xr) > limx;
    o->cly = fabs(o->yr) > limy;
    o->xc = fmin(limx, fmax(-limx, o->xr));
    o->yc = fmin(limy, fmax(-limy, o->yr));
    double J[6] = {fx / tz, 0, -fx * o->xc / tz, 0, fy / tz, -fy * o->yc / tz};
    memcpy(o->J, J, sizeof(J));
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++) {
            double v = 0;
            for (int k = 0; k < 3; k++) v += J[3 * r + k] * W[3 * k + c];
            o->T[3 * r + c] = v;
        }
    double V[4];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 2; c++) {
            double v = 0;
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++)
                    v += o->T[3 * r + k] * o->Sig[3 * k + l] * o->T[3 * c + l];
            V[2 * r + c] = v;
        }
    o->V[0] = V[0]; o->V[1] = V[1]; o->V[2] = V[3];
    o->Vd[0] = V[0] + 0.3; o->Vd[1] = V[1]; o->Vd[2] = V[3] + 0.3;
    o->det = o->Vd[0] * o->Vd[2] - o->Vd[1] * o->Vd[1];
    if (!(o->det > 0)) return;
    o->Q[0] = o->Vd[2] / o->det;
    o->Q[1] = -o->Vd[1] / o->det;
    o->Q[2] = o->Vd[0] / o->det;
    o->u[0] = fx * o->xr + cam->cx;
    o->u[1] = fy * o->yr + cam->cy;
    o->sigma = opacity[i];
    /* colour */
    if (sh_degree < 0) {
        for (int c = 0; c < 3; c++) {
            o->pre[c] = color[3 * i + c];
            o->rgb[c] = o->pre[c];
        }
    } else {
        int K = (sh_degree + 1) * (sh_degree + 1);
        double d[3], Y[64];
        for (int c = 0; c < 3; c++) d[c] = (double)mean[3 * i + c] - cam->campos[c];
        o->rdist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int c = 0; c < 3; c++) o->dir[c] = d[c] / o->rdist;
        or_sh_basis64(sh_degree, o->dir, Y);
        for (int c = 0; c < 3; c++) {
            double v = 0.5;
            for (int k = 0; k < K; k++) v += (double)color[(i * K + k) * 3 + c] * Y[k];
            o->pre[c] = v;
            o->rgb[c] = v > 0 ? v : 0;
        }
    }
    o->valid = 1;
}

/* FP64 blend of one pixel over a fixed list; returns the number of list
 * entries consumed (n_contrib) and the final T; optionally records the
 * per-entry alpha and T_k used by the backward replay. */
static void blend64(const uint32_t *list, int64_t len, const p64 *P, double px,
                    double py, const float *bg, double C[3], double *Tf,
                    uint32_t *ncontrib, uint32_t *nblend)
{
    double T = 1;
    C[0] = C[1] = C[2] = 0;
    *ncontrib = 0;
    *nblend = 0;
    for (int64_t k = 0; k < len; k++) {
        const p64 *g = &P[list[k]];
        if (!g->valid) continue;
        double dx = px - g->u[0], dy = py - g->u[1];
        double power = -0.5 * (g->Q[0] * dx * dx + g->Q[2] * dy * dy) - g->Q[1] * dx * dy;
        if (power > 0) continue;
        double G = g->sigma * exp(power);
        double alpha = G < ALPHA_MAX ? G : ALPHA_MAX;
        if (alpha < SIGMA_T) continue;
        double Tn = T * (1 - alpha);
        if (Tn < T_STOP) break;
        for (int c = 0; c < 3; c++) C[c] += alpha * T * g->rgb[c];
        T = Tn;
        *ncontrib = (uint32_t)(k + 1);
        (*nblend)++;
    }
    for (int c = 0; c < 3; c++) C[c] += T * bg[c];
    *Tf = T;
}

static p64 *project_all(int64_t n, const float *mean, const float *log_scale,
                        const float *quat, const float *opacity, const float *color,
                        int sh_degree, const or_camera *cam)
{
    p64 *P = malloc((size_t)(n > 0 ? n : 1) * sizeof(p64));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        project64(i, mean, log_scale, quat, opacity, color, sh_degree, cam, &P[i]);
    return P;
}

void or_forward64_full(int64_t n, const float *mean, const float *log_scale,
                       const float *quat, const float *opacity, const float *color,
                       int32_t sh_degree, const or_camera *cam, const int64_t *offsets,
                       const uint32_t *idx, double *image, double *final_t,
                       uint32_t *n_contrib, uint32_t *n_blend)
{
    p64 *P = project_all(n, mean, log_scale, quat, opacity, color, sh_degree, cam);
    int W = cam->width, H = cam->height, tiles_x = (W + 15) / 16;
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int64_t t = (int64_t)(y / 16) * tiles_x + x / 16;
            double C[3], Tf;
            uint32_t nc, nb;
            blend64(idx + offsets[t], offsets[t + 1] - offsets[t], P, x + 0.5, y + 0.5,
                    cam->bg, C, &Tf, &nc, &nb);
            int64_t p = (int64_t)y * W + x;
            for (int c = 0; c < 3; c++) image[(int64_t)c * W * H + p] = C[c];
            final_t[p] = Tf;
            n_contrib[p] = nc;
            n_blend[p] = nb;
        }
    free(P);
}

/* symmetric 2x2 stored (a, b, c) = [[a, b], [b, c]] */
static void sym2_mul3(const double A[3], const double B[3], const double C[3], double out[3])
{
    /* out = A B C for symmetric A, B, C (result symmetric when C = A) */
    double AB[4] = {A[0] * B[0] + A[1] * B[1], A[0] * B[1] + A[1] * B[2],
                    A[1] * B[0] + A[2] * B[1], A[1] * B[1] + A[2] * B[2]};
    out[0] = AB[0] * C[0] + AB[1] * C[1];
    out[1] = AB[0] * C[1] + AB[1] * C[2];
    out[2] = AB[2] * C[1] + AB[3] * C[2];
}

/* Per-Gaussian chain: g2 = dL/d(ux, uy, Qa, Qb, Qc, sigma, r, g, b) ->
 * parameter gradients.  Qb is the scalar off-diagonal of the conic. */
static void project64_bwd(int64_t i, const p64 *P, const double g2[9], const float *color,
                          int sh_degree, const or_camera *cam, double *dmean,
                          double *dlog_scale, double *dquat, double *dopacity,
                          double *dcolor)
{
    double W[9];
    for (int k = 0; k < 9; k++) W[k] = cam->R[k];
    double fx = cam->fx, fy = cam->fy;
    double tx = P->t[0], ty = P->t[1], tz = P->t[2];
    double dt[3] = {0, 0, 0};
    /* centre */
    dt[0] += g2[0] * fx / tz;
    dt[2] += -g2[0] * fx * tx / (tz * tz);
    dt[1] += g2[1] * fy / tz;
    dt[2] += -g2[1] * fy * ty / (tz * tz);
    /* conic -> dilated covariance -> covariance: G_V = -Q G_Q Q */
    double GQ[3] = {g2[2], 0.5 * g2[3], g2[4]}, GV[3];
    sym2_mul3(P->Q, GQ, P->Q, GV);
    for (int k = 0; k < 3; k++) GV[k] = -GV[k];
    double GVm[4] = {GV[0], GV[1], GV[1], GV[2]};
    /* V = T Sigma T^T:  G_Sigma = T^T G_V T,  G_T = 2 G_V T Sigma */
    double GSig[9], GT[6];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            double v = 0;
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++)
                    v += P->T[3 * a + r] * GVm[2 * a + b] * P->T[3 * b + c];
            GSig[3 * r + c] = v;
        }
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++) {
            double v = 0;
            for (int a = 0; a < 2; a++)
                for (int k = 0; k < 3; k++)
                    v += GVm[2 * r + a] * P->T[3 * a + k] * P->Sig[3 * k + c];
            GT[3 * r + c] = 2 * v;
        }
    /* T = J W:  G_J = G_T W^T */
    double GJ[6];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++) {
            double v = 0;
            for (int k = 0; k < 3; k++) v += GT[3 * r + k] * W[3 * c + k];
            GJ[3 * r + c] = v;
        }
    /* J = [[fx/tz, 0, -fx xc/tz], [0, fy/tz, -fy yc/tz]] */
    dt[2] += GJ[0] * (-fx / (tz * tz)) + GJ[4] * (-fy / (tz * tz)) +
             GJ[2] * (fx * P->xc / (tz * tz)) + GJ[5] * (fy * P->yc / (tz * tz));
    double dxc = GJ[2] * (-fx / tz), dyc = GJ[5] * (-fy / tz);
    if (!P->clx) {
        dt[0] += dxc / tz;
        dt[2] += -dxc * tx / (tz * tz);
    }
    if (!P->cly) {
        dt[1] += dyc / tz;
        dt[2] += -dyc * ty / (tz * tz);
    }
    /* t = W mu + t_view */
    for (int c = 0; c < 3; c++)
        dmean[3 * i + c] += W[c] * dt[0] + W[3 + c] * dt[1] + W[6 + c] * dt[2];
    /* Sigma = M M^T: G_M = 2 G_Sigma M;  M = R diag(se) */
    double GM[9];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            double v = 0;
            for (int k = 0; k < 3; k++) v += GSig[3 * r + k] * P->M[3 * k + c];
            GM[3 * r + c] = 2 * v;
        }
    double GR[9];
    for (int c = 0; c < 3; c++) {
        double gs = 0;
        for (int r = 0; r < 3; r++) {
            gs += P->R[3 * r + c] * GM[3 * r + c];
            GR[3 * r + c] = GM[3 * r + c] * P->se[c];
        }
        dlog_scale[3 * i + c] += gs * P->se[c];
    }
    /* R(q^) */
    double w = P->qh[0], x = P->qh[1], y = P->qh[2], z = P->qh[3];
    double dq[4];
    dq[0] = GR[1] * (-2 * z) + GR[2] * (2 * y) + GR[3] * (2 * z) + GR[5] * (-2 * x) +
            GR[6] * (-2 * y) + GR[7] * (2 * x);
    dq[1] = GR[1] * (2 * y) + GR[2] * (2 * z) + GR[3] * (2 * y) + GR[4] * (-4 * x) +
            GR[5] * (-2 * w) + GR[6] * (2 * z) + GR[7] * (2 * w) + GR[8] * (-4 * x);
    dq[2] = GR[0] * (-4 * y) + GR[1] * (2 * x) + GR[2] * (2 * w) + GR[3] * (2 * x) +
            GR[5] * (2 * z) + GR[6] * (-2 * w) + GR[7] * (2 * z) + GR[8] * (-4 * y);
    dq[3] = GR[0] * (-4 * z) + GR[1] * (-2 * w) + GR[2] * (2 * x) + GR[3] * (2 * w) +
            GR[4] * (-4 * z) + GR[5] * (2 * y) + GR[6] * (2 * x) + GR[7] * (2 * y);
    double dot = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
    for (int k = 0; k < 4; k++) dquat[4 * i + k] += (dq[k] - P->qh[k] * dot) / P->qn;
    /* opacity */
    dopacity[i] += g2[5];
    /* colour */
    double drgb[3];
    if (sh_degree < 0) {  /* plain RGB: no clamp */
        for (int c = 0; c < 3; c++) dcolor[3 * i + c] += g2[6 + c];
        return;
    }
    for (int c = 0; c < 3; c++) drgb[c] = P->pre[c] > 0 ? g2[6 + c] : 0.0;
    int K = (sh_degree + 1) * (sh_degree + 1);
    double Y[64];
    or_sh_basis64(sh_degree, P->dir, Y);
    for (int k = 0; k < K; k++)
        for (int c = 0; c < 3; c++) dcolor[(i * K + k) * 3 + c] += drgb[c] * Y[k];
    /* view direction: dL/ddir by a central difference of the basis */
    double ddir[3] = {0, 0, 0};
    for (int e = 0; e < 3; e++) {
        double dp[3], dm[3], Yp[64], Ym[64], h = 1e-6;
        for (int c = 0; c < 3; c++) dp[c] = dm[c] = P->dir[c];
        dp[e] += h;
        dm[e] -= h;
        or_sh_basis64(sh_degree, dp, Yp);
        or_sh_basis64(sh_degree, dm, Ym);
        for (int c = 0; c < 3; c++)
            for (int k = 0; k < K; k++)
                ddir[e] += drgb[c] * (double)color[(i * K + k) * 3 + c] * (Yp[k] - Ym[k]) / (2 * h);
    }
    /* sh64.c normalises its argument, so d/ddir of Y(dir) is already the
     * tangential derivative; dir = (mu - c)/|mu - c| */
    double dd = ddir[0] * P->dir[0] + ddir[1] * P->dir[1] + ddir[2] * P->dir[2];
    for (int c = 0; c < 3; c++) dmean[3 * i + c] += (ddir[c] - P->dir[c] * dd) / P->rdist;
}

int64_t or_grad64(int64_t n, const float *mean, const float *log_scale, const float *quat,
                  const float *opacity, const float *color, int32_t sh_degree,
                  const or_camera *cam, const int64_t *offsets, const uint32_t *idx,
                  const double *dl_dimage, double *dmean, double *dlog_scale,
                  double *dquat, double *dopacity, double *dcolor)
{
    p64 *P = project_all(n, mean, log_scale, quat, opacity, color, sh_degree, cam);
    int W = cam->width, H = cam->height, tiles_x = (W + 15) / 16;
    double *g2 = calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double));
    int64_t used = 0;
    /* per pixel: forward to find the contributors, then the reverse replay;
     * pixels are processed serially so the per-Gaussian sums are exact */
    double *al = malloc(sizeof(double) * 65536), *Tk = malloc(sizeof(double) * 65536);
    uint32_t *who = malloc(sizeof(uint32_t) * 65536);
    double *dxs = malloc(sizeof(double) * 65536), *dys = malloc(sizeof(double) * 65536),
           *Gs = malloc(sizeof(double) * 65536);
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int64_t t = (int64_t)(y / 16) * tiles_x + x / 16;
            const uint32_t *list = idx + offsets[t];
            int64_t len = offsets[t + 1] - offsets[t];
            double px = x + 0.5, py = y + 0.5, T = 1;
            int m = 0;
            for (int64_t k = 0; k < len && m < 65536; k++) {
                const p64 *g = &P[list[k]];
                if (!g->valid) continue;
                double dx = px - g->u[0], dy = py - g->u[1];
                double power = -0.5 * (g->Q[0] * dx * dx + g->Q[2] * dy * dy) - g->Q[1] * dx * dy;
                if (power > 0) continue;
                double G = g->sigma * exp(power);
                double alpha = G < ALPHA_MAX ? G : ALPHA_MAX;
                if (alpha < SIGMA_T) continue;
                double Tn = T * (1 - alpha);
                if (Tn < T_STOP) break;
                who[m] = list[k];
                al[m] = alpha;
                Tk[m] = T;
                dxs[m] = dx;
                dys[m] = dy;
                Gs[m] = G;
                m++;
                T = Tn;
            }
            int64_t p = (int64_t)y * W + x;
            double dC[3], Rr[3];
            for (int c = 0; c < 3; c++) {
                dC[c] = dl_dimage[(int64_t)c * W * H + p];
                Rr[c] = T * cam->bg[c];
            }
            for (int j = m - 1; j >= 0; j--) {
                const p64 *g = &P[who[j]];
                double a = al[j], Tj = Tk[j];
                double dalpha = 0;
                for (int c = 0; c < 3; c++) {
                    dalpha += dC[c] * (Tj * g->rgb[c] - Rr[c] / (1 - a));
                    g2[9 * who[j] + 6 + c] += a * Tj * dC[c];
                    Rr[c] += a * Tj * g->rgb[c];
                }
                if (Gs[j] < ALPHA_MAX) {
                    double dpow = dalpha * a;
                    double dx = dxs[j], dy = dys[j];
                    g2[9 * who[j] + 5] += dalpha * (Gs[j] / g->sigma);
                    /* power = -(Qa dx^2 + Qc dy^2)/2 - Qb dx dy, d = pixel - u */
                    g2[9 * who[j] + 0] += dpow * (g->Q[0] * dx + g->Q[1] * dy);
                    g2[9 * who[j] + 1] += dpow * (g->Q[2] * dy + g->Q[1] * dx);
                    g2[9 * who[j] + 2] += dpow * (-0.5 * dx * dx);
                    g2[9 * who[j] + 3] += dpow * (-dx * dy);
                    g2[9 * who[j] + 4] += dpow * (-0.5 * dy * dy);
                }
                used++;
            }
        }
    free(al); free(Tk); free(who); free(dxs); free(dys); free(Gs);
    int K = sh_degree < 0 ? 1 : (sh_degree + 1) * (sh_degree + 1);
    memset(dmean, 0, sizeof(double) * 3 * n);
    memset(dlog_scale, 0, sizeof(double) * 3 * n);
    memset(dquat, 0, sizeof(double) * 4 * n);
    memset(dopacity, 0, sizeof(double) * n);
    memset(dcolor, 0, sizeof(double) * 3 * K * n);
    for (int64_t i = 0; i < n; i++) {
        if (!P[i].valid) continue;
        int any = 0;
        for (int k = 0; k < 9; k++) any |= g2[9 * i + k] != 0.0;
        if (!any) continue;
        project64_bwd(i, &P[i], g2 + 9 * i, color, sh_degree, cam, dmean, dlog_scale, dquat,
                      dopacity, dcolor);
    }
    free(g2);
    free(P);
    return used;
}

/*
 * Tile lists and FP64 front-to-back blending.  TEST INFRASTRUCTURE (see
 * oracle.h).
 *
 * Sec. 3.1: the image is divided into 16x16 tiles, every 2D Gaussian
 * touching a tile is listed for it, each list is sorted by the Gaussians'
 * original (view-space) depth, and every pixel blends its tile's list
 * front to back.  Eq. 3 writes the blend as sum_k sigma_k c_k T_k G_k(x)
 * with the transmittance T_k = prod_{j<k} (1 - alpha_j) computed
 * incrementally (the sequential sum of Sec. 3.2, item 2).
 *
 * Readings of points the paper leaves open (prior 3DGS practice):
 *   - the pixel is sampled at its centre (x + 0.5, y + 0.5);
 *   - alpha = min(0.99, sigma exp(power)); a Gaussian with alpha < 1/255
 *     (the paper's sigma_T) or power > 0 is skipped;
 *   - blending stops before a Gaussian that would bring T below 1e-4;
 *   - equal depths are ordered by Gaussian index;
 *   - the background is added as T_final * bg.
 * The splat parameters (centre, conic, membership, order) are the FP32
 * footprint (footprint32.c); opacity, colour and every blending step are
 * evaluated in FP64.
 *
 * Flags: a decision is flagged when it lies within what a single-precision
 * evaluation of the same quantities could move it by, so that a
 * single-precision renderer may take the other branch there:
 *   - bit 0: the alpha test, ln(sigma e^power / sigma_T) = power + ln(255
 *     sigma) within max(alpha_flag_rel, EPS_P) of 0, where EPS_P =
 *     K_P u (|a| dx^2 / 2 + |b dx dy| + |c| dy^2 / 2 + |ln(255 sigma)|)
 *     bounds the error of a single-precision evaluation of the quadratic
 *     form and of the threshold (u = 2^-24, K_P a generous count of the
 *     roundings in the conic scaling, the differences, the products and
 *     the sums);
 *   - bit 1: the early stop, T (1 - alpha) within a relative
 *     max(t_flag_rel, EPS_T) of 1e-4, where EPS_T accumulates, over the
 *     Gaussians blended so far, the relative error that single-precision
 *     alpha and products carry into T: alpha / (1 - alpha) times alpha's
 *     relative error, plus K_T u per product, plus K_S u for a product
 *     formed as a scan rather than in sequence.
 * or_pixel_alternatives() renders one pixel along every combination of
 * branches at its flagged decisions (every result a single-precision
 * renderer may correctly produce there).
  */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define SIGMA_T (1.0 / 255.0)
#define T_STOP 1e-4
#define ALPHA_MAX 0.99
#define U32 (1.0 / 16777216.0) /* unit roundoff of single precision */
#define K_P 16.0  /* roundings in a single-precision power and threshold */
#define K_A 8.0   /* exp2 approximation and the opacity product */
#define K_T 3.0   /* per transmittance product */
#define K_S 16.0  /* a transmittance formed by a scan of products */

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

static int listed(const or_fp *f)
{
    return f->selected && f->ntiles > 0;
}

int64_t or_tile_lists(int64_t n, const or_fp *fp, int32_t tiles_x,
                      int32_t tiles_y, int64_t *offsets, uint32_t *idx,
                      int64_t capacity)
{
    int64_t ntiles = (int64_t)tiles_x * tiles_y;
    int64_t *count = calloc((size_t)ntiles, sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        if (!listed(&fp[i]))
            continue;
        for (int y = fp[i].rect[1]; y <= fp[i].rect[3]; y++)
            for (int x = fp[i].rect[0]; x <= fp[i].rect[2]; x++)
                count[(int64_t)y * tiles_x + x]++;
    }
    offsets[0] = 0;
    for (int64_t t = 0; t < ntiles; t++)
        offsets[t + 1] = offsets[t] + count[t];
    int64_t total = offsets[ntiles];
    if (total > capacity) {
        free(count);
        return total;
    }
    /* fill in index order, then sort each tile by (depth bits, index) */
    uint64_t *keys = malloc((size_t)(total > 0 ? total : 1) * sizeof(uint64_t));
    memset(count, 0, (size_t)ntiles * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        if (!listed(&fp[i]))
            continue;
        for (int y = fp[i].rect[1]; y <= fp[i].rect[3]; y++)
            for (int x = fp[i].rect[0]; x <= fp[i].rect[2]; x++) {
                int64_t t = (int64_t)y * tiles_x + x;
                keys[offsets[t] + count[t]++] =
                    ((uint64_t)fp[i].depth << 32) | (uint64_t)(uint32_t)i;
            }
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < ntiles; t++)
        qsort(keys + offsets[t], (size_t)(offsets[t + 1] - offsets[t]),
              sizeof(uint64_t), cmp_u64);
    for (int64_t j = 0; j < total; j++)
        idx[j] = (uint32_t)(keys[j] & 0xffffffffu);
    free(keys);
    free(count);
    return total;
}

/* One list entry evaluated at pixel centre (px, py): the unclamped
 * G = sigma exp(power), the alpha-test margin ln(G / sigma_T) and the bound
 * of its single-precision error.  Returns 0 when power > 0 (never
 * blended). */
typedef struct {
    double G, lnr, eps_p;
} entry_eval;

static int eval_entry(const or_fp *f, double sigma, double px, double py, entry_eval *e)
{
    double dx = px - (double)f->ux, dy = py - (double)f->uy;
    double a = f->conic[0], b = f->conic[1], c = f->conic[2];
    double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
    if (power > 0.0)
        return 0;
    double L = log(255.0 * sigma);
    double terms = 0.5 * fabs(a) * dx * dx + fabs(b * dx * dy) + 0.5 * fabs(c) * dy * dy;
    e->G = sigma * exp(power);
    e->lnr = power + L;
    e->eps_p = K_P * U32 * (terms + fabs(L));
    return 1;
}

/* Relative error bound that a blended alpha carries into T (1 - alpha). */
static double t_error_step(const entry_eval *e, double alpha)
{
    double eps_alpha = e->G < ALPHA_MAX ? e->eps_p + K_A * U32 : U32;
    return alpha / (1.0 - alpha) * eps_alpha + K_T * U32;
}

typedef struct {
    double C[3];
    double T;
    double epsT; /* relative error bound of a single-precision T */
    uint32_t n_contrib;
    uint8_t flags;
    int64_t evals;
} pixel_state;

static void state_init(pixel_state *st)
{
    st->C[0] = st->C[1] = st->C[2] = 0.0;
    st->T = 1.0;
    st->epsT = 0.0;
    st->n_contrib = 0;
    st->flags = 0;
    st->evals = 0;
}

/* Decisions of one entry: whether alpha passes the 1/255 test, and (for a
 * passing alpha) whether T (1 - alpha) ends the pixel; each with whether a
 * single-precision evaluation may decide it the other way. */
typedef struct {
    int pass, pass_flag;
    double alpha, Tn, epsn;
    int stop, stop_flag;
} entry_decision;

static void decide_alpha(const entry_eval *e, double alpha_flag_rel, entry_decision *d)
{
    double m = e->eps_p > alpha_flag_rel ? e->eps_p : alpha_flag_rel;
    d->alpha = e->G < ALPHA_MAX ? e->G : ALPHA_MAX;
    d->pass = d->alpha >= SIGMA_T;
    d->pass_flag = fabs(e->lnr) <= m;
}

static void decide_stop(const entry_eval *e, const pixel_state *st, double t_flag_rel,
                        entry_decision *d)
{
    d->Tn = st->T * (1.0 - d->alpha);
    d->epsn = st->epsT + t_error_step(e, d->alpha) + K_S * U32;
    double m = d->epsn > t_flag_rel ? d->epsn : t_flag_rel;
    d->stop = d->Tn < T_STOP;
    d->stop_flag = fabs(d->Tn - T_STOP) <= m * T_STOP;
}

static void accumulate(pixel_state *st, const entry_decision *d, const entry_eval *e,
                       const double *rgb_g, int64_t k)
{
    for (int ch = 0; ch < 3; ch++)
        st->C[ch] += d->alpha * st->T * rgb_g[ch];
    st->epsT += t_error_step(e, d->alpha);
    st->T = d->Tn;
    st->n_contrib = (uint32_t)(k + 1);
}

static void blend_pixel(const uint32_t *list, int64_t len, const or_fp *fp,
                        const float *opacity, const double *rgb, double px,
                        double py, double alpha_flag_rel, double t_flag_rel,
                        pixel_state *st)
{
    state_init(st);
    for (int64_t k = 0; k < len; k++) {
        uint32_t g = list[k];
        st->evals = k + 1;
        entry_eval e;
        if (!eval_entry(&fp[g], (double)opacity[g], px, py, &e))
            continue;
        entry_decision d;
        decide_alpha(&e, alpha_flag_rel, &d);
        if (d.pass_flag)
            st->flags |= 1;
        if (!d.pass)
            continue;
        decide_stop(&e, st, t_flag_rel, &d);
        if (d.stop_flag)
            st->flags |= 2;
        if (d.stop)
            break;
        accumulate(st, &d, &e, rgb + 3 * (int64_t)g, k);
    }
}

/* Every result of one pixel that follows the exact decisions wherever they
 * are unflagged and either branch wherever they are flagged (depth-first
 * over the flagged decisions).  A forced decision at entry k0 replaces the
 * exact one there: force_pass / force_stop are -1 (free), 0 or 1. */
typedef struct {
    const uint32_t *list;
    int64_t len;
    const or_fp *fp;
    const float *opacity;
    const double *rgb;
    double px, py, alpha_flag_rel, t_flag_rel;
    int32_t max_alts, n_alts;
    int overflow;
    double *out; /* [max_alts][6]: C0, C1, C2, T, n_contrib, n_eval */
} alt_ctx;

static void walk_alts(alt_ctx *c, int64_t k, pixel_state st, int force_pass, int force_stop)
{
    for (; k < c->len; k++, force_pass = force_stop = -1) {
        if (c->overflow)
            return;
        uint32_t g = c->list[k];
        st.evals = k + 1;
        entry_eval e;
        if (!eval_entry(&c->fp[g], (double)c->opacity[g], c->px, c->py, &e))
            continue;
        entry_decision d;
        decide_alpha(&e, c->alpha_flag_rel, &d);
        if (force_pass >= 0) {
            d.pass = force_pass;
        } else if (d.pass_flag) {
            walk_alts(c, k, st, !d.pass, -1);
        }
        if (!d.pass)
            continue;
        decide_stop(&e, &st, c->t_flag_rel, &d);
        if (force_stop >= 0) {
            d.stop = force_stop;
        } else if (d.stop_flag) {
            walk_alts(c, k, st, 1, !d.stop);
        }
        if (d.stop)
            break;
        accumulate(&st, &d, &e, c->rgb + 3 * (int64_t)g, k);
    }
    if (c->overflow)
        return;
    if (c->n_alts >= c->max_alts) {
        c->overflow = 1;
        return;
    }
    double *o = c->out + 6 * (int64_t)c->n_alts++;
    o[0] = st.C[0];
    o[1] = st.C[1];
    o[2] = st.C[2];
    o[3] = st.T;
    o[4] = (double)st.n_contrib;
    o[5] = (double)st.evals;
}

int32_t or_pixel_alternatives(const or_fp *fp, const float *opacity, const double *rgb,
                              const uint32_t *list, int64_t len, double px, double py,
                              double alpha_flag_rel, double t_flag_rel, int32_t max_alts,
                              double *out)
{
    alt_ctx c = {list, len, fp, opacity, rgb, px, py, alpha_flag_rel, t_flag_rel,
                 max_alts, 0, 0, out};
    pixel_state st;
    state_init(&st);
    walk_alts(&c, 0, st, -1, -1);
    return c.overflow ? -1 : c.n_alts;
}

/* Per-tile FP64 blend over the lists of step 1.  n_eval (may be NULL)
 * receives, per pixel, the list entries evaluated up to and including the
 * one that ended the pixel (the whole list if none did); the return value is
 * their sum over the rendered pixels. */
int64_t or_render64(int64_t n, const or_fp *fp, const float *opacity,
                    const double *rgb, const or_camera *cam,
                    const int64_t *offsets, const uint32_t *idx,
                    const int32_t *tile_sel, int32_t n_tile_sel,
                    double alpha_flag_rel, double t_flag_rel,
                    double *image, double *final_t, uint32_t *n_contrib,
                    uint8_t *flags, int64_t *n_eval)
{
    (void)n;
    int W = cam->width, H = cam->height;
    int tiles_x = (W + 15) / 16, tiles_y = (H + 15) / 16;
    int64_t ntiles = (int64_t)tiles_x * tiles_y;
    int64_t todo = tile_sel ? n_tile_sel : ntiles;
    int64_t evals = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : evals)
    for (int64_t s = 0; s < todo; s++) {
        int64_t t = tile_sel ? tile_sel[s] : s;
        int tx = (int)(t % tiles_x), ty = (int)(t / tiles_x);
        const uint32_t *list = idx + offsets[t];
        int64_t len = offsets[t + 1] - offsets[t];
        for (int y = 16 * ty; y < 16 * ty + 16 && y < H; y++)
            for (int x = 16 * tx; x < 16 * tx + 16 && x < W; x++) {
                pixel_state st;
                blend_pixel(list, len, fp, opacity, rgb, x + 0.5, y + 0.5,
                            alpha_flag_rel, t_flag_rel, &st);
                int64_t p = (int64_t)y * W + x;
                for (int ch = 0; ch < 3; ch++)
                    image[(int64_t)ch * W * H + p] =
                        st.C[ch] + st.T * (double)cam->bg[ch];
                final_t[p] = st.T;
                n_contrib[p] = st.n_contrib;
                flags[p] = st.flags;
                if (n_eval)
                    n_eval[p] = st.evals;
                evals += st.evals;
            }
    }
    return evals;
}

int64_t or_render64_brute(int64_t n, const or_fp *fp, const float *opacity,
                          const double *rgb, const or_camera *cam,
                          double alpha_flag_rel, double *image,
                          double *final_t, uint8_t *flags)
{
    /* every selected Gaussian, one global (depth, index) order, no tiles */
    int64_t m = 0;
    uint64_t *keys = malloc((size_t)(n > 0 ? n : 1) * sizeof(uint64_t));
    for (int64_t i = 0; i < n; i++)
        if (fp[i].selected)
            keys[m++] = ((uint64_t)fp[i].depth << 32) | (uint64_t)(uint32_t)i;
    qsort(keys, (size_t)m, sizeof(uint64_t), cmp_u64);
    uint32_t *list = malloc((size_t)(m > 0 ? m : 1) * sizeof(uint32_t));
    for (int64_t j = 0; j < m; j++)
        list[j] = (uint32_t)(keys[j] & 0xffffffffu);
    int W = cam->width, H = cam->height;
    int64_t evals = 0;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            pixel_state st;
            blend_pixel(list, m, fp, opacity, rgb, x + 0.5, y + 0.5,
                        alpha_flag_rel, 0.0, &st);
            int64_t p = (int64_t)y * W + x;
            for (int ch = 0; ch < 3; ch++)
                image[(int64_t)ch * W * H + p] =
                    st.C[ch] + st.T * (double)cam->bg[ch];
            final_t[p] = st.T;
            flags[p] = st.flags;
            evals += st.evals;
        }
    free(list);
    free(keys);
    return evals;
}

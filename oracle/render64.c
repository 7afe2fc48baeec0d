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
 * Flags: bit 0 marks a pixel where some evaluated Gaussian had
 * sigma exp(power) within a relative `alpha_flag_rel` of 1/255 (a
 * single-precision evaluation may take the other branch there); bit 1
 * marks T (1 - alpha) within a relative `t_flag_rel` of 1e-4.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define SIGMA_T (1.0 / 255.0)
#define T_STOP 1e-4
#define ALPHA_MAX 0.99

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

/* One Gaussian's contribution test at pixel centre (px, py).  Returns the
 * unclamped sigma * exp(power), or -1 if power > 0. */
static double gauss_at(const or_fp *f, double sigma, double px, double py)
{
    double dx = px - (double)f->ux, dy = py - (double)f->uy;
    double a = f->conic[0], b = f->conic[1], c = f->conic[2];
    double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
    if (power > 0.0)
        return -1.0;
    return sigma * exp(power);
}

typedef struct {
    double C[3];
    double T;
    uint32_t n_contrib;
    uint8_t flags;
    int64_t evals;
} pixel_state;

static void blend_pixel(const uint32_t *list, int64_t len, const or_fp *fp,
                        const float *opacity, const double *rgb, double px,
                        double py, double alpha_flag_rel, double t_flag_rel,
                        pixel_state *st)
{
    st->C[0] = st->C[1] = st->C[2] = 0.0;
    st->T = 1.0;
    st->n_contrib = 0;
    st->flags = 0;
    st->evals = 0;
    for (int64_t k = 0; k < len; k++) {
        uint32_t g = list[k];
        st->evals++;
        double G = gauss_at(&fp[g], (double)opacity[g], px, py);
        if (G < 0.0)
            continue;
        if (fabs(G - SIGMA_T) <= alpha_flag_rel * SIGMA_T)
            st->flags |= 1;
        double alpha = G < ALPHA_MAX ? G : ALPHA_MAX;
        if (alpha < SIGMA_T)
            continue;
        double Tn = st->T * (1.0 - alpha);
        if (fabs(Tn - T_STOP) <= t_flag_rel * T_STOP)
            st->flags |= 2;
        if (Tn < T_STOP)
            break;
        for (int ch = 0; ch < 3; ch++)
            st->C[ch] += alpha * st->T * rgb[3 * (int64_t)g + ch];
        st->T = Tn;
        st->n_contrib = (uint32_t)(k + 1);
    }
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

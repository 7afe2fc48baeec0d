/*
 * AggregateGaussians for one coarse level l_m (Alg. 1; Sec. 4.1 "Aggregate
 * to Insert Large Gaussians"; supplementary "Details of Gaussian Aggregation
 * Algorithm").  TEST INFRASTRUCTURE (see oracle.h).
 *
 * The paper's steps, in its order:
 *   1. Pixel coverage S of every Gaussian of levels 1 .. l_m - 1 in every
 *      training camera at 4^(l_m-1) downsampling (the cameras are passed
 *      already downsampled); a Gaussian splatted to a camera (valid and
 *      touching its image) contributes that camera's S.  A Gaussian whose
 *      smallest S is below S_T = 2 px is small.
 *   2. Positions are normalised (supplementary "Unbounded Scene
 *      Normalization"), per component: x / B inside [-B, B], else
 *      sign(x) (2 - B / |x|), and binned on a grid of floor(400 / l_m)
 *      voxels per axis over [-2, 2] ("Voxelization").
 *   3. The small Gaussians of each voxel are averaged (position, rotation,
 *      SH, opacity and scaling; "Average Pooling and Enlargement") and the
 *      scaling is enlarged by S_T / S_avg, S_avg being the mean of their
 *      smallest coverages.  The new Gaussian belongs to level l_m.
 * Steps 1 and 2 take their integer decisions (small or not, voxel index)
 * in FP32 with a fixed operation order; the averages are FP64.  Scaling is
 * averaged as stored (log-scale), so the enlargement adds ln(S_T / S_avg).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "oracle.h"

#define S_T 2.0f

static float norm32(float x, float B) {
    const float ax = fabsf(x);
    if (ax <= B) return x / B;
    const float t = 2.0f - B / ax;
    return x < 0.0f ? -t : t;
}

static int32_t vox32(float xn, int32_t R) {
    const float t = (xn + 2.0f) * ((float)R * 0.25f);
    int32_t v = (int32_t)floorf(t);
    if (v < 0) v = 0;
    if (v > R - 1) v = R - 1;
    return v;
}

uint32_t or_voxel_key(const float *mean3, float B, int32_t level_m) {
    const int32_t R = 400 / level_m;
    const int32_t vx = vox32(norm32(mean3[0], B), R);
    const int32_t vy = vox32(norm32(mean3[1], B), R);
    const int32_t vz = vox32(norm32(mean3[2], B), R);
    return ((uint32_t)vz * (uint32_t)R + (uint32_t)vy) * (uint32_t)R + (uint32_t)vx;
}

typedef struct {
    uint32_t key;
    int64_t idx;
} kv;

static int kv_cmp(const void *a, const void *b) {
    const kv *x = (const kv *)a, *y = (const kv *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

int64_t or_aggregate(int64_t n, const float *mean, const float *log_scale, const float *quat,
                     const float *opacity, const float *color, int32_t sh_degree,
                     const uint8_t *level, const float *scale, const float *lnop,
                     int32_t n_cams, const or_camera *cams, int32_t level_m, float B,
                     float *smin_out, float *o_mean, float *o_log_scale, float *o_quat,
                     float *o_opacity, float *o_color, uint32_t *o_key, int64_t capacity) {
    const int32_t K = sh_degree < 0 ? 1 : (sh_degree + 1) * (sh_degree + 1);
    float *smin = smin_out;
    for (int64_t i = 0; i < n; i++) smin[i] = INFINITY;
    or_fp *fp = (or_fp *)malloc((size_t)(n > 0 ? n : 1) * sizeof(or_fp));
    float *zeros = (float *)calloc((size_t)(n > 0 ? n : 1), sizeof(float));
    for (int32_t c = 0; c < n_cams; c++) {
        or_footprints32(n, mean, scale, quat, lnop, level, zeros, zeros, 1, OR_ALL_LEVELS,
                        &cams[c], fp);
        for (int64_t i = 0; i < n; i++)
            if (level[i] < level_m && fp[i].valid && fp[i].ntiles > 0 && fp[i].cover < smin[i])
                smin[i] = fp[i].cover;
    }
    free(zeros);
    free(fp);
    kv *sel = (kv *)malloc((size_t)(n > 0 ? n : 1) * sizeof(kv));
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        if (level[i] < level_m && smin[i] < S_T) {
            sel[m].key = or_voxel_key(mean + 3 * i, B, level_m);
            sel[m].idx = i;
            m++;
        }
    qsort(sel, (size_t)m, sizeof(kv), kv_cmp);
    int64_t groups = 0;
    for (int64_t a = 0; a < m;) {
        int64_t b = a;
        while (b < m && sel[b].key == sel[a].key) b++;
        if (groups < capacity) {
            double sm[3] = {0, 0, 0}, sl[3] = {0, 0, 0}, sq[4] = {0, 0, 0, 0}, so = 0, ss = 0;
            double *sc = (double *)calloc((size_t)3 * K, sizeof(double));
            for (int64_t j = a; j < b; j++) {
                const int64_t i = sel[j].idx;
                for (int k = 0; k < 3; k++) {
                    sm[k] += mean[3 * i + k];
                    sl[k] += log_scale[3 * i + k];
                }
                for (int k = 0; k < 4; k++) sq[k] += quat[4 * i + k];
                so += opacity[i];
                ss += smin[i];
                for (int k = 0; k < 3 * K; k++) sc[k] += color[(size_t)3 * K * i + k];
            }
            const double cnt = (double)(b - a);
            const double grow = log((double)S_T / (ss / cnt));
            for (int k = 0; k < 3; k++) {
                o_mean[3 * groups + k] = (float)(sm[k] / cnt);
                o_log_scale[3 * groups + k] = (float)(sl[k] / cnt + grow);
            }
            for (int k = 0; k < 4; k++) o_quat[4 * groups + k] = (float)(sq[k] / cnt);
            o_opacity[groups] = (float)(so / cnt);
            for (int k = 0; k < 3 * K; k++)
                o_color[(size_t)3 * K * groups + k] = (float)(sc[k] / cnt);
            o_key[groups] = sel[a].key;
            free(sc);
        }
        groups++;
        a = b;
    }
    free(sel);
    return groups;
}

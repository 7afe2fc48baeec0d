/*
 * Oracle for multi-scale selective Gaussian splatting (arXiv 2311.17089).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg may load this library.  It shares no code, header,
 * table or constant with the CUDA library; the two meet only through the
 * seeded inputs.
 *
 * Plain, slow, obviously-correct C:
 *   footprint32.c  per-Gaussian footprint in a fixed FP32 operation order
 *                  (the bit-exact contract for masks, coverage and tile
 *                  lists; Sec. 3.1, Sec. 4.1 "Pixel Coverage", Eq. 6)
 *   render64.c     per-tile lists sorted by depth, FP64 front-to-back
 *                  blend (Sec. 3.1, Eq. 3), brute-force variant without tiles
 *   sh64.c         real spherical harmonics from the Legendre recurrence
 *   range.c        UpdateRange (Eq. 5), FP64 coverage for pins
 *   grad64.c       FP64 forward with an FP64 projection, and its analytic
 *                  gradient (reverse replay, chain rule to the parameters)
 *   aggregate.c    AggregateGaussians (Alg. 1) for one coarse level
 *
 * Parity unpinned: nothing here reproduces the paper's PSNR/LPIPS tables
 * (they need the datasets and trained models).
 */
#ifndef MS_ORACLE_H
#define MS_ORACLE_H
#include <stdint.h>

typedef struct {
    float R[9];      /* world -> camera rotation, row-major */
    float t[3];      /* world -> camera translation         */
    float campos[3]; /* camera centre in world coordinates  */
    float fx, fy, cx, cy;
    int32_t width, height;
    float near_plane;
    float bg[3];
} or_camera;

/* Selection modes: Eq. 6 with the level exemptions of Sec. 4.1; every
 * valid Gaussian; the "Filter Small" ablation (Sec. 5), the second clause
 * of Eq. 6 alone. */
enum { OR_SELECTIVE = 0, OR_ALL_LEVELS = 1, OR_FILTER_SMALL = 2 };

/* Per-Gaussian FP32 footprint. */
typedef struct {
    uint8_t valid;     /* in front of the near plane, level set exists, finite */
    uint8_t selected;  /* valid and passes the mode's predicate               */
    float cover;       /* pixel coverage S (undilated), -1 if !valid          */
    uint32_t depth;    /* bit pattern of view-space z                         */
    int32_t rect[4];   /* tiles x0, y0, x1, y1 (inclusive); empty if x0 > x1  */
    uint32_t ntiles;   /* tiles in rect (0 if empty or !valid)                */
    float ux, uy;      /* projected centre in pixels                          */
    float conic[3];    /* inverse of the dilated 2D covariance (a, b, c)      */
} or_fp;

#ifdef __cplusplus
extern "C" {
#endif

void or_prepare(int64_t n, const float *log_scale, const float *opacity,
                float *scale, float *lnop);

void or_footprints32(int64_t n, const float *mean, const float *scale,
                     const float *quat, const float *lnop,
                     const uint8_t *level, const float *s_max,
                     const float *s_min, int32_t n_levels, int32_t mode,
                     const or_camera *cam, or_fp *out);

int64_t or_tile_lists(int64_t n, const or_fp *fp, int32_t tiles_x,
                      int32_t tiles_y, int64_t *offsets, uint32_t *idx,
                      int64_t capacity);

void or_sh_basis64(int32_t deg, const double dir[3], double *out);

void or_colors64(int64_t n, const float *mean, const float *color,
                 int32_t sh_degree, const or_camera *cam, double *rgb);

int64_t or_render64(int64_t n, const or_fp *fp, const float *opacity,
                    const double *rgb, const or_camera *cam,
                    const int64_t *offsets, const uint32_t *idx,
                    const int32_t *tile_sel, int32_t n_tile_sel,
                    double alpha_flag_rel, double t_flag_rel,
                    double *image, double *final_t, uint32_t *n_contrib,
                    uint8_t *flags, int64_t *n_eval);

int64_t or_render64_brute(int64_t n, const or_fp *fp, const float *opacity,
                          const double *rgb, const or_camera *cam,
                          double alpha_flag_rel, double *image,
                          double *final_t, uint8_t *flags);

/* Every result one pixel (centre px, py) may correctly take when the
 * decisions that render64.c flags are taken either way: up to max_alts rows
 * of (C0, C1, C2, T, n_contrib, n_eval) in out.  Returns the number of
 * rows, or -1 if there are more than max_alts. */
int32_t or_pixel_alternatives(const or_fp *fp, const float *opacity, const double *rgb,
                              const uint32_t *list, int64_t len, double px, double py,
                              double alpha_flag_rel, double t_flag_rel, int32_t max_alts,
                              double *out);

void or_update_range(int64_t n, const float *mean, const float *scale,
                     const float *quat, const float *lnop,
                     const uint8_t *level, int32_t n_levels,
                     int32_t level_r, const or_camera *cam, float *s_max,
                     float *s_min);

void or_coverage64(int64_t n, const float *mean, const float *log_scale,
                   const float *quat, const float *opacity,
                   const or_camera *cam, double *cover, double *ux,
                   double *uy, double *cov2d);

void or_forward64_full(int64_t n, const float *mean, const float *log_scale,
                       const float *quat, const float *opacity, const float *color,
                       int32_t sh_degree, const or_camera *cam, const int64_t *offsets,
                       const uint32_t *idx, double *image, double *final_t,
                       uint32_t *n_contrib, uint32_t *n_blend);

int64_t or_grad64(int64_t n, const float *mean, const float *log_scale, const float *quat,
                  const float *opacity, const float *color, int32_t sh_degree,
                  const or_camera *cam, const int64_t *offsets, const uint32_t *idx,
                  const double *dl_dimage, double *dmean, double *dlog_scale,
                  double *dquat, double *dopacity, double *dcolor);

/* Voxel key of a position for level l_m: per-component normalisation by
 * the camera extent B, floor(400 / l_m) voxels per axis over [-2, 2],
 * key = (vz R + vy) R + vx. */
uint32_t or_voxel_key(const float *mean3, float B, int32_t level_m);

/* AggregateGaussians for level l_m from n Gaussians (scale/lnop from
 * or_prepare) and n_cams cameras already downsampled by 4^(l_m-1).  Writes
 * the smallest coverage per Gaussian (+inf if none) to smin and up to
 * `capacity` new Gaussians in voxel-key order; returns their number. */
int64_t or_aggregate(int64_t n, const float *mean, const float *log_scale, const float *quat,
                     const float *opacity, const float *color, int32_t sh_degree,
                     const uint8_t *level, const float *scale, const float *lnop,
                     int32_t n_cams, const or_camera *cams, int32_t level_m, float B,
                     float *smin, float *o_mean, float *o_log_scale, float *o_quat,
                     float *o_opacity, float *o_color, uint32_t *o_key, int64_t capacity);

#ifdef __cplusplus
}
#endif
#endif

/*
 * msgs.h -- multi-scale selective Gaussian splatting on one GPU (sm_103a).
 *
 * C ABI of libmsgs.so: the rendering path of "Multi-Scale 3D Gaussian
 * Splatting for Anti-Aliased Rendering" (arXiv 2311.17089):
 *
 *   ms_scene_prepare  per-scene activations (exp(log_scale), ln(255 sigma))
 *   ms_project        EWA splat, pixel coverage, selection, SH colour
 *   ms_project_views  the same for up to MS_MAX_PROJ_VIEWS cameras in one pass
 *   ms_project_views_update  ... with UpdateRange fused for training renders
 *   ms_select         re-run the selection predicate on stored coverage
 *   ms_update_range   UpdateRange of the coverage bounds
 *   ms_bin            16x16 tile binning with a stable (tile, depth) order
 *   ms_raster         per-pixel front-to-back blend with early termination
 *   ms_raster_ex      the same with the blend's parallelisation chosen
 *   ms_raster_bwd     gradient of the image with respect to the scene
 *   ms_l1_loss_grad   L1 image loss and its gradient (training step)
 *   ms_aggregate      AggregateGaussians: insert a coarse level
 *   ms_serve_*        a render server: resident scenes, memory admission,
 *                     continuous batching of requests over CUDA streams
 *
 * Conventions shared by every call:
 *   - Every pointer inside ms_scene_t, ms_proj_t, ms_bins_t and every
 *     image pointer is DEVICE memory owned by the caller; the library never
 *     allocates, frees or retains a pointer past the call.  Arrays are
 *     dense, row-major, FP32 unless stated.  ms_camera_t is a host struct
 *     passed by value inside the call.
 *   - `stream` is a cudaStream_t (0 = legacy default stream).  Calls only
 *     enqueue work on it and return; nothing is synchronised unless the
 *     entry point says so.
 *   - Return value: MS_OK or an ms_status_t error; ms_last_error() gives a
 *     message for the calling thread.  Argument errors are detected before
 *     any work is enqueued.  Device-side conditions (duplicate capacity
 *     overflow, a bounded wait that gave up) are recorded in the device
 *     status word of ms_bins_t and reported by ms_bin_counts().
 *   - Camera: OpenCV axes (x right, y down, z forward), X_cam = R X_world + t,
 *     pixel (i, j) covers [i, i+1) x [j, j+1) and is sampled at its centre.
 */
#ifndef MSGS_H
#define MSGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MS_OK = 0,
    MS_ERR_INVALID_ARG = 1, /* bad size, null pointer, misaligned buffer */
    MS_ERR_CAPACITY = 2,    /* more tile duplicates than dup_capacity    */
    MS_ERR_CUDA = 3,        /* a CUDA runtime call failed                */
    MS_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up        */
    MS_ERR_NO_DEVICE = 5,   /* no usable sm_103 device                   */
    MS_PENDING = 6,         /* ms_serve_poll: the request has not finished */
    MS_ERR_OOM = 7,         /* serving: a request's buffers can never fit the
                               arena, or the arena could not be allocated   */
    MS_ERR_BOUNDS = 8       /* an index check of the debug build (libmsgs
                               compiled with -DMS_DEBUG) failed; the kernels
                               clamped or skipped the access (status bit 3) */
} ms_status_t;

/* Which Gaussians are rendered (Eq. 6 and the "Filter Small" ablation). */
typedef enum {
    MS_SELECTIVE = 0,    /* Eq. 6 with the level exemptions of Sec. 4.1    */
    MS_ALL_LEVELS = 1,   /* every valid Gaussian, all levels together      */
    MS_FILTER_SMALL = 2  /* second clause of Eq. 6 only, no exemption      */
} ms_mode_t;

/* How ms_raster_ex spreads a frame's blend over the GPU (the result is the
 * same blend either way, up to FP32 rounding). */
typedef enum {
    MS_RASTER_AUTO = 0,  /* LIST when the frame has fewer tiles than the GPU
                            has SMs; TILE from 4x as many, when
                            ms_raster_ex2 caps the tile kernel's CTAs, or
                            when the duplicate capacity is below 1024 per
                            tile; in between the frame's mean list length
                            decides on the device (LIST for 1024-8192
                            entries per tile)                               */
    MS_RASTER_TILE = 1,  /* one thread per pixel; long lists split into
                            segments merged exactly across CTAs             */
    MS_RASTER_LIST = 2,  /* one warp per pixel; only the list entries whose
                            level-set box reaches the pixel's half row are
                            blended, lanes take consecutive ones, a product
                            scan of (1 - alpha) decides termination        */
    MS_RASTER_GROUP8 = 3,  /* G = 8, 16 or 32 lanes per pixel, 4 consecutive */
    MS_RASTER_GROUP16 = 4, /* list entries per lane, one product scan over   */
    MS_RASTER_GROUP32 = 5  /* the group's lanes per 4 G entries              */
} ms_raster_strategy_t;

/*
 * A scene of n 3D Gaussians (Sec. 3.1: centre, covariance from scale and
 * rotation, opacity, colour; Sec. 4.1: level and coverage range).
 *   mean[n*3]       world centre
 *   log_scale[n*3]  log of the per-axis standard deviation
 *   quat[n*4]       rotation (w, x, y, z); any non-zero length; 16-B aligned
 *   opacity[n]      activated opacity sigma
 *   color           sh_degree >= 0: SH coefficients [n][(deg+1)^2][3],
 *                   16-B aligned; sh_degree == -1: plain RGB [n][3]
 *   level[n]        uint8 level, 1 (finest) .. n_levels (coarsest)
 *   s_max[n], s_min[n]  coverage range (read by ms_project, written by
 *                   ms_update_range); S_max = 0, S_min = +inf before any
 *                   update
 *   scale[n*3], lnop[n]  derived, written by ms_scene_prepare:
 *                   exp(log_scale) and ln(255 sigma), each evaluated in
 *                   FP64 and rounded to FP32
 * n <= 2^31 - 1, n_levels in 1..255, sh_degree in -1..3.
 */
typedef struct {
    int64_t n;
    int32_t n_levels;
    int32_t sh_degree;
    const float *mean;
    const float *log_scale;
    const float *quat;
    const float *opacity;
    const float *color;
    const uint8_t *level;
    float *s_max;
    float *s_min;
    float *scale;
    float *lnop;
} ms_scene_t;

/* Pinhole camera, host struct.  width, height >= 1; near_plane > 0. */
typedef struct {
    float R[9];      /* world -> camera rotation, row-major */
    float t[3];      /* world -> camera translation         */
    float campos[3]; /* camera centre in world coordinates  */
    float fx, fy, cx, cy;
    int32_t width, height;
    float near_plane;
    float bg[3];     /* background colour added as T_final * bg */
} ms_camera_t;

/*
 * Output of ms_project; device buffers sized for the scene's n.
 *   rec[n*12]     48-byte raster record of every listed Gaussian (selected
 *                 and touching >= 1 tile): ux, uy, A, B | C, opacity, r, g |
 *                 b, thr, ex, ey, where thr = -log2(e) ln(255 opacity) (so
 *                 alpha >= 1/255 exactly when power log2(e) >= thr),
 *                 (ex, ey) = the half extents sqrt(2 ln(255 opacity) V'_xx),
 *                 sqrt(2 ln(255 opacity) V'_yy) of the alpha >= 1/255 level
 *                 set (the box the tile rectangle is taken from) and
 *                 (A, B, C) = (k a, 2k b, k c), k =
 *                 -log2(e)/2 as an FP32 constant, each one FP32 product of
 *                 the conic (a, b, c) = inverse dilated covariance, so that
 *                 power * log2(e) = A dx^2 + B dx dy + C dy^2.  16-B aligned.
 *                 Entries of other Gaussians are left untouched.
 *   rect[n*2]     tile rectangle packed as (x0 | y0 << 16), (x1 | y1 << 16),
 *                 inclusive; written for every Gaussian, meaningful for
 *                 listed ones (others hold their footprint's rectangle,
 *                 possibly empty, or (0, 0xffffffff) when invalid or, in
 *                 ms_project_views, when the footprint was left out)
 *   n_tiles[n]    tiles covered if listed, else 0 (always written)
 *   depth[n]      bit pattern of view-space z, written for every Gaussian
 *                 (> 0 for listed ones)
 *   cover[n]      optional (may be NULL): pixel coverage S of every valid
 *                 Gaussian, -1 for invalid ones
 *   mask[(n+31)/32]  optional (may be NULL): selection bitset, bit i%32 of
 *                 word i/32 set iff Gaussian i is valid and selected
 *   stats[MS_STATS_WORDS]  uint32 counters written by ms_project and read
 *                 by ms_bin: survivors, duplicates, depth-digit histograms
 *   n             number of Gaussians the arrays hold (>= the scene's n);
 *                 kernels never index past it
 */
#define MS_STATS_WORDS 1040
typedef struct {
    float *rec;
    uint32_t *rect;
    uint32_t *n_tiles;
    uint32_t *depth;
    float *cover;
    uint32_t *mask;
    uint32_t *stats;
    int64_t n;
} ms_proj_t;

/*
 * Output of ms_bin.
 *   gauss_idx[dup_capacity]  Gaussian indices, grouped by tile in
 *                 row-major tile order, each group ordered by depth bits
 *                 then index
 *   ranges[tiles*2]  [start, end) of each tile's group in gauss_idx
 *   counts[4]     uint64 device words: [0] duplicates D (the number
 *                 needed, even when it exceeds the capacity), [1] survivor
 *                 count, [2] status bits (1 = capacity overflow, 2 = a
 *                 bounded wait gave up), [3] reserved
 *   dup_capacity  entries gauss_idx can hold, 1 .. 2^30 - 1
 */
typedef struct {
    uint32_t *gauss_idx;
    uint32_t *ranges;
    uint64_t *counts;
    int64_t dup_capacity;
} ms_bins_t;

/* Message describing the last error returned on the calling thread. */
const char *ms_last_error(void);

/* Library version, 100 * major + minor. */
int ms_version(void);

/*
 * Per-scene activations: scale = exp(log_scale), lnop = ln(255 * opacity)
 * = ln(sigma / sigma_T) with sigma_T = 1/255 (Sec. 4.1), both in FP64 then
 * rounded to FP32, so no transcendental enters the per-view footprint.
 * Run once per scene (and after the parameters change).
 */
int ms_scene_prepare(const ms_scene_t *scene, void *stream);

/*
 * Splat and select (Sec. 3.1, Sec. 3.2 Eq. 4, Sec. 4.1, Eq. 6; in Alg. 2 the
 * pixel coverage and the sets G1, G2).  For every Gaussian, in FP32 with a fixed
 * operation order: view transform, quaternion -> rotation, Sigma = R S^2
 * R^T, V = J W Sigma W^T J^T (Jacobian with the view ratio clamped to 1.3x
 * the half field of view), coverage S = sqrt(8 L det V / max(V_xx, V_yy))
 * on the undilated V, selection by `mode`, dilated V' = V + 0.3 I, its
 * conic, the level-set tile rectangle and, for listed Gaussians only, the
 * colour (SH of degree sh_degree evaluated towards the camera, + 0.5,
 * clamped at 0).  Valid = view z > near_plane, lnop > 0, det V' > 0 and
 * finite intermediates.
 */
int ms_project(const ms_scene_t *scene, const ms_camera_t *cam,
               ms_mode_t mode, const ms_proj_t *out, void *stream);

#define MS_MAX_PROJ_VIEWS 8

/*
 * ms_project for n_views cameras at once (1..MS_MAX_PROJ_VIEWS): outs[v]
 * receives, bit for bit, what ms_project(scene, &cams[v], mode, &outs[v])
 * writes, except the rectangles of Gaussians that are not listed (below).
 * One pass over the scene reads each Gaussian's geometry once and forms its
 * 3D covariance once; the camera-dependent steps run per view, and views
 * whose cameras share a centre (campos) share the listed Gaussians' SH
 * colour (the multi-scale setting of Sec. 4: one pose at several
 * resolutions).  When every view is a selective render with the first
 * view's R, t and campos, no cover output and no range update, the pass
 * leaves out the footprints that a bound on the coverage S (from one
 * covariance per Gaussian for all the views) shows cannot pass Eq. 6;
 * there, as for every Gaussian a view does not list, the rectangle is
 * (0, 0xffffffff).  cams and outs are host arrays of n_views entries
 * (read during the call only); the device buffers of the outs[v] are the
 * caller's and must not overlap one another.  Errors: MS_ERR_INVALID_ARG
 * for n_views outside 1..MS_MAX_PROJ_VIEWS, NULL cams/outs, or any camera
 * or output that ms_project would reject, all found before any work is
 * enqueued.
 */
int ms_project_views(const ms_scene_t *scene, const ms_camera_t *cams, int32_t n_views,
                     ms_mode_t mode, const ms_proj_t *outs, void *stream);

/*
 * ms_project_views for a multi-scale training step (Sec. 4.1 "Multi-Scale
 * Training", Alg. 2): view v with update_levels[v] = l_r >= 1 is rendered at
 * the creation scale 4^(l_r - 1) of level l_r, and after its selection
 * (which uses the coverage ranges as they stand) UpdateRange (Eq. 5)
 * updates, for every valid Gaussian of level l_r whose level-set rectangle
 * touches that view's image,
 *   s_max = max(0.95 s_max, S),  s_min = min(1.05 s_min, S)
 * in scene->s_max / scene->s_min (device arrays the call writes).  Views
 * are taken in order: view v + 1 selects with the ranges view v left, so
 * the outputs and the ranges equal those of n_views calls of ms_project,
 * each followed by ms_update_range for its level.  update_levels (host
 * array of n_views entries, 0..n_levels; 0 = the view updates nothing) may
 * be NULL (no view updates: ms_project_views).  Errors as ms_project_views,
 * and MS_ERR_INVALID_ARG for a level outside 0..n_levels.
 */
int ms_project_views_update(const ms_scene_t *scene, const ms_camera_t *cams, int32_t n_views,
                            ms_mode_t mode, const int32_t *update_levels,
                            const ms_proj_t *outs, void *stream);

/*
 * Selection predicate alone (Eq. 6, Sec. 4.1 exemptions) on a coverage
 * array produced by ms_project for the same scene: writes the bitset
 * mask[(n+31)/32].  cover < 0 marks invalid Gaussians (never selected).
 */
int ms_select(const ms_scene_t *scene, const float *cover, ms_mode_t mode,
              uint32_t *mask, void *stream);

/*
 * UpdateRange (Eq. 5, Alg. 2): for every valid Gaussian of level `level_r`
 * whose level-set rectangle touches the image of `cam`,
 *   s_max = max(0.95 s_max, S),  s_min = min(1.05 s_min, S).
 * The caller renders level l at its creation scale 4^(l-1) (Sec. 4.1).
 */
int ms_update_range(const ms_scene_t *scene, const ms_camera_t *cam,
                    int32_t level_r, void *stream);

/* Workspace bytes ms_bin needs for n Gaussians, `tiles` tiles and a
 * duplicate capacity; 0 on invalid sizes. */
size_t ms_bin_workspace_bytes(int64_t n, int64_t tiles, int64_t dup_capacity);

/*
 * Tile binning (Sec. 3.1: the Gaussians whose splats touch a tile are
 * listed for it in the order of their view depth).  n <= 2^30 - 1 (the
 * radix passes' digit counts are 30-bit).  Listed Gaussians are sorted by depth
 * bits with a stable LSD radix sort (ties keep index order), expanded to
 * one entry per covered tile in that order, and stably radix-sorted by tile
 * id, which yields every tile's list in (depth, index) order.  Fully
 * asynchronous; D is only known on the device: entries beyond
 * dup_capacity are dropped and status bit 1 set.  `ws` (16-B aligned) of
 * ms_bin_workspace_bytes(n, tiles, dup_capacity) bytes is scratch owned by
 * the call until the stream passes it.
 */
int ms_bin(const ms_proj_t *proj, int64_t n, const ms_camera_t *cam,
           const ms_bins_t *out, void *ws, size_t ws_bytes, void *stream);

/*
 * Binning of several frames of one pose (one camera at several
 * resolutions, as in a multi-scale sweep) with one shared depth sort.  A
 * Gaussian's view depth does not depend on the intrinsics, so the Gaussians
 * listed in any of the frames can be sorted by (depth bits, index) once;
 * each frame's tile lists then come from that order (directly, skipping the
 * Gaussians it does not list, or from its own part split off by
 * ms_split_order), and equal ms_bin's bit for bit.
 *
 * ms_project_views_union: ms_project_views that also forms the union of
 * the views whose bit is set in union_views (bit v: view v; at least one,
 * none at or above n_views; their cameras' R and t equal bitwise, else
 * MS_ERR_INVALID_ARG).  It writes union_flags[n] (the mask of those views
 * that list the Gaussian, bit v for view v; 0 if none) and
 * union_stats[MS_STATS_WORDS]
 * (16-B aligned; the union's count and its depth-digit histograms, zeroed
 * by the call).  The union's projection for ms_sort_depth is
 * { depth = outs[f].depth, n_tiles = union_flags, stats = union_stats,
 * n = outs[f].n }, f any view of the union (other fields unused).  The
 * other views are projected as by ms_project_views and bin with ms_bin.
 *
 * ms_sort_depth: the four stable depth passes of ms_bin over proj's listed
 * Gaussians (n_tiles > 0); writes their indices in (depth bits, index)
 * order to order[n] (device, caller-owned; the first union_stats survivors
 * entries are meaningful).  A wait that gives up is recorded in
 * proj->stats words 4-5 and reported by every ms_bin_ordered that uses the
 * order.  `ws` (16-B aligned) of ms_sort_depth_workspace_bytes(n) bytes.
 *
 * ms_split_order: the order of ms_sort_depth restricted to each view of
 * the union, in one pass: orders[v][0..s_v) receives, in the same order,
 * the Gaussians whose union_flags bit v is set (s_v = what view v lists),
 * and view_stats[v] (MS_STATS_WORDS words, 16-B aligned) receives s_v as
 * its survivor count and the union's status (the sort's waits and this
 * pass's) as its status.  union_proj is the sorted union (n_tiles =
 * union_flags, stats = union_stats); orders and view_stats are host arrays
 * of n_views (1..MS_MAX_PROJ_VIEWS) device pointers, each order of n
 * entries.  `ws` (16-B aligned) of ms_split_order_workspace_bytes(n) bytes.
 *
 * ms_bin_ordered: ms_bin for one frame, taking the depth order instead of
 * sorting: either the union's (order from ms_sort_depth, order_stats = the
 * union's stats) or the frame's own (orders[v] and view_stats[v] of
 * ms_split_order); the order must cover every Gaussian the frame lists.
 * Same workspace, outputs and errors as ms_bin.
 */
int ms_project_views_union(const ms_scene_t *scene, const ms_camera_t *cams, int32_t n_views,
                           ms_mode_t mode, const ms_proj_t *outs, uint32_t union_views,
                           uint32_t *union_flags, uint32_t *union_stats, void *stream);
size_t ms_sort_depth_workspace_bytes(int64_t n);
int ms_sort_depth(const ms_proj_t *proj, int64_t n, uint32_t *order, void *ws, size_t ws_bytes,
                  void *stream);
size_t ms_split_order_workspace_bytes(int64_t n);
int ms_split_order(const ms_proj_t *union_proj, int64_t n, const uint32_t *order,
                   int32_t n_views, uint32_t *const *orders, uint32_t *const *view_stats,
                   void *ws, size_t ws_bytes, void *stream);
int ms_bin_ordered(const ms_proj_t *proj, int64_t n, const ms_camera_t *cam,
                   const ms_bins_t *out, const uint32_t *order, const uint32_t *order_stats,
                   void *ws, size_t ws_bytes, void *stream);

/*
 * ms_bin for callers that cannot allocate device memory (the paper has no
 * counterpart; this is a deployment aid).  Examples are an engine plugin
 * whose host application owns every device allocation, and a render loop
 * under a fixed memory budget or a no-allocation rule on its frame thread.
 * Such callers cannot provide ms_bin's workspace.  This entry point takes
 * the same projection and output buffers as ms_bin, but its scratch space
 * is a static 16 MiB device array inside this library.  Every GPU that
 * loads the library keeps that array until the process exits.
 *   - Sizes whose ms_bin_workspace_bytes(n, tiles, dup_capacity) exceeds
 *     16 MiB are rejected with MS_ERR_INVALID_ARG and a message; nothing
 *     is enqueued.  For example, n = 262144 Gaussians with dup_capacity =
 *     524288 fits; larger scenes must use ms_bin with their own workspace.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current, and later calls on
 *     that device reuse it; first calls from several host threads at once
 *     are safe.  Make that first call before any stream capture on the
 *     device.  The address belongs to the device's primary context: after
 *     cudaDeviceReset the library must be unloaded and loaded again before
 *     this entry point is used on that device.
 *   - All calls share the one array.  Each call clears the parts that must
 *     start at zero, so nothing carries over between calls that run one
 *     after the other.  Calls that overlap on the GPU (different streams
 *     with no ordering between them) race on the array and corrupt each
 *     other's results.
 *   - No device memory is allocated or freed.
 */
int ms_bin_noalloc(const ms_proj_t *proj, int64_t n, const ms_camera_t *cam,
                   const ms_bins_t *out, void *stream);

/*
 * Copy the counts of a finished ms_bin to the host (synchronises
 * `stream`).  Returns MS_ERR_BOUNDS if an index check of the debug build
 * failed (in ms_bin or in an ms_raster that used these bins),
 * MS_ERR_TIMEOUT if a bounded wait gave up, MS_ERR_CAPACITY if D exceeded
 * the capacity (*d_needed tells how many are needed), else MS_OK.  Either
 * pointer may be NULL.
 */
int ms_bin_counts(const ms_bins_t *bins, int64_t *d_needed,
                  int64_t *survivors, void *stream);

/* Workspace bytes ms_raster needs for `tiles` tiles and the binning's
 * duplicate capacity; 0 on invalid sizes. */
size_t ms_raster_workspace_bytes(int64_t tiles, int64_t dup_capacity);

/*
 * Front-to-back blend (Sec. 3.1, Eq. 3), sampled at pixel centres.  For
 * each Gaussian of the tile's list in order: power = -(a dx^2 + c dy^2)/2
 * - b dx dy; skip if power > 0; alpha = min(0.99, sigma e^power); skip if
 * alpha < 1/255; stop before a Gaussian that would bring T below 1e-4;
 * C += alpha T rgb, T *= 1 - alpha.  Writes image[3][H][W] (planar,
 * C + T bg), final_t[H][W] and n_contrib[H][W] (1 + list position of the
 * last blended Gaussian, 0 if none).  n_eval[H][W] receives the number of
 * list entries the pixel evaluated up to and including the one that ended
 * it (the algorithmic work, for measurement).  final_t, n_contrib and
 * n_eval may be NULL.  `ws` (16-B aligned) of
 * ms_raster_workspace_bytes(tiles, dup_capacity) bytes is scratch owned by
 * the call until the stream passes it; it also keeps the per-segment state
 * ms_raster_bwd starts from.  A bounded wait that gives up sets status
 * bit 2 in bins->counts.  ms_raster uses MS_RASTER_AUTO.
 */
int ms_raster(const ms_proj_t *proj, const ms_bins_t *bins,
              const ms_camera_t *cam, float *image, float *final_t,
              uint32_t *n_contrib, uint32_t *n_eval, void *ws,
              size_t ws_bytes, void *stream);

/*
 * ms_raster with the blend's parallelisation chosen by `strategy`
 * (ms_raster_strategy_t; MS_ERR_INVALID_ARG for any other value).  Both
 * strategies compute the blend above (Sec. 3.1, Eq. 3) from the same tile
 * lists with the same FP32 alpha; they differ only in the rounding of the
 * transmittance products.
 */
int ms_raster_ex(const ms_proj_t *proj, const ms_bins_t *bins,
                 const ms_camera_t *cam, float *image, float *final_t,
                 uint32_t *n_contrib, uint32_t *n_eval, void *ws,
                 size_t ws_bytes, int strategy, void *stream);

/*
 * ms_raster_ex with the tile kernel's persistent CTAs capped at
 * max_ctas_per_sm per SM (0: as many as fit, as ms_raster_ex), so that the
 * kernels of other frames blended at the same time on other streams find
 * room beside it.  The frame's segmentation follows the number of CTAs (the
 * backward reads it from the workspace), so the blend's transmittance
 * products may round differently from ms_raster_ex's.  Negative values:
 * MS_ERR_INVALID_ARG.  The list and group kernels ignore the cap.
 */
int ms_raster_ex2(const ms_proj_t *proj, const ms_bins_t *bins,
                  const ms_camera_t *cam, float *image, float *final_t,
                  uint32_t *n_contrib, uint32_t *n_eval, void *ws,
                  size_t ws_bytes, int strategy, int32_t max_ctas_per_sm, void *stream);

/*
 * Gradients of a loss with respect to the scene parameters, outputs of
 * ms_raster_bwd; device buffers with the scene's shapes: dmean[n*3],
 * dlog_scale[n*3], dquat[n*4] (with respect to the unnormalised
 * quaternion), dopacity[n], dcolor (same layout as scene color).
 */
typedef struct {
    float *dmean;
    float *dlog_scale;
    float *dquat;
    float *dopacity;
    float *dcolor;
} ms_grads_t;

/* Workspace bytes ms_raster_bwd needs for n Gaussians (9 floats each, plus
 * a counter). */
size_t ms_raster_bwd_workspace_bytes(int64_t n);

/*
 * Backward of ms_project -> ms_bin -> ms_raster for one frame (the gradient
 * a multi-scale training step propagates, Sec. 4.1 "Multi-Scale
 * Training").  Inputs, all as that frame's forward left them: proj, bins,
 * the image and n_contrib written by ms_raster, and ms_raster's workspace
 * `raster_ws` (its tile segmentation and the per-pixel state after each
 * segment; raster_ws_bytes >= ms_raster_workspace_bytes(tiles,
 * bins->dup_capacity)); plus dl_dimage[3][H][W] (dL/d image, planar).
 * Every segment of every tile is walked front to back from the state the
 * forward reached before it, up to each pixel's last contributor,
 * recomputing every alpha with the forward's exact FP32 operations (so the
 * same Gaussians contribute).  With F_k the colour accumulated through
 * Gaussian k and C the pixel's final colour (background included):
 *   dC/dalpha_k = T_k c_k - (C - F_k) / (1 - alpha_k),  dC/dc_k = alpha_k T_k,
 * then through alpha = min(0.99, sigma e^power) (no gradient when clamped),
 * the centre and conic, V' = V + 0.3 I, the EWA covariance, the rotation of
 * the normalised quaternion, exp(log_scale) and the SH colour (direction
 * term included, zero where the colour was clamped at 0).  Gaussians the
 * frame did not blend get zero.  Selection and coverage are not
 * differentiated (the mask is discrete).  `ws` of
 * ms_raster_bwd_workspace_bytes(n) bytes (16-B aligned) holds the
 * per-Gaussian 2D gradients and is overwritten.  `flags` = 0 overwrites
 * every output (zero for Gaussians the frame did not blend);
 * MS_BWD_ACCUMULATE adds this frame's gradient to the outputs instead (a
 * batch of views: the first call overwrites, the others accumulate).
 * Sums are accumulated with float atomics, so the last bits of a gradient
 * may vary from run to run.
 */
#define MS_BWD_ACCUMULATE 1u
int ms_raster_bwd(const ms_scene_t *scene, const ms_camera_t *cam,
                  const ms_proj_t *proj, const ms_bins_t *bins, const float *image,
                  const uint32_t *n_contrib, const void *raster_ws, size_t raster_ws_bytes,
                  const float *dl_dimage, const ms_grads_t *grads, uint32_t flags,
                  void *ws, size_t ws_bytes, void *stream);

/*
 * One view of a batched backward: the inputs ms_raster_bwd takes for it.
 */
typedef struct {
    ms_camera_t cam;
    const ms_proj_t *proj;
    const ms_bins_t *bins;
    const float *image;
    const uint32_t *n_contrib;
    const void *raster_ws;
    size_t raster_ws_bytes;
    const float *dl_dimage;
} ms_bwd_view_t;

#define MS_MAX_BWD_VIEWS 8

/* Workspace bytes ms_raster_bwd_views needs: n_views x 9 floats per
 * Gaussian plus a counter; 0 for n_views outside 1..MS_MAX_BWD_VIEWS. */
size_t ms_raster_bwd_views_workspace_bytes(int64_t n, int32_t n_views);

/*
 * The backward of a batch of views of one scene (a multi-scale training
 * batch renders several views at different resolutions, Sec. 4.1): the
 * same result as ms_raster_bwd for views[0] followed by MS_BWD_ACCUMULATE
 * calls for the others, in two launches.  One raster pass takes the
 * segments of every view by ticket, each view's 2D gradients going to its
 * own part of `ws`; one projection pass then applies, per Gaussian, the
 * chain rule of every view that blended it and writes the sum once.
 * `flags` as for ms_raster_bwd, plus the pass selection: with
 * MS_BWD_RASTER_PASS alone only the raster pass runs (zeroing `ws` and
 * leaving the views' 2D gradients in it), with MS_BWD_PROJECT_PASS alone
 * only the projection pass (from the 2D gradients a raster pass left in
 * the same `ws`); neither or both: the two passes.
 */
#define MS_BWD_RASTER_PASS 2u
#define MS_BWD_PROJECT_PASS 4u
int ms_raster_bwd_views(const ms_scene_t *scene, const ms_bwd_view_t *views, int32_t n_views,
                        const ms_grads_t *grads, uint32_t flags, void *ws, size_t ws_bytes,
                        void *stream);

/*
 * L1 photometric loss of a training step (Sec. 4.1 trains with the image
 * loss of the single-scale method; its L1 term):
 *   dl_dimage[i] = weight * sign(image[i] - target[i])   (sign(0) = 0)
 *   *loss_sum   += weight * sum_i |image[i] - target[i]|  (if loss_sum)
 * over `count` FP32 values.  weight = 1 / count gives the mean.  All
 * pointers are device memory; loss_sum may be NULL, and it is accumulated
 * with atomics (zero it before the first view of a batch).  count = 0 is a
 * no-op.
 */
int ms_l1_loss_grad(const float *image, const float *target, int64_t count, float weight,
                    float *dl_dimage, float *loss_sum, void *stream);

/* ------------------------------------------------------------- aggregation
 *
 * AggregateGaussians (Alg. 1; Sec. 4.1 "Aggregate to Insert Large
 * Gaussians"; supplementary "Details of Gaussian Aggregation Algorithm")
 * for one coarse level level_m (2 .. scene->n_levels):
 *   - every Gaussian of levels < level_m is splatted to every camera in
 *     cams[n_cams] (host array: the training cameras ALREADY downsampled by
 *     4^(level_m - 1)); its smallest pixel coverage over the cameras where
 *     it is valid and touches the image decides: below S_T = 2 px it is
 *     small;
 *   - small Gaussians are binned by their position, normalised per
 *     component (x / B inside [-B, B], sign(x) (2 - B / |x|) outside, with
 *     B = extent, the half length of the cube spanned by the training
 *     cameras) on a grid of floor(400 / level_m) voxels per axis over
 *     [-2, 2]; voxel key = (vz R + vy) R + vx;
 *   - each voxel gives one new Gaussian of level level_m: the average of its
 *     members' mean, quat (as stored), log_scale, opacity and color, the
 *     log_scale then raised by ln(S_T / S_avg), S_avg the members' mean
 *     smallest coverage; s_max = 0 and s_min = +inf (no range yet).
 * New Gaussians are written to `out` (device arrays with the scene's
 * layout and sh_degree; out->n and out->n_levels are ignored) in
 * voxel-key order, at most `capacity`; n_out is a DEVICE int64[2]:
 * [0] = number of voxels (may exceed capacity: then only the first
 * `capacity` are written), [1] = status bits (MS status word, as in
 * ms_bins_t.counts).  The scene must be prepared (ms_scene_prepare).  The
 * caller appends the new Gaussians and repeats for the next level.
 */
size_t ms_aggregate_workspace_bytes(int64_t n);

int ms_aggregate(const ms_scene_t *scene, const ms_camera_t *cams, int32_t n_cams,
                 int32_t level_m, float extent, ms_scene_t *out, int64_t capacity,
                 int64_t *n_out, void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------ serving
 *
 * A render server keeps scenes resident on one device and renders camera
 * requests of any resolution (the 1x..128x multi-scale setting of Sec. 4)
 * as they arrive.  Admission is by memory: every request's buffers
 * (projection, tile lists, sort and raster workspaces, image) are carved
 * from one device arena of mem_budget_bytes allocated at creation; a
 * request waits in FIFO order until its buffers fit and fewer than
 * max_inflight requests are on the device.  Admitted requests are spread
 * over n_streams CUDA streams, so requests that arrive while others run
 * overlap with them on the GPU (continuous batching).  Requests for the
 * same scene and mode admitted together (the queue's head and later queued
 * requests that match it, up to max_batch_views) share one ms_project_views
 * pass: the scene's geometry is read once for all of them; each then bins
 * and blends on its own stream.  While requests are in flight, a head with
 * matching company waits until enough of max_inflight is free for the
 * batch.  A request that can never fit the arena
 * finishes with MS_ERR_OOM.  A request whose
 * tile duplicates overflow the capacity it was given is rendered again
 * with the exact count (ms_result_t.retries); the capacity of later
 * requests of the same scene, mode and tile grid is taken from the largest
 * count seen.  The paper defines no serving system; this is the runtime
 * around ms_project -> ms_bin -> ms_raster, whose results it leaves
 * unchanged: a request renders the same image alone or in a mix.
 */
typedef struct ms_server ms_server_t;

typedef struct {
    int64_t max_gaussians;     /* largest scene ms_serve_add_scene accepts     */
    int32_t max_width;         /* largest request image                        */
    int32_t max_height;
    int32_t max_inflight;      /* requests on the device at once, 1..1024      */
    int32_t n_streams;         /* CUDA streams, 1..max_inflight                */
    size_t mem_budget_bytes;   /* device arena for the requests' buffers       */
    int64_t initial_capacity;  /* tile duplicates assumed for a scene/mode/grid
                                  not seen yet (0: 2 n, at least 65536)         */
    int32_t device;            /* CUDA device ordinal                          */
    int32_t max_batch_views;   /* requests of one scene and mode admitted
                                  together share one projection pass
                                  (ms_project_views) of up to this many
                                  cameras, 1..MS_MAX_PROJ_VIEWS (0: the
                                  maximum; 1: one ms_project per request)    */
} ms_serve_cfg_t;

typedef struct {
    int32_t scene;             /* id from ms_serve_add_scene                   */
    int32_t mode;              /* ms_mode_t                                    */
    ms_camera_t cam;           /* width/height <= the configured maxima        */
    float *image_dev;          /* device [3][H][W] output, caller-owned; NULL:
                                  rendered into the server's arena             */
    float *image_host;         /* host [3][H][W] copy of the image (pinned for
                                  an asynchronous copy), or NULL               */
} ms_request_t;

typedef struct {
    int32_t status;            /* MS_OK, MS_PENDING, or the request's error    */
    int32_t retries;           /* re-renders after a capacity overflow         */
    int64_t duplicates;        /* tile duplicates of the frame                 */
    int64_t capacity;          /* duplicate capacity of its last render        */
    size_t bytes;              /* arena bytes its last render held             */
    double t_submit;           /* ms_serve_clock() at submission               */
    double t_start;            /* ... when its first render was enqueued       */
    double t_done;             /* ... when its image was complete              */
} ms_result_t;

typedef struct {
    int64_t submitted, completed, failed, retries;
    int32_t queued, inflight, peak_inflight, scenes;
    size_t arena_bytes, arena_used, arena_peak;
    int64_t renders;           /* renders enqueued (requests plus re-renders)  */
    double issue_seconds;      /* scheduler time spent enqueuing them: the
                                  host cost of the launches and copies         */
    int64_t proj_passes;       /* projection passes (one per admitted batch)   */
    double proj_seconds;       /* their summed GPU durations (CUDA events
                                  around each pass on its stream; passes that
                                  share the GPU with other work run longer)  */
} ms_serve_stats_t;

/* Seconds on the monotonic clock the server stamps results with. */
double ms_serve_clock(void);

/* Creates a server (allocates the arena and the streams on cfg->device and
 * starts its scheduler thread).  *out is NULL on failure. */
int ms_serve_create(const ms_serve_cfg_t *cfg, ms_server_t **out);

/* Registers a resident scene: its device arrays stay caller-owned and must
 * stay valid and unchanged until ms_serve_destroy; scale and lnop are
 * (re)computed here with ms_scene_prepare (synchronously). */
int ms_serve_add_scene(ms_server_t *srv, const ms_scene_t *scene, int32_t *scene_id);

/* Queues a request (copied); returns at once with its ticket.  image_dev
 * and image_host must stay valid until the request is done. */
int ms_serve_submit(ms_server_t *srv, const ms_request_t *req, uint64_t *ticket);

/* Non-blocking: res->status is MS_PENDING until the request is done.  A
 * poll that returns a finished result forgets the ticket. */
int ms_serve_poll(ms_server_t *srv, uint64_t ticket, ms_result_t *res);

/* Blocks until the request is done or timeout_s passes (then res->status
 * is MS_PENDING and the ticket stays valid). */
int ms_serve_wait(ms_server_t *srv, uint64_t ticket, double timeout_s, ms_result_t *res);

int ms_serve_stats(ms_server_t *srv, ms_serve_stats_t *stats);

/* Waits for the requests on the device, drops the queued ones, frees
 * everything.  srv may be NULL. */
int ms_serve_destroy(ms_server_t *srv);

/*
 * Test hook for the bounded device waits (the paper has no counterpart):
 * every look-back wait of ms_bin (the radix passes' and the duplication's
 * decoupled look-back) gives up after `limit` polls of a predecessor that
 * has not published, instead of the default (about half a second), sets
 * status bit 2 in ms_bins_t.counts and carries on with in-bounds writes;
 * ms_bin_counts then returns MS_ERR_TIMEOUT and the lists are not valid.
 * limit = 0 restores the default.  Process-wide; read when ms_bin enqueues
 * its kernels.  Only ms_bin is affected.  Returns MS_OK.
 */
int ms_debug_set_spin_limit(uint32_t limit);

/*
 * Measurement probes (the paper has no counterpart): the throughput of the
 * units the blend's roofline is stated against.  ms_alu_probe enqueues one
 * launch of `blocks` CTAs of 256 threads, each thread running 8 independent
 * chains of `iters` x 16 operations of one kind:
 *   MS_PROBE_FFMA   scalar fma.rn.f32            (1 FP32 operation each)
 *   MS_PROBE_FFMA2  packed fma.rn.f32x2          (2 FP32 operations each)
 *   MS_PROBE_EX2    ex2.approx.ftz.f32 on MUFU   (1 ex2 each)
 * and writes one float per thread to out[blocks * 256] (device memory owned
 * by the caller).  ms_alu_probe_ops returns the operations one such launch
 * performs (0 on invalid arguments); the caller times the launch with CUDA
 * events on `stream` and divides.  Errors: MS_ERR_INVALID_ARG, MS_ERR_CUDA.
 */
enum { MS_PROBE_FFMA = 0, MS_PROBE_FFMA2 = 1, MS_PROBE_EX2 = 2 };
int ms_alu_probe(int kind, int blocks, int iters, float *out, void *stream);
double ms_alu_probe_ops(int kind, int blocks, int iters);

#ifdef __cplusplus
}
#endif
#endif

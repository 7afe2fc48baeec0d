// List-parallel front-to-back blend (raster_list.cu): the launcher the
// ms_raster entry point calls for frames with few tiles.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace msgs {

struct ListArgs {
    const uint32_t *ranges;   // [tiles][2] list range of each tile
    const uint32_t *gidx;     // sorted Gaussian indices of all tile lists
    const float4 *rec;        // [n_rec][3] raster records
    uint32_t n_rec;
    int W, H, tiles_x, tiles;
    float bg0, bg1, bg2;
    float *image;             // [3][H][W]
    float *final_t;           // [H][W] or NULL
    uint32_t *n_contrib;      // [H][W] or NULL
    uint32_t *n_eval;         // [H][W] or NULL
    const uint32_t *seg_off;  // [tiles + 1] the frame's segmentation (segment_offsets_kernel)
    const uint32_t *seg_len;  // [1] entries per segment
    float4 *pre;              // [max_segs][256] state after each segment, for the backward
    uint32_t *rowmask;        // [dup_capacity] half rows each list entry reaches (workspace)
    const uint32_t *use_list; // NULL, or 0 when the tile kernel blends this frame instead
    uint32_t max_segs;        // upper bound of the frame's segment count
    unsigned long long *err;  // status word (the binning's), for debug-build checks
};

// Pixels one CTA of the list kernel blends: a row of 8 pixels of a tile,
// one warp each.
constexpr int kListPixelsPerCta = 8;
constexpr int kListCtasPerTile = 256 / kListPixelsPerCta;

// Enqueue the list-parallel blend of every tile on `st`: the half-row masks
// of every list entry, then the blend (no waits, no workspace zeroing
// needed).
cudaError_t launch_raster_list(const ListArgs &a, cudaStream_t st);

// Enqueue the group blend (raster_group.cu): each pixel's list walked by a
// group of `group` lanes (8, 16 or 32), 4 consecutive entries per lane.
cudaError_t launch_raster_group(const ListArgs &a, int group, cudaStream_t st);

}  // namespace msgs

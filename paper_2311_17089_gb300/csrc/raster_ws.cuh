// Layout of the ms_raster workspace.  The backward reads the forward's
// segmentation and per-segment prefix states from it, so both sides take
// the offsets from this one function.
#pragma once

#include <stdint.h>

#include <algorithm>

#include "common.cuh"

namespace msgs {

constexpr int kRasterThreads = 256;          // one thread per pixel of a 16x16 tile
constexpr int kChunk = 128;                  // records per staged sub-batch
#ifndef MS_MIN_SEGMENT_CHUNKS
#define MS_MIN_SEGMENT_CHUNKS 2
#endif
// shortest segment a tile is cut into
constexpr uint32_t kMinSegment = MS_MIN_SEGMENT_CHUNKS * kChunk;
constexpr uint32_t kTermBit = 0x80000000u;   // pixel terminated (in the n_eval word)
// Most CTAs a raster launch runs at once.  The segment length is at least
// D / resident, so a frame has at most tiles + min(D / kMinSegment,
// resident) segments; the workspace holds state for that many.
constexpr int64_t kMaxResident = 4096;

// Byte offsets inside the workspace.  ticket, flags and tile_done are zeroed
// by every ms_raster call (zero_bytes); seg_len, use_list (which of the two
// blend kernels a frame takes when both are launched) and seg_off are
// written by its first kernel; agg/agg2 hold segment-local aggregates and pre/pre2 the
// inclusive prefix state (C0, C1, C2, T) / (n_contrib, n_eval | term) per
// segment and pixel, for every segment but a tile's last; rowmask holds,
// for the list kernel, one word per tile-list entry: bit 2 r + h set when
// the entry's level-set box reaches half h of the tile's pixel row r.
struct RasterLayout {
    size_t ticket, seg_len, use_list, flags, tile_done, seg_off, agg, agg2, pre, pre2, rowmask,
        total, zero_bytes;
    int64_t max_segs;
};

// Slot of tile pixel (x, y) (0..15 each) in a segment's per-pixel state
// arrays: the tile kernel's thread layout, where warp w covers the 8x4 block
// ((w & 1) * 8, (w >> 1) * 4) and lane l its pixel (l & 7, l >> 3).  Both
// forward kernels store prefix states in this order and the backward reads
// them in it.
__host__ __device__ __forceinline__ int fwd_index(int x, int y) {
    return ((y >> 2) * 2 + (x >> 3)) * 32 + (y & 3) * 8 + (x & 7);
}

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

inline bool raster_layout(int64_t tiles, int64_t cap, RasterLayout &L) {
    if (tiles < 1 || tiles > 65536 || cap < 1 || cap > (1ll << 30) - 1) return false;
    L.max_segs = tiles + std::min(ceil_div(cap, (int64_t)kMinSegment), kMaxResident);
    size_t o = 0;
    L.ticket = o;
    o = al256(o + 4);
    L.flags = o;
    o = al256(o + (size_t)L.max_segs * 4);
    L.tile_done = o;
    o = al256(o + (size_t)tiles * 4);
    L.zero_bytes = o;
    L.seg_len = o;
    L.use_list = o + 4;
    o = al256(o + 8);
    L.seg_off = o;
    o = al256(o + (size_t)(tiles + 1) * 4);
    const size_t per4 = (size_t)L.max_segs * kRasterThreads * 16;
    const size_t per2 = (size_t)L.max_segs * kRasterThreads * 8;
    L.agg = o;
    o = al256(o + per4);
    L.agg2 = o;
    o = al256(o + per2);
    L.pre = o;
    o = al256(o + per4);
    L.pre2 = o;
    o = al256(o + per2);
    L.rowmask = o;
    o = al256(o + (size_t)cap * 4);
    L.total = o;
    return true;
}

}  // namespace msgs

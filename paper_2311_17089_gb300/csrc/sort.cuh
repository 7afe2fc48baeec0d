// The onesweep radix pass (one stable LSD step over 8-bit digits with
// decoupled look-back), shared by tile binning and the aggregation of
// small Gaussians.  Defined in bin.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace msgs {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
// Items per thread of a partition (2048-item partitions).  Passes over at
// most kSmallPassItems items run 2 CTAs per SM, so that the frames rendered
// at once share the GPU; larger passes 4, for more loads in flight (their
// 16-item, 2-CTA variant was 1-4% slower on the large passes).
constexpr int kSmallIPT = 8;
constexpr int kLargeIPT = 8;
constexpr uint64_t kSmallPassItems = 2ull << 20;
constexpr int kSmallPassCtasPerSm = 2;
constexpr int kLargePassCtasPerSm = 4;
constexpr int kDigits = 256;
constexpr int kScanWarps = kDigits / 32;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPre = 2u << 30;
constexpr uint32_t kFlagMask = 3u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;
// Most items a pass may sort: the look-back words carry 30-bit digit counts.
constexpr int64_t kMaxSortItems = (1ll << 30) - 1;
constexpr int kLookback = 16;  // predecessors polled per look-back step

template <int IPT>
struct SortCfg {
    static constexpr int kPart = kSortThreads * IPT;  // items per partition
    static constexpr int kSmem = (kSortWarps * kDigits + 2 * kPart) * 4;
};

// Partition size of a pass over at most `bound` items.
inline uint64_t sort_part(uint64_t bound) {
    return bound <= kSmallPassItems ? SortCfg<kSmallIPT>::kPart : SortCfg<kLargeIPT>::kPart;
}
inline int64_t sort_parts(uint64_t bound) {
    return (int64_t)((bound + sort_part(bound) - 1) / sort_part(bound));
}

struct PassArgs {
    const uint32_t *keys_in;
    const uint32_t *vals_in;    // nullptr: value = item index
    const uint32_t *filter;     // nullptr, or item valid iff filter[i] > 0
    uint32_t *keys_out;         // nullptr: keys not written
    uint32_t *vals_out;
    const uint32_t *n32;        // device item count (u32) or nullptr
    const unsigned long long *n64;  // device item count (u64) or nullptr
    uint64_t n_cap;             // count = min(device count, n_cap); or n_cap alone
    int shift;
    const uint32_t *hist;       // [256] digit totals of this pass
    uint32_t *status;           // [partitions][256]
    uint32_t *ticket;
    unsigned long long *err;    // status word (bit kStatusTimeout)
    uint32_t spin_limit = kSpinLimit;  // look-back polls before a wait gives up
    int ctas_per_sm = 0;               // 0: by the pass's size (below); else this many
};

// One pass: items [0, count) (count from n32 / n64 / n_cap; only items with
// filter[i] > 0 when a filter is given, compacted in index order) are
// scattered stably by digit (key >> shift) & 255 into keys_out/vals_out.
// hist holds the digit totals of the items taken; status must hold
// sort_parts(bound) x 256 zeroed words and ticket one zeroed word, `bound`
// being an upper bound of count known on the host (it picks the partition
// size and the grid).  Defined in bin.cu.
int launch_onesweep(const PassArgs &a, uint64_t bound, cudaStream_t st);

}  // namespace msgs

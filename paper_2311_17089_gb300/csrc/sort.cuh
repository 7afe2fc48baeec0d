// The onesweep radix pass (one stable LSD step over 8-bit digits with
// decoupled look-back), shared by tile binning and the aggregation of
// small Gaussians.  Defined in bin.cu.
#pragma once

#include <stdint.h>

namespace msgs {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortIPT = 16;
constexpr int kPart = kSortThreads * kSortIPT;  // items per partition
constexpr int kDigits = 256;
constexpr int kScanWarps = kDigits / 32;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPre = 2u << 30;
constexpr uint32_t kFlagMask = 3u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;
constexpr int kLookback = 16;  // predecessors polled per look-back step

constexpr int kSortSmem = (kSortWarps * kDigits + 2 * kPart) * 4;

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
};

// One pass: items [0, count) (count from n32 / n64 / n_cap; only items with
// filter[i] > 0 when a filter is given, compacted in index order) are
// scattered stably by digit (key >> shift) & 255 into keys_out/vals_out.
// hist holds the digit totals of the items taken; status must hold
// ceil(count / kPart) x 256 zeroed words and ticket one zeroed word.
__global__ void onesweep_pass(PassArgs a);

}  // namespace msgs

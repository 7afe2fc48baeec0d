// Host-side first-fit allocator over one byte range [0, size), the render
// server's device arena (serve.cu): free ranges keyed by offset, a request
// takes the lowest-offset range that holds it, and a released range is
// merged with its free neighbours.  Plain C++, no CUDA: offsets only.
#pragma once

#include <algorithm>
#include <cstddef>
#include <iterator>
#include <map>

namespace msgs {

class Arena {
  public:
    void init(size_t size) {
        size_ = size;
        free_.clear();
        if (size) free_[0] = size;
        used_ = peak_ = 0;
    }
    // Takes `bytes` from the lowest-offset free range that holds them;
    // false (and nothing taken) when no range does.
    bool alloc(size_t bytes, size_t &off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            off = it->first;
            const size_t rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[off + bytes] = rest;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }
    // Returns a range that alloc handed out (the caller keeps its offset
    // and size).
    void release(size_t off, size_t bytes) {
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }
    const std::map<size_t, size_t> &free_ranges() const { return free_; }

  private:
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

}  // namespace msgs

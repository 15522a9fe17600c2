// First-fit allocator over one device arena, the serving loop's admission
// cap: offsets into the arena in 256-byte granules; a released range merges
// with free neighbours.  Host code only (no CUDA), so it is tested on its
// own.
#pragma once

#include <cstdint>
#include <iterator>
#include <map>

namespace rk {

class Arena {
  public:
    static constexpr uint64_t kGranule = 256;

    // Bytes a request of n bytes occupies (an empty one still takes a
    // granule).  An arena of round_up(cap) bytes admits every n <= cap when
    // empty.
    static uint64_t round_up(uint64_t n) {
        return n ? (n + kGranule - 1) / kGranule * kGranule : kGranule;
    }

    // bytes: the arena's size, a multiple of kGranule.
    void reset(uint64_t bytes) {
        free_.clear();
        sizes_.clear();
        if (bytes) free_[0] = bytes;
        used_ = 0;
    }

    // The lowest free offset with room for n bytes; false when no free range
    // is large enough.
    bool alloc(uint64_t n, uint64_t *off) {
        n = round_up(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const uint64_t rest = it->second - n, at = it->first + n;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used_ += n;
            sizes_[*off] = n;
            return true;
        }
        return false;
    }

    // Free the allocation at off (an offset alloc did not return is ignored).
    void release(uint64_t off) {
        auto s = sizes_.find(off);
        if (s == sizes_.end()) return;
        uint64_t n = s->second;
        sizes_.erase(s);
        used_ -= n;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + n == next->first) {
            n += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += n;
                return;
            }
        }
        free_[off] = n;
    }

    uint64_t used() const { return used_; }
    size_t free_ranges() const { return free_.size(); }

  private:
    std::map<uint64_t, uint64_t> free_;   // offset -> bytes
    std::map<uint64_t, uint64_t> sizes_;  // allocated offset -> bytes
    uint64_t used_ = 0;
};

}  // namespace rk

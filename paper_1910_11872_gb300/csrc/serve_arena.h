// serve_arena.h -- first-fit range allocator over a fixed capacity of units (host code only).
//
// The serving loop carves one device arena (allocated once, under the HBM budget) into the frame
// slots of its camera streams; this class does the bookkeeping of which ranges of the arena are
// free. Free ranges are kept coalesced, so releasing every allocation restores one range of the
// full capacity. Allocation is first fit with an alignment in units.
#pragma once

#include <stdint.h>

#include <iterator>
#include <map>

namespace rmusic {

class RangeAllocator {
   public:
    explicit RangeAllocator(uint64_t capacity = 0) { reset(capacity); }

    void reset(uint64_t capacity) {
        capacity_ = capacity;
        free_.clear();
        used_.clear();
        if (capacity) free_[0] = capacity;
    }

    // Find `n` free units starting at a multiple of `align`; false if no free range fits.
    bool allocate(uint64_t n, uint64_t align, uint64_t* off) {
        if (n == 0 || align == 0) return false;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            const uint64_t start = it->first, len = it->second;
            const uint64_t a = (start + align - 1) / align * align;
            if (a < start || a - start > len || len - (a - start) < n) continue;
            free_.erase(it);
            if (a > start) free_[start] = a - start;
            const uint64_t tail = start + len - (a + n);
            if (tail) free_[a + n] = tail;
            used_[a] = n;
            *off = a;
            return true;
        }
        return false;
    }

    // Return a range obtained from allocate(); false if (off, n) is not a live allocation.
    bool release(uint64_t off, uint64_t n) {
        auto u = used_.find(off);
        if (u == used_.end() || u->second != n) return false;
        used_.erase(u);
        uint64_t start = off, len = n;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && next->first == off + n) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == start) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = len;
        return true;
    }

    uint64_t capacity() const { return capacity_; }
    uint64_t free_units() const {
        uint64_t s = 0;
        for (auto& kv : free_) s += kv.second;
        return s;
    }
    uint64_t largest_free() const {
        uint64_t m = 0;
        for (auto& kv : free_) m = kv.second > m ? kv.second : m;
        return m;
    }
    size_t free_ranges() const { return free_.size(); }
    size_t live() const { return used_.size(); }

   private:
    uint64_t capacity_ = 0;
    std::map<uint64_t, uint64_t> free_;  // start -> length, coalesced
    std::map<uint64_t, uint64_t> used_;  // start -> length of live allocations
};

}  // namespace rmusic

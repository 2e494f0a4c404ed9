// First-fit allocator over one reserved byte range (offsets only, no memory of
// its own): the serving loop carves request workspaces out of a single device
// allocation sized by the device-memory budget. Host-only and header-only so that
// its bookkeeping can be tested without a GPU.
#pragma once

#include <stddef.h>

#include <map>

namespace msadp {

class Arena {
  public:
    static constexpr size_t kAlign = 256;

    explicit Arena(size_t capacity = 0) { reset(capacity); }

    // Forget every allocation; the whole range is free.
    void reset(size_t capacity) {
        cap_ = capacity / kAlign * kAlign;
        free_.clear();
        used_.clear();
        in_use_ = 0;
        if (cap_) free_[0] = cap_;
    }

    // Lowest-addressed free block that fits `bytes` (rounded up to kAlign).
    bool alloc(size_t bytes, size_t *off) {
        const size_t need = round(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const size_t o = it->first, rest = it->second - need;
            free_.erase(it);
            if (rest) free_[o + need] = rest;
            used_[o] = need;
            in_use_ += need;
            *off = o;
            return true;
        }
        return false;
    }

    // Return a block; neighbouring free blocks merge. False for an unknown offset.
    bool release(size_t off) {
        auto u = used_.find(off);
        if (u == used_.end()) return false;
        size_t o = off, n = u->second;
        used_.erase(u);
        in_use_ -= n;
        auto next = free_.lower_bound(o);
        if (next != free_.end() && o + n == next->first) {
            n += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == o) {
                prev->second += n;
                return true;
            }
        }
        free_[o] = n;
        return true;
    }

    // Would a request of `bytes` fit in an empty arena?
    bool could_ever_fit(size_t bytes) const { return round(bytes ? bytes : 1) <= cap_; }
    size_t capacity() const { return cap_; }
    size_t in_use() const { return in_use_; }
    size_t blocks() const { return used_.size(); }
    size_t largest_free() const {
        size_t m = 0;
        for (const auto &f : free_) m = f.second > m ? f.second : m;
        return m;
    }

  private:
    static size_t round(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
    size_t cap_ = 0, in_use_ = 0;
    std::map<size_t, size_t> free_;  // offset -> bytes, address order
    std::map<size_t, size_t> used_;  // offset -> bytes
};

}  // namespace msadp

// serve_arena.h — host-side parts of the serving loop that need no GPU: the
// allocator of the server's device arena (the HBM budget) and the admission
// rule. Plain C++ so that it can be unit-tested without a device.
#pragma once
#include <cstdint>
#include <deque>
#include <iterator>
#include <map>

namespace hz {
namespace serve {

// First-fit allocator over [0, size) with 256-byte granules. Blocks are
// identified by their offset. shrink() returns the tail of a block.
class Arena {
 public:
  static constexpr uint64_t kAlign = 256;

  explicit Arena(uint64_t size = 0) { reset(size); }

  void reset(uint64_t size) {
    size_ = size / kAlign * kAlign;
    free_.clear();
    used_.clear();
    in_use_ = peak_ = 0;
    if (size_) free_[0] = size_;
  }

  static uint64_t round(uint64_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

  // Offset of a new block of at least `bytes` (0 bytes takes one granule).
  bool alloc(uint64_t bytes, uint64_t* off) {
    const uint64_t need = round(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= need) {
        const uint64_t o = it->first, sz = it->second;
        free_.erase(it);
        if (sz > need) free_[o + need] = sz - need;
        used_[o] = need;
        in_use_ += need;
        if (in_use_ > peak_) peak_ = in_use_;
        *off = o;
        return true;
      }
    }
    return false;
  }

  // Frees a whole block; false if `off` is not a block.
  bool release(uint64_t off) {
    auto it = used_.find(off);
    if (it == used_.end()) return false;
    const uint64_t sz = it->second;
    used_.erase(it);
    in_use_ -= sz;
    insert_free(off, sz);
    return true;
  }

  // Keeps the first `bytes` of the block at `off` and frees the rest.
  bool shrink(uint64_t off, uint64_t bytes) {
    auto it = used_.find(off);
    if (it == used_.end()) return false;
    const uint64_t keep = round(bytes ? bytes : 1);
    if (keep >= it->second) return true;
    const uint64_t tail = it->second - keep;
    it->second = keep;
    in_use_ -= tail;
    insert_free(off + keep, tail);
    return true;
  }

  uint64_t size() const { return size_; }
  uint64_t in_use() const { return in_use_; }
  uint64_t peak() const { return peak_; }
  uint64_t largest_free() const {
    uint64_t m = 0;
    for (const auto& f : free_) m = f.second > m ? f.second : m;
    return m;
  }
  size_t blocks() const { return used_.size(); }

 private:
  void insert_free(uint64_t off, uint64_t sz) {
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && off + sz == nx->first) {  // merge with the next free range
      sz += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {  // merge with the previous free range
      auto pv = std::prev(nx);
      if (pv->first + pv->second == off) {
        pv->second += sz;
        return;
      }
    }
    free_[off] = sz;
  }

  uint64_t size_ = 0, in_use_ = 0, peak_ = 0;
  std::map<uint64_t, uint64_t> free_;  // offset -> bytes
  std::map<uint64_t, uint64_t> used_;  // offset -> bytes
};

// Admission rule. Requests are taken in arrival order; a request that needs
// no output memory (a reduction) may pass a head that waits for memory, and
// nothing else may, so a large request is never starved by smaller ones.
// Returns the position in `pending` of the request to start next (its block
// already allocated into *off), or -1 when none can start.
template <class Req, class NeedFn>
long pick_next(const std::deque<Req>& pending, uint64_t now_us, Arena& arena, NeedFn&& need,
               uint64_t* off) {
  bool head_blocked = false;
  for (size_t i = 0; i < pending.size(); i++) {
    const Req& r = pending[i];
    if (r.arrival_us > now_us) break;  // arrival order: later ones have not arrived either
    const uint64_t b = need(r);
    if (!head_blocked) {
      if (b == 0) {
        *off = ~0ull;
        return (long)i;
      }
      if (arena.alloc(b, off)) return (long)i;
      head_blocked = true;
    } else if (b == 0) {
      *off = ~0ull;
      return (long)i;
    }
  }
  return -1;
}

}  // namespace serve
}  // namespace hz

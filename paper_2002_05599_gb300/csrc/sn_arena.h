// First-fit range allocator over a fixed byte range [0, capacity).
//
// Host-only C++ (no CUDA), used by the request server to carve the device
// memory of admitted requests out of one resident device buffer.  Offsets are
// aligned to `kAlign`; freed ranges are merged with their free neighbours, so
// the free list never holds two adjacent ranges.  Not thread-safe: the server
// calls it under its own lock.
#pragma once

#include <cstdint>
#include <iterator>
#include <map>

namespace sn {

class RangeArena {
 public:
  static constexpr uint64_t kAlign = 256;
  static constexpr uint64_t kFail = ~0ull;

  explicit RangeArena(uint64_t capacity = 0) { reset(capacity); }

  void reset(uint64_t capacity) {
    cap_ = capacity & ~(kAlign - 1);
    used_ = 0;
    free_.clear();
    live_.clear();
    if (cap_) free_[0] = cap_;
  }

  static uint64_t round_up(uint64_t bytes) { return (bytes + kAlign - 1) & ~(kAlign - 1); }

  // Offset of a new range of `bytes` (rounded up to kAlign), or kFail when no
  // free range is large enough.  A zero-byte request still takes kAlign bytes.
  uint64_t alloc(uint64_t bytes) {
    const uint64_t need = round_up(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < need) continue;
      const uint64_t at = it->first;
      const uint64_t left = it->second - need;
      free_.erase(it);
      if (left) free_[at + need] = left;
      live_[at] = need;
      used_ += need;
      return at;
    }
    return kFail;
  }

  // Returns false (and changes nothing) if `at` is not the start of a live range.
  bool release(uint64_t at) {
    auto lv = live_.find(at);
    if (lv == live_.end()) return false;
    uint64_t start = at, size = lv->second;
    used_ -= size;
    live_.erase(lv);
    auto next = free_.lower_bound(start);
    if (next != free_.end() && next->first == start + size) {
      size += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == start) {
        start = prev->first;
        size += prev->second;
        free_.erase(prev);
      }
    }
    free_[start] = size;
    return true;
  }

  // Whether a range of `bytes` could ever fit (ignoring current use).
  bool fits_at_all(uint64_t bytes) const { return round_up(bytes ? bytes : 1) <= cap_; }

  uint64_t capacity() const { return cap_; }
  uint64_t used() const { return used_; }
  uint64_t largest_free() const {
    uint64_t m = 0;
    for (const auto& f : free_) m = f.second > m ? f.second : m;
    return m;
  }
  size_t free_ranges() const { return free_.size(); }
  size_t live_ranges() const { return live_.size(); }

  // Invariants for tests: free and live ranges tile [0, cap) exactly, free
  // ranges are never adjacent, and `used` is the sum of the live sizes.
  bool check() const {
    std::map<uint64_t, std::pair<uint64_t, bool>> all;
    for (const auto& f : free_) all[f.first] = {f.second, true};
    for (const auto& l : live_) {
      if (all.count(l.first)) return false;
      all[l.first] = {l.second, false};
    }
    uint64_t pos = 0, live_sum = 0;
    bool prev_free = false;
    for (const auto& r : all) {
      if (r.first != pos || r.second.first == 0 || r.first % kAlign) return false;
      if (r.second.second && prev_free) return false;
      prev_free = r.second.second;
      if (!r.second.second) live_sum += r.second.first;
      pos += r.second.first;
    }
    return pos == cap_ && live_sum == used_;
  }

 private:
  uint64_t cap_ = 0, used_ = 0;
  std::map<uint64_t, uint64_t> free_;  // start -> size
  std::map<uint64_t, uint64_t> live_;  // start -> size
};

}  // namespace sn

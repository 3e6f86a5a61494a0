// gp_arena.h -- the allocator of a pool's device arena (host code: it hands out
// byte offsets and never touches device memory).  First fit over [0, capacity) with a
// coalescing free list kept in offset order; every allocation is rounded up to
// kArenaAlign bytes, so every offset it returns is kArenaAlign-aligned.
#pragma once

#include <algorithm>
#include <cstddef>
#include <iterator>
#include <map>

namespace gp_arena {

constexpr size_t kArenaAlign = 256;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

class Arena {
 public:
  void reset(size_t cap) {
    cap_ = cap;
    free_.clear();
    if (cap) free_[0] = cap;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(bytes, kArenaAlign);
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes, kArenaAlign);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t free_total() const {
    size_t t = 0;
    for (const auto& f : free_) t += f.second;
    return t;
  }
  size_t largest() const {
    size_t m = 0;
    for (const auto& f : free_) m = std::max(m, f.second);
    return m;
  }
  // end of the highest allocated byte
  size_t high_water() const {
    if (free_.empty()) return cap_;
    const auto& last = *free_.rbegin();
    return last.first + last.second == cap_ ? last.first : cap_;
  }

 private:
  size_t cap_ = 0;
  std::map<size_t, size_t> free_;
};

}  // namespace gp_arena

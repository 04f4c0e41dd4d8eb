// ga_arena.h -- host bookkeeping of the alignment server's device arena
// (plain C++, no CUDA): a first-fit allocator of byte ranges and the code
// slabs that admitted requests' codes are bump-allocated from.
#pragma once

#include <algorithm>
#include <cstdint>
#include <iterator>
#include <map>
#include <vector>

namespace ga {

// First-fit allocator of byte ranges of the device arena (host bookkeeping).
class ArenaAlloc {
 public:
  explicit ArenaAlloc(int64_t size) : size_(size) { free_[0] = size; }
  int64_t alloc(int64_t bytes) {
    bytes = (bytes + 255) & ~(int64_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const int64_t off = it->first, rest = it->second - bytes;
        free_.erase(it);
        if (rest) free_[off + bytes] = rest;
        used_ += bytes;
        high_ = std::max(high_, used_);
        return off;
      }
    }
    return -1;
  }
  void release(int64_t off, int64_t bytes) {
    bytes = (bytes + 255) & ~(int64_t)255;
    used_ -= bytes;
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
  int64_t high_water() const { return high_; }

 private:
  int64_t size_, used_ = 0, high_ = 0;
  std::map<int64_t, int64_t> free_;
};

// Codes of admitted requests are bump-allocated from slabs of the arena, so
// the codes admitted in one scheduler tick sit back to back in the arena as
// they do in the pinned staging buffer and reach the device in one copy
// (a copy per request cost more host time than everything else the
// admission does).  A slab goes back to the arena when the last request
// placed in it completes and it is no longer the one being filled; the slab
// being filled restarts from its beginning once all of its requests are
// done.  A slab that cannot be had at full size is cut to the request, and
// an idle slab is given back when a request's edges find no room, so that
// any request that fits an empty arena is still admitted.
class CodeSlabs {
 public:
  explicit CodeSlabs(int64_t arena_bytes)
      : slab_(std::min<int64_t>(16ll << 20, std::max<int64_t>(64ll << 10, arena_bytes / 64)) & ~255ll) {}
  // Arena offset of `bytes` (a multiple of 256) and the slab's id, or -1.
  int64_t alloc(ArenaAlloc &arena, int64_t bytes, int *id) {
    if (cur_ >= 0 && slabs_[cur_].refs == 0) slabs_[cur_].used = 0;
    if (cur_ < 0 || slabs_[cur_].used + bytes > slabs_[cur_].size) {
      if (cur_ >= 0 && slabs_[cur_].refs == 0) drop(arena, cur_);
      int64_t size = std::max(slab_, bytes);
      int64_t off = arena.alloc(size);
      if (off < 0 && size > bytes) off = arena.alloc(size = bytes);
      if (off < 0) return -1;
      cur_ = fresh(off, size);  // a previous slab still in use is dropped by its last release
    }
    Slab &sl = slabs_[cur_];
    const int64_t off = sl.off + sl.used;
    sl.used += bytes;
    sl.refs += 1;
    *id = cur_;
    return off;
  }
  void release(ArenaAlloc &arena, int id) {
    if (--slabs_[id].refs == 0 && id != cur_) drop(arena, id);
  }
  // Returns the slab being filled to the arena if no request uses it (an
  // idle slab must not split the space a large request needs).
  bool trim(ArenaAlloc &arena) {
    if (cur_ < 0 || slabs_[cur_].refs != 0) return false;
    drop(arena, cur_);
    return true;
  }

 private:
  struct Slab {
    int64_t off = -1, size = 0, used = 0, refs = 0;
  };
  void drop(ArenaAlloc &arena, int id) {
    arena.release(slabs_[id].off, slabs_[id].size);
    slabs_[id] = Slab{};
    free_ids_.push_back(id);
    if (id == cur_) cur_ = -1;
  }
  int fresh(int64_t off, int64_t size) {
    int id;
    if (!free_ids_.empty()) {
      id = free_ids_.back();
      free_ids_.pop_back();
    } else {
      id = (int)slabs_.size();
      slabs_.emplace_back();
    }
    slabs_[id].off = off;
    slabs_[id].size = size;
    return id;
  }
  int64_t slab_;
  int cur_ = -1;
  std::vector<Slab> slabs_;
  std::vector<int> free_ids_;
};

}  // namespace ga

// First-fit allocator of the batch runtime (fpg_batch_*) over the one device pool
// the caller passes in.  It hands out offsets only and never touches the memory, so
// it is plain host code.
#pragma once

#include <algorithm>
#include <cstddef>
#include <utility>
#include <vector>

namespace fpg {

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Free ranges as (offset, bytes), sorted by offset and coalesced.  Every request is
// rounded up to a multiple of 256 bytes, so offsets stay 256-byte aligned when the
// pool's size is a multiple of 256.
struct PoolFreeList {
  std::vector<std::pair<size_t, size_t>> ranges;

  void reset(size_t bytes) { ranges.assign(1, {0, bytes}); }

  // Carves `bytes` from the first range that holds them; false if none does.
  bool take(size_t bytes, size_t* off) {
    bytes = align256(bytes);
    for (size_t i = 0; i < ranges.size(); ++i) {
      auto& fr = ranges[i];
      if (fr.second < bytes) continue;
      *off = fr.first;
      fr.first += bytes;
      fr.second -= bytes;
      if (fr.second == 0) ranges.erase(ranges.begin() + i);
      return true;
    }
    return false;
  }

  // Returns a range that `take` handed out (the same `bytes`), merging it with the
  // free ranges on either side.
  void give(size_t off, size_t bytes) {
    bytes = align256(bytes);
    auto it = std::lower_bound(ranges.begin(), ranges.end(), std::make_pair(off, (size_t)0));
    it = ranges.insert(it, {off, bytes});
    size_t i = it - ranges.begin();
    if (i + 1 < ranges.size() && ranges[i].first + ranges[i].second == ranges[i + 1].first) {
      ranges[i].second += ranges[i + 1].second;
      ranges.erase(ranges.begin() + i + 1);
    }
    if (i > 0 && ranges[i - 1].first + ranges[i - 1].second == ranges[i].first) {
      ranges[i - 1].second += ranges[i].second;
      ranges.erase(ranges.begin() + i);
    }
  }
};

}  // namespace fpg

// Host-side merges of a rotation-sharded registration (Algorithm 2 treats
// every rotation on its own, so shards of the grid meet only where the
// algorithm reduces over all rotations):
//   - the best inlier count M* over all rotations, which the q filter
//     (1000 M >= q_milli M*) compares against;
//   - the K smallest (key, rotation) pairs over all rotations, for top-K
//     selection by (M desc, index asc) and for the K best candidates by
//     (cost, index) that the second pass centres its Euler boxes on.
// Keys carry a 32-bit rotation index in their low bits; a shard works with
// local slots (its first-pass range, then its second-pass range) and the
// merges work with the whole registration's indices, so ties break as in the
// unsharded run. Plain C++ with no CUDA dependency, tested on a CPU.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <vector>

namespace dses {

constexpr uint64_t kPadKey = ~0ull;

// Where a shard's local rotation slots sit in the whole registration: local
// slots [0, n1) are first-pass rotations [b1, b1 + n1) of the n1_total grid;
// local slots [n1, n1 + n2) are second-pass rotations [b2, b2 + n2), whose
// global indices follow the grid's (n1_total + b2 + ...).
struct ShardMap {
  int64_t b1 = 0, n1 = 0, n1_total = 0, b2 = 0, n2 = 0;

  uint32_t to_global(uint32_t local) const {
    return (int64_t)local < n1 ? (uint32_t)(b1 + local) : (uint32_t)(n1_total + b2 + ((int64_t)local - n1));
  }
  // false when the global index belongs to another shard
  bool to_local(uint32_t global, uint32_t* local) const {
    const int64_t g = global;
    if (g >= b1 && g < b1 + n1) {
      *local = (uint32_t)(g - b1);
      return true;
    }
    const int64_t f = g - n1_total - b2;
    if (g >= n1_total && f >= 0 && f < n2) {
      *local = (uint32_t)(n1 + f);
      return true;
    }
    return false;
  }
};

inline uint64_t key_to_global(uint64_t key, const ShardMap& m) {
  if (key == kPadKey) return key;
  return (key & 0xffffffff00000000ull) | m.to_global((uint32_t)(key & 0xffffffffull));
}

// Largest of the shards' values.
inline uint32_t merge_max(const uint32_t* v, int world) {
  uint32_t m = 0;
  for (int r = 0; r < world; ++r) m = std::max(m, v[r]);
  return m;
}

// The k smallest of `world` lists of k keys each (padding kPadKey anywhere),
// ascending, padded with kPadKey to k entries.
inline std::vector<uint64_t> merge_k_smallest(const uint64_t* lists, int world, int k) {
  std::vector<uint64_t> all;
  all.reserve((size_t)world * k);
  for (int64_t i = 0; i < (int64_t)world * k; ++i)
    if (lists[i] != kPadKey) all.push_back(lists[i]);
  std::sort(all.begin(), all.end());
  all.resize((size_t)k, kPadKey);
  return all;
}

}  // namespace dses

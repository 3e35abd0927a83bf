// Host-side merges of a rotation-sharded registration (csrc/exchange.h): the
// k smallest keys merged from per-shard lists equal the k smallest of all
// keys; local slots and global rotation indices map back and forth; M* is the
// largest shard value.
#include <algorithm>
#include <cstdio>
#include <random>
#include <vector>

#include "exchange.h"

#define EXPECT(c)                                         \
  do {                                                    \
    if (!(c)) {                                           \
      std::printf("FAILED line %d: %s\n", __LINE__, #c);  \
      return 1;                                           \
    }                                                     \
  } while (0)

using dses::kPadKey;

int main() {
  std::mt19937_64 rng(7);
  // shard maps over a grid of n1 rotations and a second pass of n2, world w
  for (int w : {1, 2, 3, 8}) {
    const int64_t n1 = 1000, n2 = 343 * 4;
    std::vector<int> owner(n1 + n2, -1);
    for (int r = 0; r < w; ++r) {
      dses::ShardMap m;
      m.b1 = n1 * r / w;
      m.n1 = n1 * (r + 1) / w - m.b1;
      m.n1_total = n1;
      m.b2 = n2 * r / w;
      m.n2 = n2 * (r + 1) / w - m.b2;
      for (uint32_t l = 0; l < (uint32_t)(m.n1 + m.n2); ++l) {
        const uint32_t g = m.to_global(l);
        EXPECT(g < (uint32_t)(n1 + n2));
        EXPECT(owner[g] == -1);  // every global rotation belongs to one shard
        owner[g] = r;
        uint32_t back = 0;
        EXPECT(m.to_local(g, &back) && back == l);
        // first-pass slots stay below the grid size, second-pass ones above it
        EXPECT((l < m.n1) == (g < n1));
      }
      EXPECT(dses::key_to_global(kPadKey, m) == kPadKey);
      const uint64_t key = (123ull << 32) | 0u;
      EXPECT(dses::key_to_global(key, m) == ((123ull << 32) | (uint64_t)m.to_global(0)));
    }
    for (int64_t g = 0; g < n1 + n2; ++g) EXPECT(owner[g] >= 0);
    // a shard maps exactly its own rotations
    for (int r = 0; r < w; ++r) {
      dses::ShardMap m;
      m.b1 = n1 * r / w;
      m.n1 = n1 * (r + 1) / w - m.b1;
      m.n1_total = n1;
      m.b2 = n2 * r / w;
      m.n2 = n2 * (r + 1) / w - m.b2;
      for (uint32_t g = 0; g < (uint32_t)(n1 + n2); ++g) {
        uint32_t l = 0;
        EXPECT(m.to_local(g, &l) == (owner[g] == r));
      }
    }
  }
  // k smallest: per-shard sorted k-lists (padded) merge to the global k smallest
  for (int trial = 0; trial < 200; ++trial) {
    const int w = 1 + (int)(rng() % 6), k = 1 + (int)(rng() % 40);
    std::vector<uint64_t> all, lists((size_t)w * k, kPadKey);
    for (int r = 0; r < w; ++r) {
      const int n = (int)(rng() % 60);  // may be fewer than k (padding), or none
      std::vector<uint64_t> mine;
      for (int i = 0; i < n; ++i) {
        // distinct keys: the low 32 bits are a unique rotation index
        const uint64_t key = ((rng() % 50) << 32) | (uint64_t)(r * 1000 + i);
        mine.push_back(key);
        all.push_back(key);
      }
      std::sort(mine.begin(), mine.end());
      for (int i = 0; i < std::min(n, k); ++i) lists[(size_t)r * k + i] = mine[(size_t)i];
    }
    std::sort(all.begin(), all.end());
    const std::vector<uint64_t> got = dses::merge_k_smallest(lists.data(), w, k);
    EXPECT((int)got.size() == k);
    for (int i = 0; i < k; ++i) EXPECT(got[(size_t)i] == (i < (int)all.size() ? all[(size_t)i] : kPadKey));
  }
  const uint32_t v[4] = {3, 17, 0, 9};
  EXPECT(dses::merge_max(v, 4) == 17 && dses::merge_max(v, 1) == 3);
  std::printf("ok\n");
  return 0;
}

// Host-side bound on the vote histogram's counters (no CUDA). For one source
// point the pairs voting into one lattice bin are the targets in one
// half-open cube of side delta_t (the bin's cell moved by R x_i). So the
// largest number of targets in any such cube, times the number of source
// points N, bounds every counter of the vote; the planner takes 16-bit
// counters only when that product fits.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <unordered_map>
#include <vector>

namespace dses {

// Largest number of the m points xyz (FP32, m x 3) in any 2 x 2 x 2 block of
// cells of side delta * 1.001 anchored at lo. Every half-open cube of side
// delta lies in one such block (an interval no longer than a cell meets at
// most two cells), with 0.1% to spare for the FP32 rounding of the vote's
// lattice coordinates, so the result bounds the points in any cube of side
// delta.
inline int points_in_cube_bound(const float* xyz, int64_t m, const float* lo, float delta) {
  const double cs = (double)delta * 1.001;
  std::unordered_map<uint64_t, int> cnt;
  cnt.reserve((size_t)m * 2);
  auto key = [](int64_t a, int64_t b, int64_t c) {
    return ((uint64_t)(a + (1 << 20)) << 42) | ((uint64_t)(b + (1 << 20)) << 21) | (uint64_t)(c + (1 << 20));
  };
  std::vector<int64_t> cell((size_t)m * 3);
  for (int64_t j = 0; j < m; ++j) {
    for (int a = 0; a < 3; ++a) cell[3 * j + a] = (int64_t)std::floor((xyz[3 * j + a] - lo[a]) / cs);
    cnt[key(cell[3 * j], cell[3 * j + 1], cell[3 * j + 2])]++;
  }
  int best = 0;
  // every non-empty block contains some point's cell: the 8 blocks holding it
  for (int64_t j = 0; j < m; ++j)
    for (int dx = 0; dx < 2; ++dx)
      for (int dy = 0; dy < 2; ++dy)
        for (int dz = 0; dz < 2; ++dz) {
          const int64_t bx = cell[3 * j] - dx, by = cell[3 * j + 1] - dy, bz = cell[3 * j + 2] - dz;
          int s = 0;
          for (int ex = 0; ex < 2; ++ex)
            for (int ey = 0; ey < 2; ++ey)
              for (int ez = 0; ez < 2; ++ez) {
                auto f = cnt.find(key(bx + ex, by + ey, bz + ez));
                if (f != cnt.end()) s += f->second;
              }
          best = std::max(best, s);
        }
  return best;
}

}  // namespace dses

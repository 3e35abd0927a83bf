// Row and plane strides of the 32-bit vote histogram (host-side planning; no
// CUDA). The layout stores bin (kx, ky, kz) at word kx hs0 + ky hs1 + kz with
// hs1 >= E_z and hs0 >= E_y hs1, so padding between rows and planes may be
// chosen freely: padding words are never voted and read as zero by the mode
// scan. A warp's increments come from a compact patch of targets, so the bins
// of one `red.shared` are near each other in the lattice; with the compact
// strides of an odd box (E_z and E_y E_z both odd) offsets such as (0, 1, -1)
// land 32 words apart, in the same bank. Padding spreads a neighbourhood over
// the 32 banks.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <utility>

namespace dses {

// Shared-memory bytes of a histogram slab of sx x-planes at plane stride hs0
// (16-bit counters: two per word), rounded up to 16 bytes.
inline int layout_bytes(int64_t sx, int64_t hs0, bool u16) {
  const int64_t bins = sx * hs0;
  const int64_t hb = u16 ? ((bins + 1) / 2) * 4 : bins * 4;
  return (int)((hb + 15) & ~15LL);
}

// How well strides (hs0, hs1) spread a lattice neighbourhood over the 32
// banks (32-bit counters): two bins whose word indices differ by a non-zero
// multiple of 32 share a bank. Returns the squared length of the shortest
// offset with |d|_inf <= 4 that lands in the same bank (larger is better) and,
// second, how many offsets of squared length <= 9 do (fewer is better).
inline std::pair<int, int> bank_spread(int64_t hs0, int64_t hs1) {
  int shortest = 1 << 30, close = 0;
  for (int dx = -4; dx <= 4; ++dx)
    for (int dy = -4; dy <= 4; ++dy)
      for (int dz = -4; dz <= 4; ++dz) {
        const int n2 = dx * dx + dy * dy + dz * dz;
        if (n2 == 0 || (dx * hs0 + dy * hs1 + dz) % 32 != 0) continue;
        shortest = std::min(shortest, n2);
        close += n2 <= 9 ? 1 : 0;
      }
  return {shortest, close};
}

// The strides (hs0, hs1) of a 32-bit slab of sx planes of Ey x Ez bins whose
// layout takes at most limit bytes: among hs1 in [Ez, Ez + 8) and hs0 in
// [Ey hs1, Ey hs1 + 32), the best bank_spread score (ties: fewer bytes); the
// compact strides (Ey Ez, Ez) unless a candidate scores better.
inline std::pair<int64_t, int64_t> pick_strides(int64_t Ey, int64_t Ez, int64_t sx, int64_t limit) {
  std::pair<int64_t, int64_t> pick{Ey * Ez, Ez};
  auto best = bank_spread(pick.first, pick.second);
  int bbytes = layout_bytes(sx, pick.first, false);
  for (int64_t hs1 = Ez; hs1 < Ez + 8; ++hs1)
    for (int64_t hs0 = Ey * hs1; hs0 < Ey * hs1 + 32; ++hs0) {
      const int bytes = layout_bytes(sx, hs0, false);
      if (bytes > limit) continue;
      const auto sc = bank_spread(hs0, hs1);
      if (sc.first > best.first || (sc.first == best.first && sc.second < best.second) ||
          (sc == best && bytes < bbytes)) {
        best = sc;
        pick = {hs0, hs1};
        bbytes = bytes;
      }
    }
  return pick;
}

}  // namespace dses

// Host test of the vote histogram's stride choice (strides.h): the layout
// stays one-to-one and inside its slab, keeps to the byte limit, never scores
// worse than the compact strides, and on the robot-like 33^3 box moves the
// same-bank offsets away from the unit lattice neighbours.
#include <cstdio>
#include <cstdlib>
#include <set>

#include "strides.h"

using namespace dses;

static int fails = 0;
#define CHECK(c)                                           \
  do {                                                     \
    if (!(c)) {                                            \
      std::printf("FAIL line %d: %s\n", __LINE__, #c);     \
      ++fails;                                             \
    }                                                      \
  } while (0)

// same bank (32-bit words) for the lattice offset d under strides (hs0, hs1)
static bool same_bank(int64_t hs0, int64_t hs1, int dx, int dy, int dz) {
  return (dx * hs0 + dy * hs1 + dz) % 32 == 0;
}

int main() {
  // compact 33^3: (0, 1, -1) and (1, 0, -1) are 32 and 1088 words apart
  CHECK(same_bank(33 * 33, 33, 0, 1, -1));
  CHECK(same_bank(33 * 33, 33, 1, 0, -1));
  CHECK(bank_spread(33 * 33, 33).first == 2);

  // robot-like box: 33 planes of 33 x 33, a limit 6 KB above compact
  const int compact = layout_bytes(33, 33 * 33, false);
  const auto p = pick_strides(33, 33, 33, compact + 6144);
  CHECK(p.second >= 33 && p.first >= 33 * p.second);
  CHECK(layout_bytes(33, p.first, false) <= compact + 6144);
  CHECK(bank_spread(p.first, p.second).first >= 5);
  // no offset of length <= sqrt(2) shares a bank any more
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dz = -1; dz <= 1; ++dz)
        if ((dx || dy || dz) && dx * dx + dy * dy + dz * dz <= 2) CHECK(!same_bank(p.first, p.second, dx, dy, dz));

  // no room: the compact strides
  const auto q = pick_strides(33, 33, 33, compact);
  CHECK(q.first == 33 * 33 && q.second == 33);

  // odd extents 1..15, slabs of 1..7 planes, limits from compact to +4 KB:
  // one-to-one, inside the slab, within the limit, never worse than compact
  for (int Ey = 1; Ey <= 15; Ey += 2)
    for (int Ez = 1; Ez <= 15; Ez += 2)
      for (int sx = 1; sx <= 7; sx += 3)
        for (int extra = 0; extra <= 4096; extra += 1024) {
          const int lim = layout_bytes(sx, (int64_t)Ey * Ez, false) + extra;
          const auto s = pick_strides(Ey, Ez, sx, lim);
          CHECK(s.second >= Ez && s.first >= (int64_t)Ey * s.second);
          CHECK(layout_bytes(sx, s.first, false) <= lim);
          const auto a = bank_spread(s.first, s.second), b = bank_spread((int64_t)Ey * Ez, Ez);
          CHECK(a.first > b.first || (a.first == b.first && a.second <= b.second));
          std::set<int64_t> bins;
          for (int kx = 0; kx < sx; ++kx)
            for (int ky = 0; ky < Ey; ++ky)
              for (int kz = 0; kz < Ez; ++kz) {
                const int64_t bin = kx * s.first + ky * s.second + kz;
                CHECK(bin < sx * s.first);
                bins.insert(bin);
              }
          CHECK((int64_t)bins.size() == (int64_t)sx * Ey * Ez);
        }
  if (fails) return 1;
  std::printf("ok\n");
  return 0;
}

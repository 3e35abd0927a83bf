// Host test of the 16-bit counter bound (bounds.h): on random, clustered and
// cell-edge point sets, points_in_cube_bound is at least the largest number
// of points in any half-open cube of side delta (found by brute force over
// the cubes whose lower faces touch points, where the maximum is attained),
// and at most the number of points.
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "bounds.h"

using namespace dses;

static int fails = 0;

// most points in any cube [c, c + delta)^3: some maximal cube has each lower
// face on a point's coordinate (slide it up until a face meets a point)
static int brute_max(const std::vector<float>& p, float delta) {
  const int m = (int)p.size() / 3;
  int best = 0;
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b)
      for (int c = 0; c < m; ++c) {
        const double cx = p[3 * a], cy = p[3 * b + 1], cz = p[3 * c + 2];
        int s = 0;
        for (int j = 0; j < m; ++j)
          s += p[3 * j] >= cx && p[3 * j] < cx + delta && p[3 * j + 1] >= cy && p[3 * j + 1] < cy + delta &&
               p[3 * j + 2] >= cz && p[3 * j + 2] < cz + delta;
        best = std::max(best, s);
      }
  return best;
}

static void check(const std::vector<float>& p, float delta, const char* tag) {
  const int m = (int)p.size() / 3;
  float lo[3] = {INFINITY, INFINITY, INFINITY};
  for (int j = 0; j < m; ++j)
    for (int a = 0; a < 3; ++a) lo[a] = std::min(lo[a], p[3 * j + a]);
  const int b = points_in_cube_bound(p.data(), m, lo, delta);
  const int t = brute_max(p, delta);
  if (b < t || b > m) {
    if (fails < 20) std::printf("FAIL %s m %d delta %g: bound %d, brute force %d\n", tag, m, delta, b, t);
    ++fails;
  }
}

int main() {
  std::mt19937 rng(7);
  std::uniform_real_distribution<float> u(-1.f, 1.f);
  for (int trial = 0; trial < 200; ++trial) {
    const int m = 1 + trial % 40;
    const float delta = 0.05f + 0.5f * (float)(trial % 7) / 7.f;
    std::vector<float> p(3 * m);
    // uniform in a box, then a cluster of a third of the points within delta
    for (auto& v : p) v = u(rng);
    for (int j = 0; j < m / 3; ++j)
      for (int a = 0; a < 3; ++a) p[3 * j + a] = 0.3f + 0.9f * delta * (0.5f + 0.5f * u(rng));
    check(p, delta, "random");
  }
  // points on and just below the binning's cell edges (side 1.001 delta)
  for (int trial = 0; trial < 50; ++trial) {
    const float delta = 0.1f;
    const double cs = 1.001 * delta;
    const int m = 27;
    std::vector<float> p(3 * m);
    for (int j = 0; j < m; ++j)
      for (int a = 0; a < 3; ++a) {
        const int k = (j / (a == 0 ? 1 : a == 1 ? 3 : 9)) % 3 + (trial % 3);
        const double e = (trial / 3) % 2 ? -1e-7 : 0.0;
        p[3 * j + a] = (float)(k * cs + e + 0.25 * delta * ((trial / 6) % 3));
      }
    check(p, delta, "edges");
  }
  // all points in one cube of side delta: the bound is m
  {
    std::vector<float> p;
    for (int j = 0; j < 30; ++j)
      for (int a = 0; a < 3; ++a) p.push_back(0.5f + 0.099f * (float)((j * (a + 3)) % 10) / 10.f);
    float lo[3] = {0.5f, 0.5f, 0.5f};
    if (points_in_cube_bound(p.data(), 30, lo, 0.1f) != 30) {
      std::printf("FAIL one cube\n");
      ++fails;
    }
  }
  if (fails) {
    std::printf("%d failures\n", fails);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}

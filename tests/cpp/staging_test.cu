// Host test of the rotation pass's shared-memory plan (kernels.cuh
// pass_staging and set_chunks), built with nvcc and run without a GPU: for
// every histogram size up to the budget and a range of source counts, each
// staging layout the vote kernel may use keeps its chunk's writes inside the
// staging region, the block bounds of a chunk fit their region, and the
// regions stay aligned and within the CTA's shared memory.
#include <cstdio>
#include <vector>

#include "kernels.cuh"

using namespace dses;

static int fails = 0;
#define CHECK(c, h, n, tag)                                                            \
  do {                                                                                 \
    if (!(c)) {                                                                        \
      if (fails < 20) std::printf("FAIL %s hist %d n %d: %s\n", tag, h, n, #c);       \
      ++fails;                                                                         \
    }                                                                                  \
  } while (0)

// one past the last staging byte a chunk of c sources writes in each layout
static long long plain_end(int c) { return 16LL * c; }   // float4 (cx, cy, cz, 0)
static long long packed_end(int c) { return 32LL * c; }  // (cx, cx, cy, cy), (cz, cz, 0, 0)
static long long tiled_end(int c) {                      // 8 per 192-byte tile
  const int i = c - 1;                                   // the last source: its z pair
  return (long long)(i / kTileSources) * kTileBytes + 128 + 8 * (i % kTileSources) + 8;
}

static void check(int h, int n, bool culled, bool paired) {
  int src = -1, blk = -1, list = -1;
  pass_staging(h, n, culled, paired, &src, &blk, &list);
  const char* tag = paired ? "paired" : (culled ? "culled" : "dense");
  CHECK(src > 0 && src % 32 == 0, h, n, tag);
  CHECK(blk >= 0 && blk % 32 == 0 && (culled || blk == 0), h, n, tag);
  CHECK(list == (paired ? kPairedListBytes : 0), h, n, tag);
  CHECK((long long)h + src + blk + list <= kMaxSmem - kPassStaticSmem, h, n, tag);
  PassDesc d{};
  d.N = n;
  set_chunks(d, src);
  for (int k = 0; k < 3; ++k) CHECK(d.chunk[k] >= 1 && d.chunk[k] <= n, h, n, tag);
  if (paired) {
    // the paired instances stage tiles; their block bounds cover a tiled chunk
    CHECK(tiled_end(d.chunk[2]) <= src, h, n, tag);
    CHECK(32LL * ((d.chunk[2] + 31) / 32) <= blk, h, n, tag);
  } else if (culled) {
    // the 32-point culled path stages plain float4s
    CHECK(plain_end(d.chunk[0]) <= src, h, n, tag);
    CHECK(32LL * ((d.chunk[0] + 31) / 32) <= blk, h, n, tag);
  } else {
    CHECK(plain_end(d.chunk[0]) <= src, h, n, tag);
    CHECK(packed_end(d.chunk[1]) <= src, h, n, tag);
  }
}

int main() {
  std::vector<int> hs;
  for (int h = 16; h <= kHistBudget; h += 1616) hs.push_back(h);
  hs.push_back(kHistBudget & ~15);
  hs.push_back(148768);  // a 33-plane slab at plane stride 1127 (32-bit)
  std::vector<int> ns;
  for (int n = 1; n <= 80; ++n) ns.push_back(n);
  for (int n : {255, 256, 257, 1000, 2047, 2048, 2049, 5000, 20000, 1 << 20, 1 << 24}) ns.push_back(n);
  for (int h : hs)
    for (int n : ns) {
      check(h, n, false, false);
      check(h, n, true, false);
      check(h, n, true, true);
    }
  if (fails) {
    std::printf("%d failures\n", fails);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}

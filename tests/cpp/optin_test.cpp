// Host-side check of the vote kernel's per-device shared-memory opt-in
// bookkeeping (csrc/optin.h): a size set on one device says nothing about
// another; the recorded size only grows; concurrent threads agree.
#include <cstdio>
#include <thread>
#include <vector>

#include "optin.h"

#define EXPECT(c)                                              \
  do {                                                         \
    if (!(c)) {                                                \
      std::printf("FAILED line %d: %s\n", __LINE__, #c);       \
      return 1;                                                \
    }                                                          \
  } while (0)

int main() {
  dses::OptIn o;
  EXPECT(o.needed(0, 200000));
  o.done(0, 200000);
  EXPECT(!o.needed(0, 200000));
  EXPECT(!o.needed(0, 100000));
  EXPECT(o.needed(0, 200001));
  // device 1 never configured: the first launch there must set the attribute
  EXPECT(o.needed(1, 1));
  EXPECT(o.needed(1, 100000));
  o.done(1, 50000);
  EXPECT(!o.needed(1, 50000) && o.needed(1, 50001));
  // a smaller size recorded later does not lower the limit
  o.done(0, 1000);
  EXPECT(!o.needed(0, 200000));
  // out-of-range devices are never cached
  EXPECT(o.needed(-1, 1) && o.needed(dses::kOptInDevices, 1));
  o.done(dses::kOptInDevices, 10);
  EXPECT(o.needed(dses::kOptInDevices, 1));
  // many threads on several devices: each device ends at its largest size
  dses::OptIn p;
  std::vector<std::thread> th;
  for (int t = 0; t < 16; ++t)
    th.emplace_back([&p, t] {
      for (int i = 0; i < 20000; ++i) {
        const int dev = (t + i) % 4, want = 1000 + (i * 7919 + t) % 100000;
        if (p.needed(dev, want)) p.done(dev, want);
      }
    });
  for (auto& x : th) x.join();
  for (int dev = 0; dev < 4; ++dev) {
    int mx = 0;
    for (int t = 0; t < 16; ++t)
      for (int i = 0; i < 20000; ++i)
        if ((t + i) % 4 == dev) mx = std::max(mx, 1000 + (i * 7919 + t) % 100000);
    EXPECT(!p.needed(dev, mx) && p.needed(dev, mx + 1));
  }
  EXPECT(p.needed(4, 1));
  std::printf("ok\n");
  return 0;
}

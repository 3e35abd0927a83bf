// Per-device bookkeeping of a kernel's dynamic shared-memory opt-in.
//
// cudaFuncSetAttribute(..., cudaFuncAttributeMaxDynamicSharedMemorySize, n)
// applies to the current device only, so a process that launches one kernel
// on several GPUs must raise the limit once per device. OptIn keeps, per
// device, the largest size set so far; it is lock-free and may be used from
// several host threads (two threads that race both set the attribute, which
// is harmless, and the recorded size only grows). Host-only code with no CUDA
// dependency, so its logic is tested on a CPU.
#pragma once

#include <atomic>

namespace dses {

constexpr int kOptInDevices = 64;

struct OptIn {
  std::atomic<int> bytes[kOptInDevices];

  OptIn() {
    for (auto& b : bytes) b.store(0, std::memory_order_relaxed);
  }
  // true when `want` bytes exceed what was recorded for `device` (the caller
  // then sets the attribute on that device and calls done()); devices outside
  // [0, kOptInDevices) are never cached, so they always need the call
  bool needed(int device, int want) const {
    if (device < 0 || device >= kOptInDevices) return true;
    return bytes[device].load(std::memory_order_acquire) < want;
  }
  // records a successful cudaFuncSetAttribute of `set` bytes on `device`
  void done(int device, int set) {
    if (device < 0 || device >= kOptInDevices) return;
    int cur = bytes[device].load(std::memory_order_relaxed);
    while (cur < set && !bytes[device].compare_exchange_weak(cur, set, std::memory_order_acq_rel)) {
    }
  }
};

}  // namespace dses

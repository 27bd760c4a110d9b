// Host-side, per-device one-time setup of the kernel launchers.  CUDA keeps
// kernel attributes (such as the dynamic shared-memory limit) per device, and
// grid sizes follow the device's multiprocessor count, so a process that
// launches on several devices sets and queries them once for each device.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

namespace claire {

constexpr int kSetupDevices = 64;

inline int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  return dev;
}

// fn() once for each device it is called on (on every call for device ordinals
// beyond the table).
template <typename F>
inline void once_per_device(std::once_flag (&flags)[kSetupDevices], F&& fn) {
  const int dev = current_device();
  if (dev < 0 || dev >= kSetupDevices) {
    fn();
    return;
  }
  std::call_once(flags[dev], fn);
}

// Multiprocessor count of the current device (cached per device), 0 if the
// query fails.
inline int device_sm_count() {
  static std::atomic<int> cache[kSetupDevices];
  const int dev = current_device();
  const bool slot = dev >= 0 && dev < kSetupDevices;
  int n = slot ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    return 0;
  if (slot) cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

}  // namespace claire

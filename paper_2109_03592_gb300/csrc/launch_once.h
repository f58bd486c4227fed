// Per-device, thread-safe one-time launch set-up.
//
// Kernel attributes (cudaFuncSetAttribute) and occupancy-derived grid sizes
// belong to a device, and server threads may issue their first launch of a
// kernel at the same time.  Each launcher keeps one DeviceOnce per kernel
// instantiation: the set-up runs once per device under a mutex, and later
// launches on that device read the cached value.
#pragma once

#include <cuda_runtime.h>

#include <mutex>

namespace sem {

struct DeviceOnce {
  static constexpr int kMaxDevices = 64;
  std::mutex mu;
  int value[kMaxDevices] = {};
  bool done[kMaxDevices] = {};

  // setup(device, &value) runs once per device; *out receives the value.
  template <typename F>
  cudaError_t get(F&& setup, int* out = nullptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
      int v = 0;
      e = setup(dev, &v);
      if (e != cudaSuccess) return e;
      value[dev] = v;
      done[dev] = true;
    }
    if (out) *out = value[dev];
    return cudaSuccess;
  }
};

}  // namespace sem

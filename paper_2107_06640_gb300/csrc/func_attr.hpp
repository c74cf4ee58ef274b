// Per-device kernel attributes.  cudaFuncSetAttribute (e.g. the dynamic
// shared-memory limit) is a setting of the current device, so a kernel that
// needs it is configured once on every device that launches it.
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <set>
#include <utility>

namespace adg {

// Run configure() for `kernel` on the current device unless that already
// succeeded there; returns a cudaError_t as int.
template <class F>
int configure_on_device(const void* kernel, F&& configure) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = -1;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return (int)ce;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({kernel, dev})) return 0;
  ce = configure();
  if (ce == cudaSuccess) done.insert({kernel, dev});
  return (int)ce;
}

}  // namespace adg

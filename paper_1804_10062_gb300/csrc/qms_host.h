// Host-side helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>
#include <set>
#include <utility>

namespace qms {

// Raises the dynamic shared-memory limit of kernel f to `bytes` on the
// current device.  The attribute belongs to the device that is current when
// it is set, so it is set once per (kernel, device), under a lock (several
// host threads may launch at once).
inline cudaError_t smem_attr(const void* f, size_t bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({f, dev})) return cudaSuccess;
  e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  if (e == cudaSuccess) done.insert({f, dev});
  return e;
}

}  // namespace qms

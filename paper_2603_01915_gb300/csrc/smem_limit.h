// Raising a kernel's dynamic shared-memory limit once per device.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

namespace dtans {

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) applies to the current
// device's context only, so each launcher keeps one bit per device ordinal
// (`done`, one per kernel instance) and sets the attribute the first time it
// launches on that device.  Ordinals of 64 and above are not cached: the
// attribute is set on every call there.
template <typename F>
inline cudaError_t ensure_smem_limit(F *kern, int bytes, std::atomic<uint64_t> &done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = (dev >= 0 && dev < 64) ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
  return e;
}

}  // namespace dtans

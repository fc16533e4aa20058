// launch_util.h -- grid sizing of the persistent task kernels.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>
#include <utility>

namespace chol {

// CTAs of `kernel` that fit on the device at once (SMs x resident CTAs per SM), cached per
// (kernel, block size, dynamic shared memory); at least one.
inline int resident_ctas(const void* kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::unordered_map<const void*, std::unordered_map<size_t, int>> cache;
  static int sms = 0;
  std::lock_guard<std::mutex> lock(mu);
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
      cudaGetLastError();
      sms = 1;
    }
  }
  const size_t key = smem * 4096 + (size_t)threads;
  auto& m = cache[kernel];
  auto it = m.find(key);
  if (it != m.end()) return it->second;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
      per_sm <= 0) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int r = per_sm * sms;
  m[key] = r;
  return r;
}

// Grid of a task launch.  Every CTA takes tasks from the launch's work queue until it is
// empty.  Measured on GB300, a grid of one CTA per task (the hardware block scheduler then
// refills SMs as CTAs finish) balances the uneven task costs of a level better than a
// single resident wave, so the grid is the task count, never less than one resident wave
// would need; the queue makes any grid size correct.
template <typename K>
inline int persistent_grid(K kernel, int threads, size_t smem, int ntasks) {
  (void)kernel;
  (void)threads;
  (void)smem;
  return ntasks;
}

}  // namespace chol

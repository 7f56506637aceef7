// launch.cuh -- small host helpers shared by the launchers.
#pragma once
#include "kernels.h"

namespace mmp {

static inline int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

template <typename K>
static inline cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace mmp

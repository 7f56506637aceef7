// peak.cu -- measured FP32 FMA throughput of the device (the ALU ceiling
// the passes' arithmetic rate is compared with).  Eight independent FMA
// chains per thread, full occupancy, no memory traffic inside the loop.
#include <cuda_runtime.h>

#include "mmp.h"

namespace mmp {
int report_error(int code, const char* msg);
}

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) k_fma_peak(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1e-3f * (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int mmp_fp32_peak(void* stream, int reps, double* gflops, double* ms_per_launch) {
  if (!gflops || reps < 1) return mmp::report_error(MMP_E_INVAL, "mmp_fp32_peak: bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return mmp::report_error(MMP_E_CUDA, "mmp_fp32_peak: no device");
  }
  const int threads = 256, blocks = sms * 8, iters = 4096;
  float* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return mmp::report_error(MMP_E_OOM, "mmp_fp32_peak: allocation failed");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  k_fma_peak<<<blocks, threads, 0, s>>>(out, iters, 0.999999f, 1e-7f);   // warm-up
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, s);
    k_fma_peak<<<blocks, threads, 0, s>>>(out, iters, 0.999999f, 1e-7f);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return mmp::report_error(MMP_E_CUDA, cudaGetErrorString(err));
  const double flops = 2.0 * kChains * kUnroll * (double)iters * blocks * threads;
  *gflops = flops / (best * 1e-3) / 1e9;
  if (ms_per_launch) *ms_per_launch = best;
  return MMP_OK;
}

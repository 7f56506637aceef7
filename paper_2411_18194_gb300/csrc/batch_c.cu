// batch_c.cu -- batched pass C (inverse x FFT + local field + LLG torque
// + error estimate): one block per (member, tile) item; and the accept
// kernel of fixed-step graphs.
#include "batch.h"
#include "field.cuh"
#include "launch.cuh"

namespace mmp {

__global__ void __launch_bounds__(kBatchThreads) k_batch_field(const BatchInst* __restrict__ insts,
                                                               const BatchItem* __restrict__ items, int stage) {
  extern __shared__ __align__(16) float smem[];
  __shared__ BatchInst si;
  __shared__ StageArgs sa;
  __shared__ FieldArgs fa;
  const BatchItem w = batch_item(insts, items, si);
  if (threadIdx.x == 0) batch_args(si, stage, sa, fa);
  __syncthreads();
  field_tile<1, true, true>(smem, si.g, si.d, si.co, fa, w.b, w.a * si.g.tyc);
}

// Accept the step of every member (fixed-step graphs): flip the ping-pong.
__global__ void k_batch_accept(BatchInst* insts, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) insts[i].par ^= 1;
}

cudaError_t launch_batch_field(const BatchInst* insts, const BatchItem* items, int nitems, int stage, int threads,
                               size_t smem, cudaStream_t s) {
  cudaError_t e = set_smem(k_batch_field, smem);
  if (e != cudaSuccess) return e;
  k_batch_field<<<nitems, threads, smem, s>>>(insts, items, stage);
  return cudaGetLastError();
}

cudaError_t launch_batch_accept(BatchInst* insts, int n, cudaStream_t s) {
  k_batch_accept<<<(n + 127) / 128, 128, 0, s>>>(insts, n);
  return cudaGetLastError();
}

}  // namespace mmp

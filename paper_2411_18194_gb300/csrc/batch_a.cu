// batch_a.cu -- batched pass A: one block per (member, tile) item.
#include "batch.h"
#include "launch.cuh"
#include "pass_a.cuh"

namespace mmp {

template <bool ASSEMBLE>
__global__ void __launch_bounds__(kBatchThreads, 2) k_batch_passA(const BatchInst* __restrict__ insts,
                                                               const BatchItem* __restrict__ items, int stage) {
  extern __shared__ __align__(16) unsigned char sraw[];
  __shared__ BatchInst si;
  __shared__ StageArgs sa;
  __shared__ FieldArgs fa;
  const BatchItem w = batch_item(insts, items, si);
  if (threadIdx.x == 0) batch_args(si, stage, sa, fa);
  __syncthreads();
  passA_tile<1, ASSEMBLE>(sraw, si.g, sa, si.d, si.co, w.b, w.a * si.g.ty);
}

cudaError_t launch_batch_passA(const BatchInst* insts, const BatchItem* items, int nitems, int stage, int threads,
                               size_t smem, cudaStream_t s) {
  cudaError_t e;
  if (stage == 0) {
    if ((e = set_smem(k_batch_passA<false>, smem)) != cudaSuccess) return e;
    k_batch_passA<false><<<nitems, threads, smem, s>>>(insts, items, stage);
  } else {
    if ((e = set_smem(k_batch_passA<true>, smem)) != cudaSuccess) return e;
    k_batch_passA<true><<<nitems, threads, smem, s>>>(insts, items, stage);
  }
  return cudaGetLastError();
}

}  // namespace mmp

// batch_b.cu -- batched pass B: one block per (member, kx plane) item, one
// CTA per plane (R = 1, kernel rows read from L2); one kernel per z-extent
// group like the per-context path (nz = 1, 2, 4, 8, other).
#include "batch.h"
#include "launch.cuh"
#include "pass_b.cuh"

namespace mmp {

template <int NZ>
__global__ void __launch_bounds__(kBatchThreads) k_batch_passB(const BatchInst* __restrict__ insts,
                                                               const BatchItem* __restrict__ items) {
  extern __shared__ __align__(16) unsigned char sraw[];
  __shared__ BatchInst si;
  const BatchItem w = batch_item(insts, items, si);
  passB_plane<NZ, false>(sraw, si.g, si.d, w.a, 0);
}

template <int NZ>
static cudaError_t launch_b(const BatchInst* insts, const BatchItem* items, int nitems, int threads, size_t smem,
                            cudaStream_t s) {
  cudaError_t e = set_smem(k_batch_passB<NZ>, smem);
  if (e != cudaSuccess) return e;
  k_batch_passB<NZ><<<nitems, threads, smem, s>>>(insts, items);
  return cudaGetLastError();
}

cudaError_t launch_batch_passB(int nz_group, const BatchInst* insts, const BatchItem* items, int nitems,
                               int threads, size_t smem, cudaStream_t s) {
  switch (nz_group) {
    case 1: return launch_b<1>(insts, items, nitems, threads, smem, s);
    case 2: return launch_b<2>(insts, items, nitems, threads, smem, s);
    case 4: return launch_b<4>(insts, items, nitems, threads, smem, s);
    case 8: return launch_b<8>(insts, items, nitems, threads, smem, s);
    default: return launch_b<0>(insts, items, nitems, threads, smem, s);
  }
}

}  // namespace mmp

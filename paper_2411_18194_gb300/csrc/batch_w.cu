// batch_w.cu -- the warp-engine passes for batch members whose shape runs
// them (passes A and C on row-pair tiles at Px = 2048, pass B on warp
// transforms of folded y length 1024): the same tile bodies as the
// per-context kernels (xfft_w.cuh, passb_w.cuh), with the stage and field
// arguments built on the device from the member's descriptor, whose
// ping-pong parity changes inside fixed-step graphs.  One launch per pass
// and such member, beside the work-list launches of the other members.
#include "batch.h"
#include "xfft_w.cuh"
#include "passb_w.cuh"

namespace mmp {

namespace {

// The member's descriptor and its stage/field arguments in shared memory.
__device__ __forceinline__ void batch_member(const BatchInst* insts, int inst, int stage, BatchInst& si,
                                             StageArgs& sa, FieldArgs& fa) {
  const int* src = reinterpret_cast<const int*>(insts + inst);
  int* dst = reinterpret_cast<int*>(&si);
  for (int i = threadIdx.x; i < (int)(sizeof(BatchInst) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  if (threadIdx.x == 0) batch_args(si, stage, sa, fa);
  __syncthreads();
}

template <bool ASSEMBLE>
__global__ void __launch_bounds__(kXwThreads, 4) k_batch_passA_w(const BatchInst* __restrict__ insts, int inst,
                                                                  int stage) {
  extern __shared__ __align__(16) unsigned char sraw[];
  __shared__ BatchInst si;
  __shared__ StageArgs sa;
  __shared__ FieldArgs fa;
  batch_member(insts, inst, stage, si, sa, fa);
  passA_w_tile<1, ASSEMBLE>(sraw, si.g, sa, si.d, si.co, blockIdx.y, 2 * blockIdx.x);
}

__global__ void __launch_bounds__(kXwThreads, 4) k_batch_field_w(const BatchInst* __restrict__ insts, int inst,
                                                                  int stage) {
  extern __shared__ __align__(16) unsigned char sraw[];
  __shared__ BatchInst si;
  __shared__ StageArgs sa;
  __shared__ FieldArgs fa;
  batch_member(insts, inst, stage, si, sa, fa);
  field_w_tile<1, true>(sraw, si.g, si.d, si.co, fa, blockIdx.y, 2 * blockIdx.x);
}

template <int NZ>
__global__ void __launch_bounds__(32 * passb_w_warps(NZ, 32), 1) k_batch_passB_w(const BatchInst* __restrict__ insts,
                                                                                  int inst) {
  extern __shared__ __align__(16) unsigned char sraw[];
  __shared__ BatchInst si;
  __shared__ StageArgs sa;
  __shared__ FieldArgs fa;
  batch_member(insts, inst, 0, si, sa, fa);
  passB_w_plane<NZ, 32, passb_w_warps(NZ, 32), false>(sraw, si.g, si.d, blockIdx.y, (int)(blockIdx.x % si.d.R));
}

template <int NZ>
cudaError_t launch_b(const BatchInst* insts, int inst, const Grid& g, int R, cudaStream_t s) {
  const size_t sm = passb_w_smem(NZ, 32);
  const int threads = 32 * passb_w_warps(NZ, 32);
  if (R == 1) {
    k_batch_passB_w<NZ><<<dim3(1, g.kxn), threads, sm, s>>>(insts, inst);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(R, g.kxn);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = R;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch_passB_w<NZ>, insts, inst);
}

}  // namespace

bool batch_warp_supported(const Grid& g, int R) { return xw_supported(g) && passb_w_supported(g, R) && g.Py / R == 1024; }

// (the attribute is set whatever the size: with the static copy of the
// descriptor a 48 KB dynamic allocation exceeds the default limit)
template <typename K>
cudaError_t smem_attr(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t batch_warp_prepare() {
  cudaError_t e;
  if ((e = smem_attr(k_batch_passA_w<true>, passa_w_smem())) != cudaSuccess) return e;
  if ((e = smem_attr(k_batch_passA_w<false>, passa_w_smem())) != cudaSuccess) return e;
  if ((e = smem_attr(k_batch_field_w, field_w_smem())) != cudaSuccess) return e;
  if ((e = smem_attr(k_batch_passB_w<1>, passb_w_smem(1, 32))) != cudaSuccess) return e;
  if ((e = smem_attr(k_batch_passB_w<2>, passb_w_smem(2, 32))) != cudaSuccess) return e;
  if ((e = smem_attr(k_batch_passB_w<4>, passb_w_smem(4, 32))) != cudaSuccess) return e;
  return smem_attr(k_batch_passB_w<8>, passb_w_smem(8, 32));
}

cudaError_t launch_batch_warp(int kind, const BatchInst* insts, int inst, const Grid& g, int R, int stage,
                              cudaStream_t s) {
  if (kind == 0) {
    const dim3 grid((g.ny + 1) / 2, g.nz);
    if (stage == 0) k_batch_passA_w<false><<<grid, kXwThreads, passa_w_smem(), s>>>(insts, inst, stage);
    else k_batch_passA_w<true><<<grid, kXwThreads, passa_w_smem(), s>>>(insts, inst, stage);
    return cudaGetLastError();
  }
  if (kind == 2) {
    k_batch_field_w<<<dim3((g.ny + 1) / 2, g.nz), kXwThreads, field_w_smem(), s>>>(insts, inst, stage);
    return cudaGetLastError();
  }
  switch (g.nz) {
    case 1: return launch_b<1>(insts, inst, g, R, s);
    case 2: return launch_b<2>(insts, inst, g, R, s);
    case 4: return launch_b<4>(insts, inst, g, R, s);
    case 8: return launch_b<8>(insts, inst, g, R, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mmp

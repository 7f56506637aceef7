// pass_b.cu -- pass B of the demag convolution (body in pass_b.cuh): the
// per-context kernel, launched as clusters of R CTAs per kx plane.
#include <cooperative_groups.h>
#include "kernels.h"
#include "launch.cuh"
#include "stage.cuh"
#include "pass_b.cuh"

namespace mmp {

template <int NZ, bool KS>
__global__ void __launch_bounds__(512) k_passB(Grid g, DemagArgs d) {
  extern __shared__ __align__(16) unsigned char sraw[];
  passB_plane<NZ, KS>(sraw, g, d, blockIdx.y, (int)(blockIdx.x % d.R));
}

size_t smem_passB(const Grid& g, int R, bool ks) { return passb_smem(g.ny, g.nz, g.Py, g.kzn, R, ks).total; }

template <int NZ, bool KS>
static cudaError_t launch_passB_k(const Grid& g, const DemagArgs& d, int threads, cudaStream_t s) {
  size_t sm = smem_passB(g, d.R, KS);
  cudaError_t e = set_smem(k_passB<NZ, KS>, sm);
  if (e != cudaSuccess) return e;
  if (d.R == 1) {
    k_passB<NZ, KS><<<dim3(1, g.kxn), threads, sm, s>>>(g, d);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(d.R, g.kxn);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = d.R;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_passB<NZ, KS>, g, d);
}

template <int NZ>
static cudaError_t launch_passB_t(const Grid& g, const DemagArgs& d, int threads, cudaStream_t s) {
  return d.ks ? launch_passB_k<NZ, true>(g, d, threads, s) : launch_passB_k<NZ, false>(g, d, threads, s);
}

cudaError_t launch_passB(const Grid& g, const DemagArgs& d, int threads, cudaStream_t s) {
  if (d.engine == 1) {
    switch (g.Py / d.R) {
      case 256: return launch_passB_w_len<8>(g, d, s);
      case 512: return launch_passB_w_len<16>(g, d, s);
      case 1024: return launch_passB_w_len<32>(g, d, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (g.nz) {
    case 1: return launch_passB_t<1>(g, d, threads, s);
    case 2: return launch_passB_t<2>(g, d, threads, s);
    case 4: return launch_passB_t<4>(g, d, threads, s);
    case 8: return launch_passB_t<8>(g, d, threads, s);
    default: return launch_passB_t<0>(g, d, threads, s);
  }
}

}  // namespace mmp

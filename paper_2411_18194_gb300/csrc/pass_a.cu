// pass_a.cu -- Dormand-Prince stage assembly and pass A of the demag
// convolution (body in pass_a.cuh): kernels and launchers of the
// per-context path.
#include <cooperative_groups.h>
#include "kernels.h"
#include "launch.cuh"
#include "stage.cuh"
#include "pass_a.cuh"

namespace cg = cooperative_groups;

namespace mmp {

__global__ void k_assemble(Grid g, StageArgs a) {
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < g.n;
       cell += (long long)gridDim.x * blockDim.x)
    assemble_cell(g, a, g.n, cell);
}

__global__ void k_normalize(float* m, long long n) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    float x = m[c], y = m[n + c], z = m[2 * n + c];
    if (x * x + y * y + z * z > 0.0f) {
      float r = rnorm3df(x, y, z);
      m[c] = x * r; m[n + c] = y * r; m[2 * n + c] = z * r;
    }
  }
}

template <int NSUB, bool ASSEMBLE>
__global__ void __launch_bounds__(512, 2) k_passA(Grid g, StageArgs a, DemagArgs d, Coefs co) {
  extern __shared__ __align__(16) unsigned char sraw[];
  passA_tile<NSUB, ASSEMBLE>(sraw, g, a, d, co, blockIdx.y, blockIdx.x * g.ty);
}

size_t smem_passA(const Grid& g) { return passa_inv_offset(g.Px, g.ty, g.xb); }
static size_t smem_passA_launch(const Grid& g, const StageArgs& a) {
  return passa_inv_offset(g.Px, g.ty, g.xb) + (a.normalize ? (size_t)a.nsub * g.ty * g.nx * sizeof(float) : 0);
}

cudaError_t launch_assemble(const Grid& g, const StageArgs& a, cudaStream_t s) {
  k_assemble<<<grid_for(g.n, 256), 256, 0, s>>>(g, a);
  return cudaGetLastError();
}

cudaError_t launch_normalize(float* m, long long n, cudaStream_t s) {
  k_normalize<<<grid_for(n, 256), 256, 0, s>>>(m, n);
  return cudaGetLastError();
}

cudaError_t launch_passA(const Grid& g, const StageArgs& a, const DemagArgs& d, const Coefs& c, int threads,
                         cudaStream_t s) {
  dim3 grid((g.ny + g.ty - 1) / g.ty, g.nz);
  size_t sm = smem_passA_launch(g, a);
  bool assemble = a.stage != nullptr && a.y != nullptr;
  cudaError_t e;
#define MMP_PA(NS, AS)                                                      \
  do {                                                                      \
    if ((e = set_smem(k_passA<NS, AS>, smem_passA(g) + 2 * g.ty * g.nx * sizeof(float))) != cudaSuccess) \
      return e;                                                             \
    k_passA<NS, AS><<<grid, threads, sm, s>>>(g, a, d, c);                 \
  } while (0)
  if (a.nsub == 1) { if (assemble) MMP_PA(1, true); else MMP_PA(1, false); }
  else { if (assemble) MMP_PA(2, true); else MMP_PA(2, false); }
#undef MMP_PA
  return cudaGetLastError();
}

}  // namespace mmp

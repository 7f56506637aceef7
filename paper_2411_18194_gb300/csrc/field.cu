// field.cu -- pass C (body in field.cuh): the per-context kernel and its
// launcher.
#include <cooperative_groups.h>
#include "kernels.h"
#include "launch.cuh"
#include "stage.cuh"
#include "field.cuh"

namespace cg = cooperative_groups;

namespace mmp {

template <int NSUB, bool DEMAG, bool UNI>
__global__ void __launch_bounds__(512) k_field(Grid g, DemagArgs d, Coefs co, FieldArgs f) {
  extern __shared__ float smem[];
  field_tile<NSUB, DEMAG, UNI>(smem, g, d, co, f, blockIdx.y, blockIdx.x * g.tyc);
}

size_t smem_field(const Grid& g, bool demag) {
  if (!demag) return 0;
  return (size_t)((3 * g.tyc * g.nx + 3) & ~3) * sizeof(float) +
         ((size_t)g.xbc * (g.tyc >> 1) * fft_pitch(g.Px) + g.Px) * sizeof(float2);
}

cudaError_t launch_field(const Grid& g, const DemagArgs& d, const Coefs& c, const FieldArgs& f, int nsub,
                         bool demag, int threads, cudaStream_t s) {
  dim3 grid((g.ny + g.tyc - 1) / g.tyc, g.nz);
  size_t sm = smem_field(g, demag);
  cudaError_t e;
#define MMP_F(NS, DM, UN)                                               \
  do {                                                                  \
    if ((e = set_smem(k_field<NS, DM, UN>, sm)) != cudaSuccess) return e; \
    k_field<NS, DM, UN><<<grid, threads, sm, s>>>(g, d, c, f);          \
  } while (0)
  if (nsub == 1) {
    if (demag) { if (c.uniform) MMP_F(1, true, true); else MMP_F(1, true, false); }
    else { if (c.uniform) MMP_F(1, false, true); else MMP_F(1, false, false); }
  } else {
    if (demag) { if (c.uniform) MMP_F(2, true, true); else MMP_F(2, true, false); }
    else { if (c.uniform) MMP_F(2, false, true); else MMP_F(2, false, false); }
  }
#undef MMP_F
  return cudaGetLastError();
}

}  // namespace mmp

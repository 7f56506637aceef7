// passa_w.cu -- pass A on the warp FFT engine (body in xfft_w.cuh): kernel
// instantiations and launcher.
#include "kernels.h"
#include "launch.cuh"
#include "xfft_w.cuh"

namespace mmp {

cudaError_t launch_passA_w(const Grid& g, const StageArgs& a, const DemagArgs& d, const Coefs& c, cudaStream_t s) {
  const dim3 grid((g.ny + 1) / 2, g.nz);
  const size_t sm = passa_w_smem();
  const bool assemble = a.stage != nullptr && a.y != nullptr;
  cudaError_t e;
#define MMP_PAW(NS, AS)                                                \
  do {                                                                 \
    if ((e = set_smem(k_passA_w<NS, AS>, sm)) != cudaSuccess) return e; \
    k_passA_w<NS, AS><<<grid, kXwThreads, sm, s>>>(g, a, d, c);         \
  } while (0)
  if (a.nsub == 1) { if (assemble) MMP_PAW(1, true); else MMP_PAW(1, false); }
  else { if (assemble) MMP_PAW(2, true); else MMP_PAW(2, false); }
#undef MMP_PAW
  return cudaGetLastError();
}

}  // namespace mmp

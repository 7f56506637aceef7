// field_w.cu -- pass C on the warp FFT engine (body in xfft_w.cuh): kernel
// instantiations and launcher.
#include "kernels.h"
#include "launch.cuh"
#include "xfft_w.cuh"

namespace mmp {

cudaError_t launch_field_w(const Grid& g, const DemagArgs& d, const Coefs& c, const FieldArgs& f, int nsub,
                           cudaStream_t s) {
  const dim3 grid((g.ny + 1) / 2, g.nz);
  const size_t sm = field_w_smem();
  cudaError_t e;
#define MMP_FW(NS, UN)                                                 \
  do {                                                                 \
    if ((e = set_smem(k_field_w<NS, UN>, sm)) != cudaSuccess) return e; \
    k_field_w<NS, UN><<<grid, kXwThreads, sm, s>>>(g, d, c, f);         \
  } while (0)
  if (nsub == 1) { if (c.uniform) MMP_FW(1, true); else MMP_FW(1, false); }
  else { if (c.uniform) MMP_FW(2, true); else MMP_FW(2, false); }
#undef MMP_FW
  return cudaGetLastError();
}

}  // namespace mmp

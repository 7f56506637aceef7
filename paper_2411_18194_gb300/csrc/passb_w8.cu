// passb_w8.cu -- the warp pass B kernels of folded y length Ly = 32 * 8
// (body in passb_w.cuh), one translation unit per length so that they
// compile in parallel.
#include "kernels.h"
#include "passb_w.cuh"

namespace mmp {
template <>
cudaError_t launch_passB_w_len<8>(const Grid& g, const DemagArgs& d, cudaStream_t s) {
  return launch_passB_w_m<8>(g, d, s);
}
}  // namespace mmp

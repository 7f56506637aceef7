// stage.cuh -- Dormand-Prince stage assembly of one cell (shared by the
// assembly kernel and pass A).
#pragma once
#include "kernels.h"

namespace mmp {

__device__ __forceinline__ void assemble_cell(const Grid& g, const StageArgs& a, long long n, long long cell) {
  for (int p = 0; p < a.nparts; ++p) {
    float v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      long long idx = (long long)(3 * p + c) * n + cell;
      if (!MMP_IN(g, idx, g.lim_state)) { v[c] = 0.0f; continue; }
      float acc = a.y[idx];
#pragma unroll
      for (int j = 0; j < 7; ++j)
        if (j < a.nk) acc = fmaf(a.coef[j], a.k[j][idx], acc);
      v[c] = acc;
    }
    if (a.normalize && p < a.nsub) {
      float nn = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
      if (nn > 0.0f) {
        float r = rnorm3df(v[0], v[1], v[2]);
        v[0] *= r; v[1] *= r; v[2] *= r;
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long idx = (long long)(3 * p + c) * n + cell;
      if (MMP_IN(g, idx, g.lim_state)) a.stage[idx] = v[c];
    }
  }
}

}  // namespace mmp

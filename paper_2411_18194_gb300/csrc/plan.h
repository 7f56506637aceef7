// plan.h -- host helpers shared by the C-ABI entry points: padded FFT
// lengths, radix plans and FP64-built twiddle tables.
#pragma once
#include <math.h>

#include <algorithm>
#include <vector>

#include "kernels.h"

namespace mmp {

inline int nice_length(int n) {
  // smallest even 2^a or 3*2^a >= 2n - 1 (1 when n == 1)
  if (n == 1) return 1;
  int best = 1 << 30;
  for (int p = 2; p < (1 << 30); p *= 2)
    if (p >= 2 * n - 1) { best = std::min(best, p); break; }
  for (int p = 6; p < (1 << 30); p *= 2)
    if (p >= 2 * n - 1) { best = std::min(best, p); break; }
  return best;
}

inline bool make_plan(int L, FftPlan& p) {
  p.L = L;
  p.n16 = p.n8 = p.n4 = p.n2 = p.n3 = 0;
  int r = L, a = 0;
  while (r % 3 == 0) { r /= 3; p.n3++; }
  while (r % 2 == 0) { r /= 2; a++; }
  if (r != 1) return false;
  p.n16 = a / 4;
  p.n8 = (a % 4) == 3;
  p.n4 = (a % 4) == 2;
  p.n2 = (a % 4) == 1;
  return true;
}

inline std::vector<float2> roots(int P) {
  std::vector<float2> w(P);
  for (int t = 0; t < P; ++t) {
    double a = 2.0 * 3.14159265358979323846 * (double)t / (double)P;
    w[t] = make_float2((float)cos(a), (float)(-sin(a)));
  }
  return w;
}

// Residue classes of ky per pass-B cluster: the smallest power of two (<= 8)
// that keeps a plane of 3 nz columns of Py/R complex values <= ~100 KB.
inline int pick_residues(const Grid& g) {
  int R = 1;
  while (R < 8 && (size_t)3 * g.nz * (g.Py / R) * sizeof(float2) > 100 * 1024 && g.Py % (2 * R) == 0 &&
         g.Py / (2 * R) >= 2)
    R *= 2;
  return R;
}

// Block sizes of passes A, B and C (at most 32 FFT elements per thread).
inline void launch_threads(const Grid& g, int R, int* thrA, int* thrB, int* thrC) {
  auto r32 = [](long long v) { return (int)((v + 31) / 32 * 32); };
  *thrA = std::min(512, std::max(128, r32((long long)MMP_NP * g.Px / 32)));
  long long elB = (long long)3 * g.nz * (g.Py / R);
  *thrB = std::min(512, std::max(64, r32(std::max(elB / 32, (long long)(g.Py / R)))));
  *thrC = std::min(512, std::max(std::max(128, r32((long long)MMP_NP * g.Px / 32)), r32((long long)MMP_TY * g.nx / 8)));
}

}  // namespace mmp

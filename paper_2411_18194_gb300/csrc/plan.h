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

// Pass-ordered Stockham twiddles of a plan: for every pass with Ns > 1, in
// the order block_fft applies them, the entries w_{Ns R}^{r k} for
// r = 1..R-1 (outer) and k = 0..Ns-1 (inner); L - 1 entries (padded to L).
// Built in FP64 and rounded once.
inline std::vector<float2> pass_twiddles(const FftPlan& p) {
  std::vector<float2> w;
  w.reserve(p.L);
  int Ns = 1;
  auto add = [&](int R) {
    if (Ns > 1)
      for (int r = 1; r < R; ++r)
        for (int k = 0; k < Ns; ++k) {
          double a = 2.0 * 3.14159265358979323846 * (double)r * (double)k / ((double)Ns * R);
          w.push_back(make_float2((float)cos(a), (float)(-sin(a))));
        }
    Ns *= R;
  };
  for (int s = 0; s < p.n16; ++s) add(16);
  if (p.n8) add(8);
  if (p.n4) add(4);
  if (p.n2) add(2);
  for (int s = 0; s < p.n3; ++s) add(3);
  while ((int)w.size() < p.L) w.push_back(make_float2(1.0f, 0.0f));
  return w;
}

inline std::vector<float2> roots(int P) {
  std::vector<float2> w(P);
  for (int t = 0; t < P; ++t) {
    double a = 2.0 * 3.14159265358979323846 * (double)t / (double)P;
    w[t] = make_float2((float)cos(a), (float)(-sin(a)));
  }
  return w;
}

// Residue classes of ky per pass-B cluster: the smallest power of two
// (<= 8) whose CTA shared memory (columns, twiddles, kernel slice) fits in
// the 227 KB a block may use, with at most 32 FFT elements per thread of a
// 512-thread block.  0 when none fits.
inline int pick_residues(const Grid& g) {
  for (int R = 1; R <= 8; R *= 2) {
    if (g.Py % R != 0 || (R > 1 && g.Py / R < 2)) break;
    size_t sm = passb_smem(g.ny, g.nz, g.Py, g.kzn, R).total;
    long long el = (long long)3 * g.nz * (g.Py / R);
    if (sm <= 227 * 1024 && el <= 32LL * 512) return R;
  }
  return 0;
}

// Rows per tile of passes A and C: 8, or fewer (down to one row pair) while
// the grid would give fewer than two tiles per SM of the 152.
inline int pick_tile_rows(int ny, int nz) {
  int ty = 8;
  while (ty > 2 && (long long)((ny + ty - 1) / ty) * nz < 2 * 152) ty >>= 1;
  return ty;
}

// Block sizes of passes A, B and C (at most 32 FFT elements per thread).
inline void launch_threads(const Grid& g, int R, int* thrA, int* thrB, int* thrC) {
  auto r32 = [](long long v) { return (int)((v + 31) / 32 * 32); };
  const int np = g.ty >> 1;
  *thrA = std::min(512, std::max(128, r32((long long)np * g.Px / 32)));
  long long elB = (long long)3 * g.nz * (g.Py / R);
  *thrB = std::min(512, std::max(64, r32(std::max(elB / 32, (long long)(g.Py / R)))));
  *thrC = std::min(512, std::max(std::max(128, r32((long long)np * g.Px / 32)), r32((long long)g.ty * g.nx / 8)));
}

}  // namespace mmp

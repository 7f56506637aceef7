// plan.h -- host helpers shared by the C-ABI entry points: padded FFT
// lengths, radix plans and FP64-built twiddle tables.
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

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

// Radix plan of length L = 2^a 3^b.  variant 0: as many radix-16 passes as
// possible (then one 8, 4 or 2); variant 1: radix-8 passes (then one 4 or
// 2).  Both are exact; they differ in FP32 rounding order and speed.
inline bool make_plan(int L, FftPlan& p, int variant = 0) {
  p.L = L;
  p.n16 = p.n8 = p.n4 = p.n2 = p.n3 = 0;
  int r = L, a = 0;
  while (r % 3 == 0) { r /= 3; p.n3++; }
  while (r % 2 == 0) { r /= 2; a++; }
  if (r != 1 || variant < 0 || variant > 1) return false;
  if (variant == 0) {
    p.n16 = a / 4;
    p.n8 = (a % 4) == 3;
    p.n4 = (a % 4) == 2;
    p.n2 = (a % 4) == 1;
  } else {
    p.n8 = a / 3;
    p.n4 = (a % 3) == 2;
    p.n2 = (a % 3) == 1;
  }
  // uniform-stride addressing of stockham_pass: loads need L/R a multiple
  // of 16 (or the transform within 16), stores Ns a multiple of 16 (or a
  // power-of-two radix with R Ns <= 16)
  p.lin = 1;
  int Ns = 1;
  auto check = [&](int R) {
    const int nbf = L / R;
    const bool ld = nbf % 16 == 0 || R * nbf <= 16;
    const bool st = Ns % 16 == 0 || ((R & (R - 1)) == 0 && R * Ns <= 16);
    if (!ld || !st) p.lin = 0;
    Ns *= R;
  };
  for (int s = 0; s < p.n16; ++s) check(16);
  for (int s = 0; s < p.n8; ++s) check(8);
  if (p.n4) check(4);
  if (p.n2) check(2);
  for (int s = 0; s < p.n3; ++s) check(3);
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
  for (int s = 0; s < p.n8; ++s) add(8);
  if (p.n4) add(4);
  if (p.n2) add(2);
  for (int s = 0; s < p.n3; ++s) add(3);
  while ((int)w.size() < p.L) w.push_back(make_float2(1.0f, 0.0f));
  return w;
}

// Complex values one thread holds in a pass of block_fft<.., 32>: 32, but
// 30 for plans with a radix-3 pass (10 butterflies of 3).
inline int fft_cap(const FftPlan& p) { return p.n3 ? 30 : 32; }
inline int fft_cap(int L) {
  FftPlan p;
  return make_plan(L, p) ? fft_cap(p) : 32;
}
// Pass A holds half of that (kCapA = 16 values a thread, two blocks per SM).
inline int fft_cap_a(const FftPlan& p) { return fft_cap(p) / 2; }
inline int fft_cap_a(int L) { return fft_cap(L) / 2; }

// Twiddle table of the warp FFT of length N = 32 M (wfft.cuh):
// entry k1 * 32 + l = w_N^(l k1), k1 < M.  Built in FP64, rounded once.
inline std::vector<float2> warp_twiddles(int N) {
  const int M = N / 32;
  std::vector<float2> w((size_t)32 * M);
  for (int k1 = 0; k1 < M; ++k1)
    for (int l = 0; l < 32; ++l) {
      double a = 2.0 * 3.14159265358979323846 * (double)(l * k1) / (double)N;
      w[k1 * 32 + l] = make_float2((float)cos(a), (float)(-sin(a)));
    }
  return w;
}

// The DFT32 matrices of the tensor-core stage (tcdft.cuh): F = w32^(m k)
// real and imaginary parts, each split into TF32 hi (round to nearest,
// ties away) and the FP32 remainder, in the no-swizzle core-matrix layout:
// element (k, n) at float (8 (n / 8) + k / 4) * 32 + 4 (n % 8) + k % 4 of its
// 1024-float matrix; order Fr hi, Fr lo, Fi hi, Fi lo.  Built in FP64.
inline float tf32_round_host(float x) {
  uint32_t b;
  memcpy(&b, &x, 4);
  b = (b + 0x1000u) & ~0x1FFFu;
  float y;
  memcpy(&y, &b, 4);
  return y;
}
inline std::vector<float> tc_dft32_table() {
  std::vector<float> B(4 * 1024);
  for (int k = 0; k < 32; ++k)
    for (int n = 0; n < 32; ++n) {
      const double a = 2.0 * 3.14159265358979323846 * (double)((k * n) % 32) / 32.0;
      const double fr = cos(a), fi = -sin(a);
      const int off = (8 * (n / 8) + (k / 4)) * 32 + 4 * (n % 8) + (k % 4);
      const float frh = tf32_round_host((float)fr), fih = tf32_round_host((float)fi);
      B[0 * 1024 + off] = frh;
      B[1 * 1024 + off] = (float)(fr - (double)frh);
      B[2 * 1024 + off] = fih;
      B[3 * 1024 + off] = (float)(fi - (double)fih);
    }
  return B;
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
// the 227 KB a block may use, with the FFT elements within what a
// 512-thread block holds (fft_cap per thread).  0 when none fits.
inline int pick_residues(const Grid& g) {
  for (int R = 1; R <= 8; R *= 2) {
    if (g.Py % R != 0 || (R > 1 && g.Py / R < 2)) break;
    size_t sm = passb_smem(g.ny, g.nz, g.Py, g.kzn, R, true).total;
    long long el = (long long)3 * g.nz * (g.Py / R);
    if (sm <= 227 * 1024 && el <= (long long)fft_cap(g.Py / R) * 512) return R;
  }
  return 0;
}

// Rows per tile of passes A and C: 8, or fewer (down to one row pair) while
// the grid would give fewer than two tiles per SM of the 152, or while pass
// A's row pairs exceed what a 512-thread block of it holds.
// Pass C: pass A's tile height, fewer rows while its row pairs exceed what
// a 512-thread block of it holds.
inline int pick_tile_rows_c(int ty, int Px) {
  int tyc = ty;
  while (tyc > 2 && (long long)(tyc / 2) * Px > (long long)fft_cap(Px) * 512) tyc >>= 1;
  return tyc;
}

inline int pick_tile_rows(int ny, int nz, int Px) {
  int ty = 8;
  while (ty > 2 && (long long)((ny + ty - 1) / ty) * nz < 2 * 152) ty >>= 1;
  while (ty > 2 && (long long)(ty / 2) * Px > (long long)fft_cap_a(Px) * 512) ty >>= 1;
  return ty;
}

// Block sizes of passes A, B and C (at most fft_cap FFT elements per
// thread; pick_residues and the x-length limit keep them within 512).
inline void launch_threads(const Grid& g, int R, int* thrA, int* thrB, int* thrC) {
  auto r32 = [](long long v) { return (int)((v + 31) / 32 * 32); };
  auto need = [](long long el, int cap) { return (el + cap - 1) / cap; };
  const int np = g.ty >> 1;
  const long long fa = need((long long)g.xb * np * g.Px, fft_cap_a(g.Px));
  *thrA = std::min(512, std::max(128, r32(fa)));
  const int Ly = g.Py / R;
  const long long elB = (long long)3 * g.nz * Ly;
  *thrB = std::min(512, std::max(64, r32(std::max(need(elB, fft_cap(Ly)), (long long)Ly))));
  const long long fc = need((long long)g.xbc * (g.tyc >> 1) * g.Px, fft_cap(g.Px));
  *thrC = std::min(512, std::max(std::max(128, r32(fc)), r32((long long)g.tyc * g.nx / 8)));
}

}  // namespace mmp

// common.cuh -- shared device definitions of libmmp (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define MMP_MAX_REGIONS 256
#define MMP_TY 8              // largest number of rows (y) per tile of the x-FFT passes

namespace mmp {

constexpr double kGamma = 1.7595e11;           // rad s^-1 T^-1
constexpr double kMu0 = 4e-7 * 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Double-float arithmetic (value = hi + lo, |lo| <= ulp(hi)/2).  Used where a
// field term far exceeds the tolerance of the sum (the exchange field of a
// random state reaches ~1e2 T, the homogeneous AFM exchange ~2e3 T): the
// differences m_nb - m are formed exactly (TwoSum, Knuth) and products
// with FMA-based TwoProduct (Dekker), so one rounding remains at the end.
// ---------------------------------------------------------------------------
struct df { float hi, lo; };

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  float e = s.lo + (a.lo + b.lo);
  return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, s.lo + a.lo);
}
// (c.hi + c.lo) * (d.hi + d.lo), error O(eps^2)
__device__ __forceinline__ df df_mul(df c, df d) {
  float p = c.hi * d.hi;
  float e = fmaf(c.hi, d.hi, -p);
  e = fmaf(c.hi, d.lo, fmaf(c.lo, d.hi, e));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_mul_f(df c, float x) {
  float p = c.hi * x;
  float e = fmaf(c.hi, x, -p);
  e = fmaf(c.lo, x, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ float df_round(df a) { return a.hi + a.lo; }

// ---------------------------------------------------------------------------
// Per (sublattice, region) coefficients, derived on the host in FP64 and
// rounded once.  `exch` and `afm0` keep a second float for the double-float
// products above.
// ---------------------------------------------------------------------------
struct RegionCoef {
  float ms;            // Ms (A/m); 0 = empty cell
  float alpha;         // Gilbert damping
  float tq;            // -gamma / (1 + alpha^2)
  float2 exch[3];      // 2 A / (Ms h_a^2) per axis (hi, lo)
  float two_over_ms_h2[3];  // 2 / (Ms h_a^2) (multi-region pair coefficient factor)
  float2 two_over_ms_h2_df[3];
  float aex;           // A
  float dind;          // D
  float dmi[3];        // D / (Ms h_a) for a = x, y (index 2 unused)
  float ghost[3];      // h_a D / (2 A) (ghost offset factor), 0 when A = 0
  float exbc[3];       // D / (Ms h_a) exchange term of the boundary ghost, 0 when A = 0
  float inv_ms;        // 1 / Ms
  float ku1, ku2, kb1; // 2 Ku1/Ms, 4 Ku2/Ms, 2 Kb1/Ms
  float u[3], ub[3];   // anisotropy axes (unit)
  float bext[3];       // external field (T)
  float afm12[3];      // A12 / (Ms h_a^2)
  float2 afm0;         // 4 A0 / (Ms a^2) (hi, lo)
  float kc1;           // 2 Kc1 / Ms (cubic anisotropy)
  float c1[3], c2[3], c3[3];   // cubic axes (orthonormal)
  float mel1, mel2;    // -2 B1 / Ms, -2 B2 / Ms
  float b1, b2;        // B1, B2 (J/m^3) for the magnetoelastic force
};

}  // namespace mmp

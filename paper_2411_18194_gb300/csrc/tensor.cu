// tensor.cu -- FP64 construction of the demag kernel spectrum on the device.
//
// Methods, "Magnetostatic field": the cell-to-cell demag tensor N is the
// analytical result of Newell, Williams and Dunlop below a cutoff radius and
// an asymptotic result above it.  Built here in FP64 (the Newell second
// differences cancel catastrophically) and transformed in FP64; only the
// final spectrum is rounded to FP32.
//
//  * Newell: N_xx is the 27-point second difference (weights 2, -1, -1 per
//    axis) of f(x, y, z), N_xy that of g(x, y, z), divided by 4 pi V.
//  * Far field: N_ab(r) = -V/(4 pi) sum_{alpha even, |alpha| <= 2P}
//    E[s^alpha]/alpha! d^(alpha + e_a + e_b)(1/r), the expansion of the
//    cell-pair average over the difference s of two uniform points of a
//    cell (triangular per axis, E[s^2k] = 2 D^2k / ((2k+1)(2k+2))).  The
//    derivatives of 1/r = F(r^2), F(q) = q^(-1/2), use the Hermite-type
//    chain rule  d^t_x F(x^2 + ...) = sum_i t!/(i!(t-2i)!) (2x)^(t-2i) F^(t-i)
//    applied per axis, with F^(n)(r^2) = (-1)^n (2n-1)!!/2^n r^(-2n-1).
//  * Spectrum: the kernel of the zero-padded convolution is even or odd in
//    each axis, so its DFT is real: along an axis with padded length P the
//    transform is N(0) + 2 sum_i N(i) cos(2 pi k i / P) (even) or
//    -2i sum_i N(i) sin(2 pi k i / P) (odd); two odd axes give the factor
//    (-i)^2 = -1.  Only the octant 0 <= k <= P/2 is stored.
#include <math.h>
#include "kernels.h"

namespace mmp {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kOrder = 4;                  // expansion through E[s^8]
constexpr int kNmax = 2 * kOrder + 2;      // highest derivative order of 1/r

__device__ __noinline__ double newell_f(double x, double y, double z) {
  x = fabs(x); y = fabs(y); z = fabs(z);
  double x2 = x * x, y2 = y * y, z2 = z * z;
  double R = sqrt(x2 + y2 + z2);
  double out = (2.0 * x2 - y2 - z2) * R / 6.0;
  double rxz = sqrt(x2 + z2), rxy = sqrt(x2 + y2);
  if (rxz > 0) out += 0.5 * y * (z2 - x2) * asinh(y / rxz);
  if (rxy > 0) out += 0.5 * z * (y2 - x2) * asinh(z / rxy);
  if (x > 0) out -= x * y * z * atan(y * z / (x * R));
  return out;
}

__device__ __noinline__ double newell_g(double x, double y, double z) {
  double sgn = ((x < 0) != (y < 0)) ? -1.0 : 1.0;
  if (x == 0 || y == 0) sgn = 0.0;
  x = fabs(x); y = fabs(y); z = fabs(z);
  double x2 = x * x, y2 = y * y, z2 = z * z;
  double R = sqrt(x2 + y2 + z2);
  double out = -x * y * R / 3.0;
  double rxy = sqrt(x2 + y2), ryz = sqrt(y2 + z2), rxz = sqrt(x2 + z2);
  if (rxy > 0) out += x * y * z * asinh(z / rxy);
  if (ryz > 0) out += y / 6.0 * (3.0 * z2 - y2) * asinh(x / ryz);
  if (rxz > 0) out += x / 6.0 * (3.0 * z2 - x2) * asinh(y / rxz);
  if (z > 0) out -= z * z2 / 6.0 * atan(x * y / (z * R));
  if (y > 0) out -= z * y2 / 2.0 * atan(x * z / (y * R));
  if (x > 0) out -= z * x2 / 2.0 * atan(y * z / (x * R));
  return sgn * out;
}

template <bool G>
__device__ double second_difference(double X, double Y, double Z, double a, double b, double c) {
  const double w[3] = {-1.0, 2.0, -1.0};
  double acc = 0.0;
#pragma unroll 1
  for (int i = 0; i < 3; ++i)
#pragma unroll 1
    for (int j = 0; j < 3; ++j)
#pragma unroll 1
      for (int k = 0; k < 3; ++k) {
        double f = G ? newell_g(X + (i - 1) * a, Y + (j - 1) * b, Z + (k - 1) * c)
                     : newell_f(X + (i - 1) * a, Y + (j - 1) * b, Z + (k - 1) * c);
        acc += w[i] * w[j] * w[k] * f;
      }
  return acc / (4.0 * kPi * a * b * c);
}

__device__ double moment(double d, int k) {
  if (k == 0) return 1.0;
  double p = 1.0;
  for (int i = 0; i < 2 * k; ++i) p *= d;
  return 2.0 * p / ((2 * k + 1) * (2 * k + 2));
}

__device__ __forceinline__ double fact(int n) {
  const double f[11] = {1.0, 1.0, 2.0, 6.0, 24.0, 120.0, 720.0, 5040.0, 40320.0, 362880.0, 3628800.0};
  return f[n];
}

// d^t_x d^u_y d^v_z (1/r) from powers p{x,y,z}[e] = (2X)^e etc. and
// Fn[n] = F^(n)(r^2).
__device__ __noinline__ double inv_r_derivative(int t, int u, int v, const double* px, const double* py,
                                   const double* pz, const double* Fn) {
  double acc = 0.0;
#pragma unroll 1
  for (int i = 0; 2 * i <= t; ++i) {
    double hi = fact(t) / (fact(i) * fact(t - 2 * i)) * px[t - 2 * i];
    for (int j = 0; 2 * j <= u; ++j) {
      double hj = hi * fact(u) / (fact(j) * fact(u - 2 * j)) * py[u - 2 * j];
      for (int k = 0; 2 * k <= v; ++k)
        acc += hj * fact(v) / (fact(k) * fact(v - 2 * k)) * pz[v - 2 * k] * Fn[t + u + v - i - j - k];
    }
  }
  return acc;
}

// N octant: out[comp][k][j][i] for offsets (i dx, j dy, k dz); cell sizes
// scaled by the largest one (N is scale invariant).
__global__ void k_tensor_octant(double* __restrict__ out, int nx, int ny, int nz, double dx,
                                double dy, double dz, double rc) {
  long long n = (long long)nx * ny * nz;
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n) return;
  int i = idx % nx, j = (idx / nx) % ny, k = idx / ((long long)nx * ny);
  double X = i * dx, Y = j * dy, Z = k * dz;
  double N6[6];
  if (sqrt(X * X + Y * Y + Z * Z) < rc) {
    N6[0] = second_difference<false>(X, Y, Z, dx, dy, dz);
    N6[1] = second_difference<false>(Y, X, Z, dy, dx, dz);
    N6[2] = second_difference<false>(Z, Y, X, dz, dy, dx);
    N6[3] = second_difference<true>(X, Y, Z, dx, dy, dz);
    N6[4] = second_difference<true>(X, Z, Y, dx, dz, dy);
    N6[5] = second_difference<true>(Y, Z, X, dy, dz, dx);
  } else {
    double px[kNmax + 1], py[kNmax + 1], pz[kNmax + 1], Fn[kNmax + 1];
    px[0] = py[0] = pz[0] = 1.0;
    for (int e = 1; e <= kNmax; ++e) {
      px[e] = px[e - 1] * 2.0 * X;
      py[e] = py[e - 1] * 2.0 * Y;
      pz[e] = pz[e - 1] * 2.0 * Z;
    }
    double r2 = X * X + Y * Y + Z * Z;
    double p = 1.0 / sqrt(r2), c = 1.0;   // F^(n) = (-1)^n (2n-1)!!/2^n r^(-2n-1)
    for (int m = 0; m <= kNmax; ++m) {
      Fn[m] = c * p;
      c *= -(2.0 * m + 1.0) / 2.0;
      p /= r2;
    }
    const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
    double V = dx * dy * dz;
    for (int c6 = 0; c6 < 6; ++c6) N6[c6] = 0.0;
#pragma unroll 1
    for (int a = 0; a <= kOrder; ++a)
      for (int b = 0; b <= kOrder - a; ++b)
        for (int e = 0; e <= kOrder - a - b; ++e) {
          double coef = moment(dx, a) * moment(dy, b) * moment(dz, e) /
                        (fact(2 * a) * fact(2 * b) * fact(2 * e));
          for (int c6 = 0; c6 < 6; ++c6) {
            int t = 2 * a + (pa[c6] == 0) + (pb[c6] == 0);
            int u = 2 * b + (pa[c6] == 1) + (pb[c6] == 1);
            int v = 2 * e + (pa[c6] == 2) + (pb[c6] == 2);
            N6[c6] += coef * inv_r_derivative(t, u, v, px, py, pz, Fn);
          }
        }
    for (int c = 0; c < 6; ++c) N6[c] *= -V / (4.0 * kPi);
  }
  for (int c = 0; c < 6; ++c) out[c * n + idx] = N6[c];
}

// One axis of the real cos/sin transform.  in: [6][e2][e1][e0] with the
// transformed axis of extent nin; out: same with extent nout = P/2+1.
// trig[t] = (cos, sin)(2 pi t / P), t in [0, P).
__global__ void k_tensor_axis(const double* __restrict__ in, double* __restrict__ out, int e0, int e1,
                              int e2, int axis, int nin, int nout, int P, const double2* __restrict__ trig,
                              int odd_mask) {
  int o0 = axis == 0 ? nout : e0, o1 = axis == 1 ? nout : e1, o2 = axis == 2 ? nout : e2;
  long long per = (long long)o0 * o1 * o2;
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= 6 * per) return;
  int comp = idx / per;
  long long r = idx - comp * per;
  int i0 = r % o0, i1 = (r / o0) % o1, i2 = r / ((long long)o0 * o1);
  int kk = axis == 0 ? i0 : (axis == 1 ? i1 : i2);
  long long stride = axis == 0 ? 1 : (axis == 1 ? (long long)e0 : (long long)e0 * e1);
  long long base = (long long)comp * e0 * e1 * e2 + (long long)(axis == 0 ? 0 : i0) +
                   (long long)(axis == 1 ? 0 : i1) * e0 + (long long)(axis == 2 ? 0 : i2) * e0 * e1;
  bool odd = (odd_mask >> comp) & 1;
  double acc = odd ? 0.0 : in[base];
  for (int i = 1; i < nin; ++i) {
    int t = (int)(((long long)kk * i) % P);
    double w = odd ? trig[t].y : trig[t].x;
    acc += 2.0 * w * in[base + i * stride];
  }
  out[comp * per + r] = acc;
}

// Final scaling and layout change to float [kx][ky][krow], row = 6 floats
// per kz (xx, yy, zz, xy, xz, yz) and zero padding to krow.
__global__ void k_tensor_store(const double* __restrict__ in, float* __restrict__ out, int mx, int my,
                               int mz, int krow, double scale_even, double scale_odd2) {
  long long per = (long long)mx * my * mz;
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= per) return;
  int ix = idx % mx, iy = (idx / mx) % my, iz = idx / ((long long)mx * my);
  long long row = ((long long)ix * my + iy) * krow;
  if (iz == 0)
    for (int c = 6 * mz; c < krow; ++c) out[row + c] = 0.0f;
  long long o = row + iz * 6;
  for (int c = 0; c < 6; ++c) out[o + c] = (float)(in[c * per + idx] * (c < 3 ? scale_even : scale_odd2));
}

}  // namespace

cudaError_t build_kernel_spectrum(const KernelBuild& kb, cudaStream_t s) {
  const int nx = kb.n[0], ny = kb.n[1], nz = kb.n[2];
  double L = fmax(kb.cell[0], fmax(kb.cell[1], kb.cell[2]));
  long long n = (long long)nx * ny * nz;
  k_tensor_octant<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(kb.buf0, nx, ny, nz, kb.cell[0] / L,
                                                              kb.cell[1] / L, kb.cell[2] / L, kb.rc);
  // odd masks per axis: x odd for xy, xz; y odd for xy, yz; z odd for xz, yz
  const int odd[3] = {(1 << 3) | (1 << 4), (1 << 3) | (1 << 5), (1 << 4) | (1 << 5)};
  int e[3] = {nx, ny, nz};
  double* src = kb.buf0;
  double* dst = kb.buf1;
  for (int a = 0; a < 3; ++a) {
    if (kb.P[a] == 1) continue;
    int nout = kb.P[a] / 2 + 1;
    long long total = 6LL * nout * (a == 0 ? 1 : e[0]) * (a == 1 ? 1 : e[1]) * (a == 2 ? 1 : e[2]);
    k_tensor_axis<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(src, dst, e[0], e[1], e[2], a, e[a], nout,
                                                                  kb.P[a], kb.trig[a], odd[a]);
    e[a] = nout;
    double* t = src; src = dst; dst = t;
  }
  double scale = -kMu0 / ((double)kb.P[0] * kb.P[1] * kb.P[2]);
  long long per = (long long)e[0] * e[1] * e[2];
  k_tensor_store<<<(unsigned)((per + 127) / 128), 128, 0, s>>>(src, kb.out, e[0], e[1], e[2], kb.krow, scale,
                                                                -scale);
  return cudaGetLastError();
}

}  // namespace mmp

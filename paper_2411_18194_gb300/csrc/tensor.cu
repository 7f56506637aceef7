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
//    The far-field terms are evaluated in FP32 (no cancellation there that
//    FP32 cannot carry: the kernel is smooth and ~1/r^3 above the cutoff).
//  * Spectrum: the kernel of the zero-padded convolution is even or odd in
//    each axis, so its DFT is real: along an axis with padded length P the
//    transform is N(0) + 2 sum_i N(i) cos(2 pi k i / P) (even) or
//    -2i sum_i N(i) sin(2 pi k i / P) (odd); two odd axes give the factor
//    (-i)^2 = -1.  Only the octant 0 <= k <= P/2 is stored.  Axes with
//    P >= 64 are transformed by an FP64 FFT of the evenly or oddly extended
//    line, shorter ones by the direct sums.
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

// Far field in FP32.  Above the cutoff the kernel is smooth and of size
// ~1/r^3; its terms are evaluated in single precision (relative rounding
// ~1e-7 of the kernel's scale there, against the 1e-5 Ms field bar), with
// every index a compile-time constant after unrolling.
// c(t, i) = t! / (i! (t - 2i)!), the coefficients of the chain rule
// d^t_x F(x^2 + ..) = sum_i c(t, i) (2x)^(t - 2i) F^(t - i).
__host__ __device__ constexpr float chain_coef(int t, int i) {
  float v = 1.0f;
  for (int m = t - 2 * i + 1; m <= t; ++m) v *= (float)m;   // t! / (t - 2i)!
  for (int m = 2; m <= i; ++m) v /= (float)m;               // / i!
  return v;
}
// d^t_x d^u_y d^v_z (1/r) from px[e] = (2X)^e (etc.) and Fn[n] = F^(n)(r^2)
__device__ __forceinline__ float inv_r_derivative(int t, int u, int v, const float (&px)[kNmax + 1],
                                                  const float (&py)[kNmax + 1], const float (&pz)[kNmax + 1],
                                                  const float (&Fn)[kNmax + 1]) {
  float acc = 0.0f;
#pragma unroll
  for (int i = 0; i <= kNmax / 2; ++i) {
    if (2 * i > t) break;
#pragma unroll
    for (int j = 0; j <= kNmax / 2; ++j) {
      if (2 * j > u) break;
#pragma unroll
      for (int k = 0; k <= kNmax / 2; ++k) {
        if (2 * k > v) break;
        const float c = chain_coef(t, i) * chain_coef(u, j) * chain_coef(v, k);
        acc = fmaf(c * px[t - 2 * i] * py[u - 2 * j], pz[v - 2 * k] * Fn[t + u + v - i - j - k], acc);
      }
    }
  }
  return acc;
}

// N octant: out[comp][k][j][i] for offsets (i dx, j dy, k dz); cell sizes
// scaled by the largest one (N is scale invariant).
// Moment weights of the far-field expansion, w[a][b][e] =
// E[s_x^2a] E[s_y^2b] E[s_z^2e] / ((2a)! (2b)! (2e)!) (a + b + e <= kOrder),
// E[s^2k] = 2 d^2k / ((2k+1)(2k+2)) for the difference s of two uniform
// points of a cell of width d (1 for k = 0); built on the host in FP64.
struct FarWeights {
  float w[kOrder + 1][kOrder + 1][kOrder + 1];
};

__global__ void k_tensor_octant(double* __restrict__ out, int nx, int ny, int nz, double dx,
                                double dy, double dz, double rc, FarWeights fw) {
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
    const float x = (float)X, y = (float)Y, z = (float)Z;
    float px[kNmax + 1], py[kNmax + 1], pz[kNmax + 1], Fn[kNmax + 1];
    px[0] = py[0] = pz[0] = 1.0f;
#pragma unroll
    for (int e = 1; e <= kNmax; ++e) {
      px[e] = px[e - 1] * 2.0f * x;
      py[e] = py[e - 1] * 2.0f * y;
      pz[e] = pz[e - 1] * 2.0f * z;
    }
    const float r2 = x * x + y * y + z * z, ir2 = 1.0f / r2;
    Fn[0] = 1.0f / sqrtf(r2);   // F^(n) = (-1)^n (2n-1)!!/2^n r^(-2n-1)
#pragma unroll
    for (int m = 1; m <= kNmax; ++m) Fn[m] = Fn[m - 1] * (-(2.0f * m - 1.0f) / 2.0f) * ir2;
    float acc[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    constexpr int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int a = 0; a <= kOrder; ++a)
#pragma unroll
      for (int b = 0; b <= kOrder; ++b)
#pragma unroll
        for (int e = 0; e <= kOrder; ++e) {
          if (a + b + e > kOrder) continue;
          const float w = fw.w[a][b][e];
#pragma unroll
          for (int c6 = 0; c6 < 6; ++c6) {
            const int t = 2 * a + (pa[c6] == 0) + (pb[c6] == 0);
            const int u = 2 * b + (pa[c6] == 1) + (pb[c6] == 1);
            const int v = 2 * e + (pa[c6] == 2) + (pb[c6] == 2);
            acc[c6] = fmaf(w, inv_r_derivative(t, u, v, px, py, pz, Fn), acc[c6]);
          }
        }
    const double V = dx * dy * dz;
    for (int c = 0; c < 6; ++c) N6[c] = -V / (4.0 * kPi) * (double)acc[c];
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

// One axis of the real cos/sin transform by an FP64 FFT, for padded
// lengths P >= 64 (P = 2^a or 3 * 2^a): one block per line.  The line is
// extended to length P evenly (N(P - i) = N(i)) or oddly (N(P - i) = -N(i))
// in shared memory, transformed by a forward Stockham FFT (a radix-3 pass
// first when 3 divides P, then radix-2 passes; pass of radix R with Ns
// outputs per sub-transform: inputs j + r P/R, twiddle w_(Ns R)^(r (j mod Ns)),
// outputs at (j / Ns) Ns R + j mod Ns + r Ns), and the outputs k <= P/2
// are the real part (even: N(0) + 2 sum N(i) cos) or minus the imaginary
// part (odd: 2 sum N(i) sin), the same values as k_tensor_axis.
template <int R>
__device__ __forceinline__ void fft64_pass(const double2* __restrict__ x, double2* __restrict__ y, int P, int Ns,
                                           const double2* __restrict__ trig) {
  const int NR = P / R, step = P / (Ns * R);
  for (int j = threadIdx.x; j < NR; j += blockDim.x) {
    const int k = j % Ns;
    double2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[j + r * NR];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const double2 w = trig[(r * k * step) % P];   // (cos, sin): the forward twiddle is its conjugate
      v[r] = make_double2(v[r].x * w.x + v[r].y * w.y, v[r].y * w.x - v[r].x * w.y);
    }
    double2 o[R];
    if (R == 2) {
      o[0] = make_double2(v[0].x + v[1].x, v[0].y + v[1].y);
      o[1] = make_double2(v[0].x - v[1].x, v[0].y - v[1].y);
    } else {
      // w3 = exp(-2 pi i / 3) = (-1/2, -s3)
      const double s3 = 0.86602540378443864676;
      const double2 t = make_double2(v[1].x + v[2].x, v[1].y + v[2].y);
      const double2 d = make_double2(v[1].x - v[2].x, v[1].y - v[2].y);
      const double2 m = make_double2(v[0].x - 0.5 * t.x, v[0].y - 0.5 * t.y);
      o[0] = make_double2(v[0].x + t.x, v[0].y + t.y);
      o[1] = make_double2(m.x + s3 * d.y, m.y - s3 * d.x);
      o[2] = make_double2(m.x - s3 * d.y, m.y + s3 * d.x);
    }
    const int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) y[base + r * Ns] = o[r];
  }
  __syncthreads();
}

__global__ void k_tensor_axis_fft(const double* __restrict__ in, double* __restrict__ out, int e0, int e1, int e2,
                                  int axis, int nin, int nout, int P, const double2* __restrict__ trig,
                                  int odd_mask) {
  extern __shared__ double2 fbuf[];
  double2* x = fbuf;
  double2* y = fbuf + P;
  // the line: its coordinates (i0, i1, i2) with 0 on the transformed axis
  const int l0 = axis == 0 ? 1 : e0, l1 = axis == 1 ? 1 : e1, l2 = axis == 2 ? 1 : e2;
  const long long lines = (long long)l0 * l1 * l2;
  const int comp = (int)(blockIdx.x / lines);
  const long long rem = blockIdx.x - comp * lines;
  const int i0 = (int)(rem % l0), i1 = (int)((rem / l0) % l1), i2 = (int)(rem / ((long long)l0 * l1));
  const long long istride = axis == 0 ? 1 : (axis == 1 ? (long long)e0 : (long long)e0 * e1);
  const long long ibase = (long long)comp * e0 * e1 * e2 + i0 + (long long)i1 * e0 + (long long)i2 * e0 * e1;
  const bool odd = (odd_mask >> comp) & 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) x[i] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int i = threadIdx.x; i < nin; i += blockDim.x) {   // nin <= P / 2: no overlap of i and P - i
    const double v = in[ibase + i * istride];
    if (i == 0) {
      x[0].x = odd ? 0.0 : v;
    } else {
      x[i].x = v;
      x[P - i].x = odd ? -v : v;
    }
  }
  __syncthreads();
  int Ns = 1;
  if (P % 3 == 0) {
    fft64_pass<3>(x, y, P, Ns, trig);
    double2* t = x; x = y; y = t;
    Ns = 3;
  }
  while (Ns < P) {
    fft64_pass<2>(x, y, P, Ns, trig);
    double2* t = x; x = y; y = t;
    Ns *= 2;
  }
  const int q0 = axis == 0 ? nout : e0, q1 = axis == 1 ? nout : e1, q2 = axis == 2 ? nout : e2;
  const long long ostride = axis == 0 ? 1 : (axis == 1 ? (long long)q0 : (long long)q0 * q1);
  const long long obase = (long long)comp * q0 * q1 * q2 + i0 + (long long)i1 * q0 + (long long)i2 * q0 * q1;
  for (int k = threadIdx.x; k < nout; k += blockDim.x) out[obase + k * ostride] = odd ? -x[k].y : x[k].x;
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
  FarWeights fw;
  {
    const double d[3] = {kb.cell[0] / L, kb.cell[1] / L, kb.cell[2] / L};
    double m[3][kOrder + 1];
    double f2[kOrder + 1];
    for (int k = 0; k <= kOrder; ++k) {
      double f = 1.0;
      for (int q = 2; q <= 2 * k; ++q) f *= q;
      f2[k] = f;                                   // (2k)!
      for (int ax = 0; ax < 3; ++ax)
        m[ax][k] = k == 0 ? 1.0 : 2.0 * pow(d[ax], 2 * k) / ((2.0 * k + 1.0) * (2.0 * k + 2.0));
    }
    for (int a = 0; a <= kOrder; ++a)
      for (int b = 0; b <= kOrder; ++b)
        for (int e = 0; e <= kOrder; ++e)
          fw.w[a][b][e] = a + b + e > kOrder ? 0.0f
                                             : (float)(m[0][a] * m[1][b] * m[2][e] / (f2[a] * f2[b] * f2[e]));
  }
  k_tensor_octant<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(kb.buf0, nx, ny, nz, kb.cell[0] / L,
                                                              kb.cell[1] / L, kb.cell[2] / L, kb.rc, fw);
  // odd masks per axis: x odd for xy, xz; y odd for xy, yz; z odd for xz, yz
  const int odd[3] = {(1 << 3) | (1 << 4), (1 << 3) | (1 << 5), (1 << 4) | (1 << 5)};
  int e[3] = {nx, ny, nz};
  double* src = kb.buf0;
  double* dst = kb.buf1;
  for (int a = 0; a < 3; ++a) {
    if (kb.P[a] == 1) continue;
    int nout = kb.P[a] / 2 + 1;
    const long long lines = 6LL * (a == 0 ? 1 : e[0]) * (a == 1 ? 1 : e[1]) * (a == 2 ? 1 : e[2]);
    if (kb.P[a] >= 64) {   // FP64 FFT per line
      const size_t sm = (size_t)2 * kb.P[a] * sizeof(double2);
      cudaError_t err = cudaFuncSetAttribute(k_tensor_axis_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (err != cudaSuccess) return err;
      k_tensor_axis_fft<<<(unsigned)lines, 256, sm, s>>>(src, dst, e[0], e[1], e[2], a, e[a], nout, kb.P[a],
                                                         kb.trig[a], odd[a]);
    } else {               // short axes: the direct sums
      const long long total = lines * nout;
      k_tensor_axis<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(src, dst, e[0], e[1], e[2], a, e[a], nout,
                                                                    kb.P[a], kb.trig[a], odd[a]);
    }
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

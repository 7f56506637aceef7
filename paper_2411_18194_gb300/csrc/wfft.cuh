// wfft.cuh -- warp-level FFTs of power-of-two lengths N = 32 M (M = 1, 2,
// 4, 8, 16, 32), the transform engine of the warp passes (passb_w.cuh,
// xfft_w.cuh).
//
// The zero-padded convolution of the paper's magnetostatic field (Methods,
// "Magnetostatic field") needs, per padded axis of length 2N, the DFT of N
// nonzero values and its inverse cropped to N outputs.  Both split exactly
// into two length-N transforms (the even and the odd outputs), so every
// transform here has length N = 32 M and is done by one warp:
//
//   n = l + 32 m (lane l, register m),  k = k1 + M k2,
//   X[k] = sum_l w32^(l k2) [ w_N^(l k1) sum_m x[l + 32 m] w_M^(m k1) ],
//
// i.e. an in-register DFT of length M per lane, one twiddle per value, one
// transpose through the warp's own 8 KB of shared memory (XOR-swizzled, so
// both its stores and its loads are bank-conflict free), and an
// in-register DFT of length 32.  A warp holds 32 complex values per lane:
// B = 32 / M transforms at once.  There is no block barrier inside a
// transform (only __syncwarp), and every index is a compile-time constant
// plus the lane.
#pragma once
#include "fft.cuh"

namespace mmp {

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// cos(2 pi k / 32) and sin(2 pi k / 32) for k = 0..8 (quarter wave); other k
// by symmetry at compile time.
__host__ __device__ constexpr float kCos32q(int k) {
  return k == 0 ? 1.0f
       : k == 1 ? 0.98078528040323044913f
       : k == 2 ? 0.92387953251128675613f
       : k == 3 ? 0.83146961230254523708f
       : k == 4 ? 0.70710678118654752440f
       : k == 5 ? 0.55557023301960222474f
       : k == 6 ? 0.38268343236508977173f
       : k == 7 ? 0.19509032201612826785f
       : 0.0f;
}
__host__ __device__ constexpr float cos32(int k) {
  return (k & 31) <= 8 ? kCos32q(k & 31)
       : (k & 31) <= 16 ? -kCos32q(16 - (k & 31))
       : (k & 31) <= 24 ? -kCos32q((k & 31) - 16)
       : kCos32q(32 - (k & 31));
}
__host__ __device__ constexpr float sin32(int k) { return cos32(k - 8); }

// a * w32^(K) (forward: exp(-2 pi i K / 32)) or its conjugate (inverse),
// with the trivial and the 45-degree cases done without a full product.
template <int K, bool INV>
__device__ __forceinline__ float2 mul_w32(float2 a) {
  constexpr int k = K & 31;
  if constexpr (k == 0) return a;
  else if constexpr (k == 8) return mul_mi<INV>(a);                   // -i
  else if constexpr (k == 16) return make_float2(-a.x, -a.y);
  else if constexpr (k == 24) return mul_mi<!INV>(a);                 // +i
  else {
    constexpr float c = cos32(k), s = sin32(k);
    // forward: (c - i s) a; inverse: (c + i s) a
    return INV ? make_float2(fmaf(c, a.x, -s * a.y), fmaf(c, a.y, s * a.x))
               : make_float2(fmaf(c, a.x, s * a.y), fmaf(c, a.y, -s * a.x));
  }
}

// In-register DFT of length 32 (natural order in and out): two length-16
// DFTs of the even and odd elements, then one radix-2 step.
template <bool INV>
__device__ __forceinline__ void dft32(float2 (&v)[32]) {
  float2 e[16], o[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    e[i] = v[2 * i];
    o[i] = v[2 * i + 1];
  }
  dft16<INV>(e);
  dft16<INV>(o);
  float2 t;
#define MMP_R2(K)                      \
  t = mul_w32<K, INV>(o[K]);           \
  v[K] = cadd(e[K], t);                \
  v[K + 16] = csub(e[K], t);
  MMP_R2(0) MMP_R2(1) MMP_R2(2) MMP_R2(3) MMP_R2(4) MMP_R2(5) MMP_R2(6) MMP_R2(7)
  MMP_R2(8) MMP_R2(9) MMP_R2(10) MMP_R2(11) MMP_R2(12) MMP_R2(13) MMP_R2(14) MMP_R2(15)
#undef MMP_R2
}

// In-register DFT of length M in {1, 2, 4, 8, 16, 32}.
template <int M, bool INV>
__device__ __forceinline__ void dft_m(float2 (&t)[M]) {
  if constexpr (M == 2) dft2<INV>(t[0], t[1]);
  else if constexpr (M == 4) dft4<INV>(t[0], t[1], t[2], t[3]);
  else if constexpr (M == 8) dft8<INV>(t);
  else if constexpr (M == 16) dft16<INV>(t);
  else if constexpr (M == 32) dft32<INV>(t);
}

// Twiddle table of the warp transform of length N = 32 M: twT[k1 * 32 + l]
// = w_N^(l k1), k1 < M (built on the host in FP64, rounded once).
__host__ __device__ __forceinline__ int wfft_twiddles(int M) { return 32 * M; }

// Forward warp FFT of B = 32 / M transforms of length N = 32 M.
// On entry lane l holds v[b M + m] = x_b[l + 32 m].
// On exit lane j holds v[k2] = X_b[k1 + M k2] with b = j / M, k1 = j mod M.
// `scr`: the warp's 1024 float2 of shared memory (free on entry; holds
// nothing on exit).  `twT`: the twiddle table above (shared memory).
// Stage 1: the in-register DFTs of length M over m.
template <int M>
__device__ __forceinline__ void wfft_stage1(float2 (&v)[32]) {
  constexpr int B = 32 / M;
#pragma unroll
  for (int b = 0; b < B; ++b) {
    float2 t[M];
#pragma unroll
    for (int m = 0; m < M; ++m) t[m] = v[b * M + m];
    dft_m<M, false>(t);
#pragma unroll
    for (int m = 0; m < M; ++m) v[b * M + m] = t[m];
  }
}

// Stage 1, twiddles and transpose (forward): on return lane j holds the 32
// inputs of its final DFT32 (stage 2).  TWG: twT is in global memory (read
// through the read-only path), else in shared memory.
template <int M, bool TWG = false>
__device__ __forceinline__ void wfft_head(float2 (&v)[32], float2* scr, const float2* twT) {
  constexpr bool INV = false;
  constexpr int B = 32 / M;
  const int l = lane_id();
  wfft_stage1<M>(v);
  if constexpr (M > 1) {
#pragma unroll
    for (int k1 = 1; k1 < M; ++k1) {
      float2 w = TWG ? __ldg(twT + k1 * 32 + l) : twT[k1 * 32 + l];
      if (INV) w.y = -w.y;
#pragma unroll
      for (int b = 0; b < B; ++b) v[b * M + k1] = cmul(v[b * M + k1], w);
    }
  }
  // transpose: row r = b M + k1, column l, stored at r * 32 + (l ^ r)
#pragma unroll
  for (int r = 0; r < 32; ++r) scr[r * 32 + (l ^ r)] = v[r];
  __syncwarp();
#pragma unroll
  for (int c = 0; c < 32; ++c) v[c] = scr[l * 32 + (c ^ l)];
  __syncwarp();
}

template <int M, bool TWG = false>
__device__ __forceinline__ void wfft_fwd(float2 (&v)[32], float2* scr, const float2* twT) {
  wfft_head<M, TWG>(v, scr, twT);
  dft32<false>(v);
}

// Forward (INV = false) or inverse (INV = true, exp(+2 pi i k n / N), no
// 1/N) warp FFT, same data layout.  The inverse is the conjugate of the
// forward transform of the conjugate, so one unrolled body serves both
// (the negations fold into the neighbouring additions and stores); the
// kernels are large enough for instruction fetch to matter.
template <int M, bool INV, bool TWG = false>
__device__ __forceinline__ void wfft(float2 (&v)[32], float2* scr, const float2* twT) {
  if (INV) {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i].y = -v[i].y;
  }
  wfft_fwd<M, TWG>(v, scr, twT);
  if (INV) {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i].y = -v[i].y;
  }
}

}  // namespace mmp

// fft.cuh -- FP32 complex FFT building blocks for the demag convolution.
//
// The zero-padded convolution of the paper's magnetostatic field is done
// with our own mixed-radix (2, 3, 4, 8, 16) FFTs: in-register DFT codelets
// and an in-place Stockham autosort pass over a batch of transforms held in
// shared memory.  Forward transforms use exp(-2 pi i k n / L), inverse ones
// exp(+2 pi i k n / L) without the 1/L factor (folded into the kernel
// spectrum).  Twiddles come from per-length tables built in FP64 on the
// host and rounded once.
#pragma once
#include "common.cuh"

namespace mmp {

// L = 16^n16 * 8^n8 * (4 or 2 once) * 3^n3, applied in that order.  (A
// runtime list of radices dispatched in one loop made the compiler keep the
// pass registers in local memory; fixed branches do not.)
struct FftPlan {
  int L;
  int n16, n8, n4, n2, n3;
  int lin;   // every pass takes the uniform-stride addressing (stockham_pass)
};

// Shared-memory layout of a batch of transforms: element i of transform t
// sits at t * fft_pitch(L) + pad(i), pad(i) = i + i/16.  One padding slot
// per 16 complex values (128 bytes, one pass over the 32 banks) turns the
// stride-16 stores of a first radix-16 pass into stride 17, conflict-free;
// the odd pitch staggers the starts of successive transforms.
__host__ __device__ __forceinline__ int fft_pitch(int L) { return L + (L >> 4) + 1; }
__device__ __forceinline__ int fpad(int i) { return i + (i >> 4); }
__device__ __forceinline__ int fidx(int t, int i, int pitch) { return t * pitch + fpad(i); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// multiply by the constant w (forward) or conj(w) (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_w(float2 a, float wr, float wi) {
  return INV ? cmul(a, make_float2(wr, -wi)) : cmul(a, make_float2(wr, wi));
}

// ------------------------------- codelets ---------------------------------
template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  float2 a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = mul_mi<INV>(csub(x1, x3));
  x0 = cadd(a, c);
  x2 = csub(a, c);
  x1 = cadd(b, d);
  x3 = csub(b, d);
}

template <bool INV>
__device__ __forceinline__ void dft3(float2& x0, float2& x1, float2& x2) {
  const float s3 = 0.86602540378443864676f;  // sqrt(3)/2
  float2 t1 = cadd(x1, x2);
  float2 t2 = make_float2(x0.x - 0.5f * t1.x, x0.y - 0.5f * t1.y);
  float2 t3 = mul_mi<INV>(cscale(csub(x1, x2), s3));   // -i sqrt(3)/2 (x1 - x2)
  x0 = cadd(x0, t1);
  x1 = cadd(t2, t3);
  x2 = csub(t2, t3);
}

// radix 8 = 2 x 4 (decimation in time)
template <bool INV>
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
  const float c = 0.70710678118654752440f;
  dft4<INV>(v[0], v[2], v[4], v[6]);   // E_k in v[2k]
  dft4<INV>(v[1], v[3], v[5], v[7]);   // O_k in v[2k+1]
  float2 o1 = mul_w<INV>(v[3], c, -c);
  float2 o2 = mul_mi<INV>(v[5]);
  float2 o3 = mul_w<INV>(v[7], -c, -c);
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}

// radix 16 = 4 x 4: x[4 n1 + n2] -> X[k1 + 4 k2]
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
  const float c8 = 0.92387953251128675613f;   // cos(pi/8)
  const float s8 = 0.38268343236508977173f;   // sin(pi/8)
  const float c4 = 0.70710678118654752440f;   // cos(pi/4)
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
  // v[4 k1 + n2] = Y[n2][k1]; twiddle by w16^(n2 k1)
  v[5] = mul_w<INV>(v[5], c8, -s8);     // n2=1,k1=1: w^1
  v[9] = mul_w<INV>(v[9], c4, -c4);     // n2=1,k1=2: w^2
  v[13] = mul_w<INV>(v[13], s8, -c8);   // n2=1,k1=3: w^3
  v[6] = mul_w<INV>(v[6], c4, -c4);     // n2=2,k1=1: w^2
  v[10] = mul_mi<INV>(v[10]);           // n2=2,k1=2: w^4
  v[14] = mul_w<INV>(v[14], -c4, -c4);  // n2=2,k1=3: w^6
  v[7] = mul_w<INV>(v[7], s8, -c8);     // n2=3,k1=1: w^3
  v[11] = mul_w<INV>(v[11], -c4, -c4);  // n2=3,k1=2: w^6
  v[15] = mul_w<INV>(v[15], -c8, s8);   // n2=3,k1=3: w^9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  // v[4 k1 + k2] = X[k1 + 4 k2]: transpose the 4x4 block
  float2 t;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = a + 1; b < 4; ++b) {
      t = v[4 * a + b];
      v[4 * a + b] = v[4 * b + a];
      v[4 * b + a] = t;
    }
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
  if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 3) dft3<INV>(v[0], v[1], v[2]);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 16) dft16<INV>(v);
}

// ------------------------------ block passes ------------------------------
// Butterflies a thread holds in one pass: CAP complex values in registers
// (CAP = 16 or 32).
template <int R, int CAP>
struct PassCap { static constexpr int B = (R == 3) ? CAP / 3 : CAP / R; };

// One in-place Stockham pass of radix R over `nbatch` transforms of length L
// held in shared memory with the padded layout above.  Ns (the product of
// the radices already applied) is a power of two for every pass of the
// plans used here (the one radix-3 pass comes last on lengths 3*2^a).
// Twiddles of this pass: tw[(r-1) Ns + k] = w_{Ns R}^{r k} (pass-ordered
// table, see pass_twiddles() on the host), so lanes with consecutive k read
// consecutive words.
//
// Addressing: pad(a + b) = pad(a) + pad(b) whenever (a mod 16) + (b mod 16)
// < 16.  So the loads j + r L/R (j < L/R) of a pass sit at
// pad(j) + r * ls, ls = pad(L/R), when L/R is a multiple of 16 (or the whole
// transform is shorter than 16), and the stores o + r Ns (o = (j - k) R + k,
// k < Ns) at pad(o) + r * ss when Ns is a multiple of 16 (ss = pad(Ns)) or a
// power-of-two radix keeps R Ns <= 16 (ss = Ns).  Every pass of the
// power-of-two lengths from 256 up is of that kind: one padded base per
// butterfly and a uniform stride.  Other passes form each index.
// Requires L*nbatch <= (CAP/R)*R*blockDim.x (checked by the host).
template <int R, bool INV, int CAP, bool LIN>
__device__ __forceinline__ void stockham_pass(float2* data, int L, int nbatch, int Ns, const float2* tw) {
  constexpr int MAXB = PassCap<R, CAP>::B;
  const int nbf = L / R;
  const int total = nbf * nbatch;
  const int pitch = fft_pitch(L);
  const int ls = (nbf & 15) == 0 ? fpad(nbf) : nbf;   // used when LIN
  const int ss = (Ns & 15) == 0 ? fpad(Ns) : Ns;
  // t = b / nbf without an integer division: (b + 1/2) / nbf is at least
  // 1/(2 nbf) away from an integer and b, nbf < 2^15, so the FP32 quotient
  // truncates exactly.
  const float rnbf = 1.0f / (float)nbf;
  float2 v[MAXB][R];
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    int b = threadIdx.x + i * blockDim.x;
    if (b < total) {
      int t = (int)(((float)b + 0.5f) * rnbf), j = b - t * nbf;
      const float2* src = data + t * pitch;
      if (LIN) {
        const float2* p = src + fpad(j);
#pragma unroll
        for (int r = 0; r < R; ++r, p += ls) v[i][r] = *p;
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[i][r] = src[fpad(j + r * nbf)];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    int b = threadIdx.x + i * blockDim.x;
    if (b < total) {
      int t = (int)(((float)b + 0.5f) * rnbf), j = b - t * nbf;
      int k = j & (Ns - 1);
      if (Ns > 1) {
        const float2* w = tw + k;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 wr = w[(r - 1) * Ns];
          if (INV) wr.y = -wr.y;
          v[i][r] = cmul(v[i][r], wr);
        }
      }
      dft<R, INV>(v[i]);
      const int o = (j - k) * R + k;
      float2* dst = data + t * pitch;
      if (LIN) {
        float2* p = dst + fpad(o);
#pragma unroll
        for (int r = 0; r < R; ++r, p += ss) *p = v[i][r];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) dst[fpad(o + r * Ns)] = v[i][r];
      }
    }
  }
  __syncthreads();
}

// Full transform of a batch in shared memory (natural order in and out).
// Callers __syncthreads() before (data written) and may read right after.
// `tw` is the pass-ordered twiddle table of the plan (L - 1 entries) in
// shared or global memory.  The addressing variant is chosen once per
// transform (p.lin): mixing both in one pass loop made the compiler keep the
// address offsets of both live and spill.
template <bool INV, int CAP, bool LIN>
__device__ __forceinline__ void block_fft_v(float2* data, const FftPlan p, int nbatch, const float2* tw) {
  int Ns = 1;
#pragma unroll 1
  for (int s = 0; s < p.n16; ++s) {
    stockham_pass<16, INV, CAP, LIN>(data, p.L, nbatch, Ns, tw);
    if (Ns > 1) tw += 15 * Ns;
    Ns *= 16;
  }
#pragma unroll 1
  for (int s = 0; s < p.n8; ++s) {
    stockham_pass<8, INV, CAP, LIN>(data, p.L, nbatch, Ns, tw);
    if (Ns > 1) tw += 7 * Ns;
    Ns *= 8;
  }
  if (p.n4) { stockham_pass<4, INV, CAP, LIN>(data, p.L, nbatch, Ns, tw); if (Ns > 1) tw += 3 * Ns; Ns *= 4; }
  if (p.n2) { stockham_pass<2, INV, CAP, LIN>(data, p.L, nbatch, Ns, tw); if (Ns > 1) tw += Ns; Ns *= 2; }
#pragma unroll 1
  for (int s = 0; s < p.n3; ++s) {
    stockham_pass<3, INV, CAP, LIN>(data, p.L, nbatch, Ns, tw);
    if (Ns > 1) tw += 2 * Ns;
    Ns *= 3;
  }
}

template <bool INV, int CAP = 32>
__device__ __forceinline__ void block_fft(float2* data, const FftPlan p, int nbatch, const float2* tw) {
  if (p.lin) block_fft_v<INV, CAP, true>(data, p, nbatch, tw);
  else block_fft_v<INV, CAP, false>(data, p, nbatch, tw);
}

}  // namespace mmp

// pass_b.cuh -- device body of pass B of the demag convolution, per kx
// plane: the ky residue class r (mod R) of the zero-padded y transform as a
// folded length-Py/R FFT, the z transform + 3x3 symmetric demag-kernel
// multiply + inverse z transform in registers, the inverse y FFT, and the
// recombination of the R classes through distributed shared memory of an
// R-CTA thread-block cluster (only y < ny is formed).  Used by the
// per-context kernel (pass_b.cu, clusters of R CTAs) and the batched stage
// kernel (batch.cu, R = 1).
//
// Shared memory per CTA: the 3 nz columns (padded FFT layout), the
// Stockham twiddles of length Py/R, for R > 1 the fold and recombination
// twiddles of this residue class, and optionally this CTA's slice of the
// kernel octant.
#pragma once
#include <cooperative_groups.h>
#include "kernels.h"
#include "copy.cuh"

namespace mmp {

namespace cg = cooperative_groups;

// 3x3 symmetric kernel times a complex 3-vector.  K points at the six
// components (xx, yy, zz, xy, xz, yz) of octant entry (|ky|, |kz|); sy, sz
// flip the components odd in ky, kz.
// KG: K is in global memory (read-only: non-coherent loads that need not wait
// for earlier shared-memory stores); else in shared memory.
template <bool KG>
__device__ __forceinline__ void kmul(const float* K, float sy, float sz, float2& a, float2& b, float2& c) {
  const float2* K2 = reinterpret_cast<const float2*>(K);
  const float2 k01 = KG ? __ldg(K2) : K2[0];
  const float2 k23 = KG ? __ldg(K2 + 1) : K2[1];
  const float2 k45 = KG ? __ldg(K2 + 2) : K2[2];
  float xx = k01.x, yy = k01.y, zz = k23.x, xy = k23.y * sy, xz = k45.x * sz, yz = k45.y * sy * sz;
  float2 ha = make_float2(xx * a.x + xy * b.x + xz * c.x, xx * a.y + xy * b.y + xz * c.y);
  float2 hb = make_float2(xy * a.x + yy * b.x + yz * c.x, xy * a.y + yy * b.y + yz * c.y);
  float2 hc = make_float2(xz * a.x + yz * b.x + zz * c.x, xz * a.y + yz * b.y + zz * c.y);
  a = ha; b = hb; c = hc;
}

template <int N, bool INV>
__device__ __forceinline__ void dft_small(float2 (&f)[N]) {
  if constexpr (N == 2) dft2<INV>(f[0], f[1]);
  else if constexpr (N == 4) dft4<INV>(f[0], f[1], f[2], f[3]);
  else dft8<INV>(f);
}

// nz = 1: the kernel multiply alone, one thread per column.
template <bool KG>
__device__ __forceinline__ void zkz_single(float2* W, int pitch, int kp, const float* Kc, float sy) {
  float2 a = W[fidx(0, kp, pitch)], b = W[fidx(1, kp, pitch)], c = W[fidx(2, kp, pitch)];
  kmul<KG>(Kc, sy, 1.0f, a, b, c);
  W[fidx(0, kp, pitch)] = a; W[fidx(1, kp, pitch)] = b; W[fidx(2, kp, pitch)] = c;
}

// nz = NZ in {2, 4, 8} (Pz = 2 NZ): two lanes per ky column, lane parity
// `par` handles kz of that parity:  F[2q+par] = DFT_NZ(v[z] w^(par z))[q],
// multiply, inverse DFT_NZ, times w^(-par z); the two lanes add their halves
// through a shuffle and each writes NZ/2 of the z outputs.  Both lanes read
// the column before the shuffle, so neither writes before the other read.
template <int NZ, bool KG>
__device__ __forceinline__ void zkz_pair(float2* W, int pitch, int kp, bool valid, int par, const float* Kc,
                                         float sy, const float2* __restrict__ twz) {
  float2 f[3][NZ];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int z = 0; z < NZ; ++z) {
      float2 v = valid ? W[fidx(c * NZ + z, kp, pitch)] : make_float2(0.0f, 0.0f);
      f[c][z] = par ? cmul(v, __ldg(twz + z)) : v;
    }
#pragma unroll
  for (int c = 0; c < 3; ++c) dft_small<NZ, false>(f[c]);
#pragma unroll
  for (int q = 0; q < NZ; ++q) {
    int kz = 2 * q + par;
    int ikz = kz <= NZ ? kz : 2 * NZ - kz;
    float sz = kz <= NZ ? 1.0f : -1.0f;
    kmul<KG>(Kc + ikz * 6, sy, sz, f[0][q], f[1][q], f[2][q]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) dft_small<NZ, true>(f[c]);
  if (par) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int z = 0; z < NZ; ++z) f[c][z] = cmul(f[c][z], cconj(__ldg(twz + z)));
  }
  constexpr int H = NZ / 2;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int z = 0; z < H; ++z) {
      float2 send = par ? f[c][z] : f[c][z + H];
      float2 keep = par ? f[c][z + H] : f[c][z];
      float2 recv;
      recv.x = __shfl_xor_sync(0xffffffffu, send.x, 1);
      recv.y = __shfl_xor_sync(0xffffffffu, send.y, 1);
      if (valid) W[fidx(c * NZ + z + (par ? H : 0), kp, pitch)] = cadd(keep, recv);
    }
}

// Any nz <= 16: direct DFT over the padded length Pz, one thread per column.
template <bool KG>
static __device__ void zkz_generic(float2* W, int kp, int pitch, int nz, int Pz, const float* Kc, float sy,
                            const float2* __restrict__ twz) {
  float2 out[3][16];
  for (int c = 0; c < 3; ++c)
    for (int zz = 0; zz < 16; ++zz) out[c][zz] = make_float2(0.0f, 0.0f);
  for (int kz = 0; kz < Pz; ++kz) {
    float2 F[3];
    for (int c = 0; c < 3; ++c) {
      float2 acc = make_float2(0.0f, 0.0f);
      for (int zz = 0; zz < nz; ++zz)
        acc = cadd(acc, cmul(W[fidx(c * nz + zz, kp, pitch)], __ldg(twz + (kz * zz) % Pz)));
      F[c] = acc;
    }
    int ikz = kz <= Pz / 2 ? kz : Pz - kz;
    float sz = kz <= Pz / 2 ? 1.0f : -1.0f;
    kmul<KG>(Kc + ikz * 6, sy, sz, F[0], F[1], F[2]);
    for (int zz = 0; zz < nz; ++zz) {
      float2 w = cconj(__ldg(twz + (kz * zz) % Pz));
      for (int c = 0; c < 3; ++c) out[c][zz] = cadd(out[c][zz], cmul(F[c], w));
    }
  }
  for (int c = 0; c < 3; ++c)
    for (int zz = 0; zz < nz; ++zz) W[fidx(c * nz + zz, kp, pitch)] = out[c][zz];
}

// Pass B of plane kx, residue class r of R (the cluster rank; R = d.R).
// KS: the kernel rows of the plane are staged in shared memory with
// cp.async while the fold and the forward FFT run; otherwise the z
// transforms read them from global memory (L2).
template <int NZ, bool KS>
__device__ __forceinline__ void passB_plane(unsigned char* sraw, const Grid& g, const DemagArgs& d, int kx, int r) {
  const int R = d.R;                 // cluster size = residue classes of ky
  const int ny = g.ny, nz = g.nz, Py = g.Py, kzn = g.kzn;
  const int Ly = Py / R;
  const int pitch = fft_pitch(Ly);
  const int ncol = 3 * nz;
  const PassBSmem L = passb_smem(ny, nz, Py, kzn, R, KS);
  float2* W = reinterpret_cast<float2*>(sraw);
  float2* twl = reinterpret_cast<float2*>(sraw + L.twl);
  float2* twf = reinterpret_cast<float2*>(sraw + L.twf);
  float2* twc = reinterpret_cast<float2*>(sraw + L.twc);
  float* Ks = reinterpret_cast<float*>(sraw + L.ks);
  float2* Tk = d.T + (long long)kx * ncol * ny;

  // 0a. when ny <= Ly the fold has one term: the plane's rows go straight
  // into the columns, as asynchronous 8-byte copies (all in flight at once,
  // no registers held); issued before the kernel rows so that waiting for
  // them leaves the kernel rows in flight
  const bool one_term = ny <= Ly;
  if (one_term) {
    const float rny = 1.0f / (float)ny;   // e / ny by the exact FP32 quotient (e < 2^22)
    for (int e = threadIdx.x; e < ncol * ny; e += blockDim.x) {
      const int col = (int)(((float)e + 0.5f) * rny), j = e - col * ny;
      if (MMP_IN(g, (long long)kx * ncol * ny + e, g.lim_T)) cp_async8(W + fidx(col, j, pitch), Tk + e);
    }
    cp_async_commit();
  }
  // 0. prefetch this CTA's kernel rows (|ky| of ky = R k' + r) asynchronously
  const int krow = g.krow;
  const float* kbase = d.khat + (long long)kx * g.kyn * krow;
  if (KS) {
    for (int kp = threadIdx.x; kp < Ly; kp += blockDim.x) {
      int ky = R * kp + r;
      int iky = ky <= Py / 2 ? ky : Py - ky;
      const float4* src = reinterpret_cast<const float4*>(kbase + (long long)iky * krow);
      float4* dst = reinterpret_cast<float4*>(Ks + kp * krow);
      if (!MMP_IN(g, ((long long)kx * g.kyn + iky) * krow + krow - 1, g.lim_khat)) continue;
      for (int w = 0; w < (krow >> 2); ++w) cp_async16(dst + w, src + w);
    }
    cp_async_commit();
  }
  // 1. twiddles: Stockham (pass-ordered, length Ly), fold w^(r j), recombination w^y
  const int ylo = (int)((long long)ny * r / R), yhi = (int)((long long)ny * (r + 1) / R);
  const int cnt = yhi - ylo;
  for (int i = threadIdx.x; i < Ly; i += blockDim.x) twl[i] = __ldg(d.tw_ly + i);
  if (R > 1) {
    for (int i = threadIdx.x; i < Ly; i += blockDim.x) twf[i] = __ldg(d.tw_y + r * i);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) twc[i] = __ldg(d.tw_y + ylo + i);
  }
  __syncthreads();
  // 2. fold the ky residue class r: g_r[j] = w^(r j) sum_q T[j + q Ly] w_R^(r q).
  if (one_term) {
    // rows ny .. Ly-1 of the zero padding, then g_r[j] = w^(r j) T[j]
    for (int e = threadIdx.x; e < ncol * (Ly - ny); e += blockDim.x) {
      const int col = e / (Ly - ny), j = ny + e - col * (Ly - ny);
      W[fidx(col, j, pitch)] = make_float2(0.0f, 0.0f);
    }
    if (KS) cp_async_wait_one();
    else cp_async_wait_all();
    __syncthreads();
    if (r > 0) {
      const float rny = 1.0f / (float)ny;
      for (int e = threadIdx.x; e < ncol * ny; e += blockDim.x) {
        const int col = (int)(((float)e + 0.5f) * rny), j = e - col * ny;
        float2* p = W + fidx(col, j, pitch);
        *p = cmul(*p, twf[j]);
      }
    }
  }
  // Otherwise four columns per step keep several independent loads in flight.
  for (int col0 = 0; col0 < (one_term ? 0 : ncol); col0 += 4) {
    for (int j = threadIdx.x; j < Ly; j += blockDim.x) {
      float2 acc[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        acc[u] = (col0 + u < ncol && j < ny &&
                  MMP_IN(g, (long long)kx * ncol * ny + (long long)(col0 + u) * ny + j, g.lim_T))
                     ? __ldcg(Tk + (long long)(col0 + u) * ny + j)
                     : make_float2(0.0f, 0.0f);
      int tq = 0;
      for (int y = j + Ly; y < ny; y += Ly) {
        tq += r;
        if (tq >= R) tq -= R;
        const float2 ph = __ldg(d.tw_y + tq * Ly);
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          v[u] = col0 + u < ncol && MMP_IN(g, (long long)kx * ncol * ny + (long long)(col0 + u) * ny + y, g.lim_T)
                     ? __ldcg(Tk + (long long)(col0 + u) * ny + y)
                     : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = cadd(acc[u], cmul(v[u], ph));
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (col0 + u < ncol) W[fidx(col0 + u, j, pitch)] = r > 0 ? cmul(acc[u], twf[j]) : acc[u];
    }
  }
  __syncthreads();
  // columns per transform call: what the block holds -- all of them on the
  // per-context path; a larger plane (batched path) in two chunks, which the
  // host guarantees suffice.  Two straight-line calls: a loop around the FFT
  // body makes the compiler cut the registers and spill.
  const int c1 = min(ncol, max(1, (d.plan_ly.n3 ? 30 : 32) * (int)blockDim.x / Ly));
  block_fft<false>(W, d.plan_ly, c1, twl);
  if (ncol > c1) block_fft<false>(W + c1 * pitch, d.plan_ly, ncol - c1, twl);
  if (KS) cp_async_wait_all();
  __syncthreads();
  const float* Kb = KS ? Ks : kbase;   // row of ky' = R k' + r at Kb + (KS ? k' : |ky|) krow
  // 3. z transform + kernel multiply + inverse z transform per ky column
  if constexpr (NZ == 1) {
    for (int kp = threadIdx.x; kp < Ly; kp += blockDim.x) {
      int ky = R * kp + r;
      int iky = ky <= Py / 2 ? ky : Py - ky;
      if (!KS && !MMP_IN(g, ((long long)kx * g.kyn + iky) * krow + krow - 1, g.lim_khat)) iky = 0;
      zkz_single<!KS>(W, pitch, kp, Kb + (long long)(KS ? kp : iky) * krow, ky <= Py / 2 ? 1.0f : -1.0f);
    }
  } else if constexpr (NZ > 1) {
    const int half = blockDim.x >> 1;
    for (int base = 0; base < Ly; base += half) {
      int kp = base + (threadIdx.x >> 1);
      bool valid = kp < Ly;
      int ky = valid ? R * kp + r : r;
      int iky = ky <= Py / 2 ? ky : Py - ky;
      if (!KS && !MMP_IN(g, ((long long)kx * g.kyn + iky) * krow + krow - 1, g.lim_khat)) iky = 0;
      zkz_pair<NZ, !KS>(W, pitch, valid ? kp : 0, valid, threadIdx.x & 1,
                   Kb + (long long)(KS ? (valid ? kp : 0) : iky) * krow, ky <= Py / 2 ? 1.0f : -1.0f, d.tw_z);
    }
  } else {
    for (int kp = threadIdx.x; kp < Ly; kp += blockDim.x) {
      int ky = R * kp + r;
      int iky = ky <= Py / 2 ? ky : Py - ky;
      if (!KS && !MMP_IN(g, ((long long)kx * g.kyn + iky) * krow + krow - 1, g.lim_khat)) iky = 0;
      zkz_generic<!KS>(W, kp, pitch, nz, g.Pz, Kb + (long long)(KS ? kp : iky) * krow, ky <= Py / 2 ? 1.0f : -1.0f,
                  d.tw_z);
    }
  }
  __syncthreads();
  block_fft<true>(W, d.plan_ly, c1, twl);
  if (ncol > c1) block_fft<true>(W + c1 * pitch, d.plan_ly, ncol - c1, twl);
  // 4. recombine: out[y] = sum_q w^(-q y) h_q[y mod Ly], y < ny
  if (R == 1) {
    for (int e = threadIdx.x; e < ncol * ny; e += blockDim.x) {
      int col = e / ny, y = e - col * ny;
      if (MMP_IN(g, (long long)kx * ncol * ny + e, g.lim_T)) Tk[e] = W[fidx(col, y, pitch)];
    }
  } else {
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    for (int col0 = 0; col0 < ncol; col0 += 4) {
      for (int yi = threadIdx.x; yi < cnt; yi += blockDim.x) {
        const int y = ylo + yi;
        int j = y;
        while (j >= Ly) j -= Ly;
        const float2 w1 = cconj(twc[yi]);   // w^(-y)
        float2 acc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float2* W0 = cl.map_shared_rank(W, 0);
          acc[u] = col0 + u < ncol ? W0[fidx(col0 + u, j, pitch)] : make_float2(0.0f, 0.0f);
        }
        float2 wq = w1;
        for (int q = 1; q < R; ++q) {
          float2 v[4];
          const float2* Wr = cl.map_shared_rank(W, q);
#pragma unroll
          for (int u = 0; u < 4; ++u)
            v[u] = col0 + u < ncol ? Wr[fidx(col0 + u, j, pitch)] : make_float2(0.0f, 0.0f);
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[u] = cadd(acc[u], cmul(v[u], wq));
          wq = cmul(wq, w1);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (col0 + u < ncol && MMP_IN(g, (long long)kx * ncol * ny + (long long)(col0 + u) * ny + y, g.lim_T))
            Tk[(long long)(col0 + u) * ny + y] = acc[u];
      }
    }
    cl.sync();
  }
}

}  // namespace mmp

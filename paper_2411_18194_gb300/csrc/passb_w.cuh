// passb_w.cuh -- pass B of the demag convolution on the warp FFT engine
// (wfft.cuh), for planes whose folded y length Ly = Py / R is 32 M
// (M = 8, 16, 32), with ny <= Ly (the fold has one term) and R = 1 or 2.
//
// One CTA (or one CTA of an R = 2 cluster) handles one kx plane of the
// spectrum T[kx][c][z][y] (3 nz columns of ny values) for its ky residue
// class r:
//   0. the plane is copied into shared memory W[col][y] with asynchronous
//      16-byte copies (rows ny..Ly-1 zero), and this CTA's half of the
//      kernel rows of the plane is prefetched into L2;
//   1. forward y transform of every column (the class twiddle w_Py^(r y) on
//      the way from W into registers), one warp per column group, result
//      back in W[col][ky'];
//   2. per ky' = (ky - r) / R, one thread: the z transform (padded length
//      2 nz, as its even and odd halves), the 3x3 symmetric demag-kernel
//      multiply of every kz, and the inverse z transform, in registers, the
//      z twiddles compile-time constants;
//   3. inverse y transform of every column; with R = 1 the y < ny outputs go
//      to T, with R = 2 (times w_Py^(-r y)) to W;
//   4. (R = 2) the two classes are added through distributed shared memory,
//      each CTA writing half of the y range of T.
#pragma once
#include <cooperative_groups.h>
#include "kernels.h"
#include "wfft.cuh"
#include "copy.cuh"
#include "tcdft.cuh"

namespace mmp {

// Layout of the warp pass B's shared memory: the W columns at pitch
// passb_w_pitch (a group of B = 32 / M columns spans at least the 1024
// float2 of its warp's transpose scratch; the 8-float2 skew of B > 1 keeps
// the columns of a group on different banks), then the warp twiddle table
// (32 M float2).
__host__ __device__ __forceinline__ int passb_w_pitch(int M) { return 32 * M + (M < 32 ? 8 : 0); }
__host__ __device__ __forceinline__ int passb_w_groups(int nz, int M) { return (3 * nz + 32 / M - 1) / (32 / M); }
__host__ __device__ __forceinline__ size_t passb_w_smem(int nz, int M, bool tc = false) {
  return ((size_t)passb_w_groups(nz, M) * (32 / M) * passb_w_pitch(M) + 32 * M) * sizeof(float2) +
         (tc ? (size_t)4 * kTcB * sizeof(float) + 64 : 0);
}
// Warps per CTA of the warp pass B: 12 when there are at least 12 column
// groups (two per warp at nz = 8, Ly = 1024), else 8.
__host__ __device__ constexpr int passb_w_warps(int nz, int M) {
  return (3 * nz + 32 / M - 1) / (32 / M) >= 12 ? 12 : 8;
}

// K: octant entry (xx, yy, zz, xy, xz, yz) as three float2; sy, sz: signs of
// the components odd in ky, kz.
__device__ __forceinline__ void kmul3(float2 k01, float2 k23, float2 k45, float sy, float sz, float2& a,
                                      float2& b, float2& c) {
  const float xx = k01.x, yy = k01.y, zz = k23.x, xy = k23.y * sy, xz = k45.x * sz, yz = k45.y * (sy * sz);
  const float2 ha = make_float2(fmaf(xx, a.x, fmaf(xy, b.x, xz * c.x)), fmaf(xx, a.y, fmaf(xy, b.y, xz * c.y)));
  const float2 hb = make_float2(fmaf(xy, a.x, fmaf(yy, b.x, yz * c.x)), fmaf(xy, a.y, fmaf(yy, b.y, yz * c.y)));
  const float2 hc = make_float2(fmaf(xz, a.x, fmaf(yz, b.x, zz * c.x)), fmaf(xz, a.y, fmaf(yz, b.y, zz * c.y)));
  a = ha;
  b = hb;
  c = hc;
}

// Kernel row of one ky column from global memory (read-only path), loaded
// whole with 16-byte loads (rows are krow = 6 kzn rounded up to 4 floats,
// 16-byte aligned) before the z transforms start.
template <int NZ>
struct RowsGlobal {
  static constexpr int KQ = (6 * (NZ + 1) + 3) / 4;   // float4 per row (kzn = NZ + 1)
  float4 q[KQ];
  __device__ __forceinline__ explicit RowsGlobal(const float* row) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
    for (int j = 0; j < KQ; ++j) q[j] = __ldg(r4 + j);
  }
  __device__ __forceinline__ float at(int i) const {   // compile-time i after unrolling
    const float4& v = q[i >> 2];
    return (i & 3) == 0 ? v.x : (i & 3) == 1 ? v.y : (i & 3) == 2 ? v.z : v.w;
  }
  __device__ __forceinline__ float2 pair(int kz, int u) const { return make_float2(at(6 * kz + 2 * u), at(6 * kz + 2 * u + 1)); }
  template <int N0>
  __device__ __forceinline__ void even(float2 (&k)[N0][3]) const {
#pragma unroll
    for (int i = 0; i < N0; ++i)
#pragma unroll
      for (int u = 0; u < 3; ++u) k[i][u] = pair(2 * i, u);
  }
  template <int N1>
  __device__ __forceinline__ void odd(float2 (&k)[N1][3]) const {
#pragma unroll
    for (int i = 0; i < N1; ++i)
#pragma unroll
      for (int u = 0; u < 3; ++u) k[i][u] = pair(2 * i + 1, u);
  }
};
// z stage of one ky column for NZ in {1, 2, 4, 8} (Pz = 2 NZ, or 1 when
// NZ = 1).  W column c*NZ+z at W + (c NZ + z) * LP, element kp.
//   F[2q + p] = DFT_NZ(x[z] w_Pz^(p z))[q],  x[z] = sum_p w_Pz^(-p z) IDFT_NZ(F[2q + p])[z]
// The kernel rows of a parity are fetched before its transforms, so that
// their latency overlaps the arithmetic.
template <int NZ, typename Rows>
__device__ __forceinline__ void zstage_w(float2* W, int LP, int kp, const Rows& rows, float sy) {
  if constexpr (NZ == 1) {
    float2 k[1][3];
    rows.even(k);
    float2 a = W[kp], b = W[LP + kp], c = W[2 * LP + kp];
    kmul3(k[0][0], k[0][1], k[0][2], sy, 1.0f, a, b, c);
    W[kp] = a;
    W[LP + kp] = b;
    W[2 * LP + kp] = c;
  } else {
    constexpr int P = 2 * NZ;           // padded z length
    constexpr int TS = 32 / P;          // w_P^z = w32^(TS z)
    constexpr int NR0 = NZ / 2 + 1;     // distinct rows |kz| of the even kz: 0, 2, .., NZ
    constexpr int NR1 = NZ / 2;         // of the odd kz: 1, 3, .., NZ - 1
    float2 out[3][NZ];
    float2 kr0[NR0][3];
    rows.even(kr0);
    {
      float2 f[3][NZ];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int z = 0; z < NZ; ++z) f[c][z] = W[(c * NZ + z) * LP + kp];
#pragma unroll
      for (int c = 0; c < 3; ++c) dft_m<NZ, false>(f[c]);
#pragma unroll
      for (int q = 0; q < NZ; ++q) {
        const int kz = 2 * q;                       // compile-time after unrolling
        const int i = (kz <= NZ ? kz : P - kz) / 2;
        kmul3(kr0[i][0], kr0[i][1], kr0[i][2], sy, kz <= NZ ? 1.0f : -1.0f, f[0][q], f[1][q], f[2][q]);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) dft_m<NZ, true>(f[c]);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int z = 0; z < NZ; ++z) out[c][z] = f[c][z];
    }
    float2 kr1[NR1][3];
    rows.odd(kr1);
    {
      float2 f[3][NZ];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int z = 0; z < NZ; ++z) f[c][z] = W[(c * NZ + z) * LP + kp];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        f[c][1] = mul_w32<TS * 1, false>(f[c][1]);
        if constexpr (NZ > 2) {
          f[c][2] = mul_w32<TS * 2, false>(f[c][2]);
          f[c][3] = mul_w32<TS * 3, false>(f[c][3]);
        }
        if constexpr (NZ > 4) {
          f[c][4] = mul_w32<TS * 4, false>(f[c][4]);
          f[c][5] = mul_w32<TS * 5, false>(f[c][5]);
          f[c][6] = mul_w32<TS * 6, false>(f[c][6]);
          f[c][7] = mul_w32<TS * 7, false>(f[c][7]);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) dft_m<NZ, false>(f[c]);
#pragma unroll
      for (int q = 0; q < NZ; ++q) {
        const int kz = 2 * q + 1;
        const int i = ((kz <= NZ ? kz : P - kz) - 1) / 2;
        kmul3(kr1[i][0], kr1[i][1], kr1[i][2], sy, kz <= NZ ? 1.0f : -1.0f, f[0][q], f[1][q], f[2][q]);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) dft_m<NZ, true>(f[c]);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        out[c][0] = cadd(out[c][0], f[c][0]);
        out[c][1] = cadd(out[c][1], mul_w32<TS * 1, true>(f[c][1]));
        if constexpr (NZ > 2) {
          out[c][2] = cadd(out[c][2], mul_w32<TS * 2, true>(f[c][2]));
          out[c][3] = cadd(out[c][3], mul_w32<TS * 3, true>(f[c][3]));
        }
        if constexpr (NZ > 4) {
          out[c][4] = cadd(out[c][4], mul_w32<TS * 4, true>(f[c][4]));
          out[c][5] = cadd(out[c][5], mul_w32<TS * 5, true>(f[c][5]));
          out[c][6] = cadd(out[c][6], mul_w32<TS * 6, true>(f[c][6]));
          out[c][7] = cadd(out[c][7], mul_w32<TS * 7, true>(f[c][7]));
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int z = 0; z < NZ; ++z) W[(c * NZ + z) * LP + kp] = out[c][z];
  }
}

// L2 prefetch, by one thread, of this class's share of the kernel rows of
// the plane (class r of R takes the r-th part of the |ky| rows).
__device__ __forceinline__ void prefetch_rows_l2(const float* kplane, const Grid& g, int R, int r) {
  const int lo = (g.kyn * r) / R, hi = (g.kyn * (r + 1)) / R;
  const char* p = reinterpret_cast<const char*>(kplane + (long long)lo * g.krow);
  for (long long bytes = (long long)(hi - lo) * g.krow * 4; bytes > 0; bytes -= 65536, p += 65536)
    prefetch_l2(p, (unsigned)(bytes < 65536 ? bytes : 65536));
}

// The y transform of one column group: on the warp FFT alone, or (TC) with
// its stage 1 (the in-register DFT32) as a split-TF32 GEMM on the tensor
// cores for the whole warpgroup (tcdft.cuh).  The inverse is the conjugate
// of the forward transform of the conjugate.
struct TcCtx {
  uint32_t tbase;   // the CTA's tensor memory
  const float* Bs;  // the DFT32 matrices (shared memory)
  uint64_t* mbar;   // per warpgroup
  uint32_t phase;   // this thread's next phase parity of its warpgroup's mbarrier
  unsigned* err;
};
// `valid` = false: a warp without a column this round (only with TC, where
// all four warps of a warpgroup take part in its GEMM): it contributes zeros
// and its results are not used.
template <int M, bool INV, bool TC>
__device__ __forceinline__ void ytransform(float2 (&v)[32], float2* scr, const float2* twT, TcCtx& tc,
                                           bool valid) {
  if constexpr (!TC) {
    wfft<M, INV>(v, scr, twT);
  } else {
    if (valid) {
      if (INV) {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i].y = -v[i].y;
      }
      wfft_head<M>(v, scr, twT);
    }
    const int g = threadIdx.x >> 7;
    tc_stage32(v, tc.tbase, g * kTcCols, tc.Bs, tc.mbar + g, tc.phase, tc.err);
    if (INV) {
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i].y = -v[i].y;
    }
  }
}

// Pass B of plane kx, class r, on NW warps.  M = Ly / 32.  TC: the final
// DFT32 of every y transform on the tensor cores (whole warpgroups).
template <int NZ, int M, int NW, bool TC = false>
__device__ __forceinline__ void passB_w_plane(unsigned char* sraw, const Grid& g, const DemagArgs& d, int kx,
                                              int r) {
  constexpr int Ly = 32 * M;
  constexpr int B = 32 / M;              // columns per warp transform
  constexpr int NCOL = 3 * NZ;
  constexpr int NGRP = (NCOL + B - 1) / B;
  constexpr int LP = 32 * M + (M < 32 ? 8 : 0);   // passb_w_pitch(M)
  constexpr int NT = NW * 32;
  const int R = d.R;
  const int ny = g.ny, Py = g.Py;
  static_assert(!TC || (NW % 4 == 0 && (NW / 4) * kTcCols <= 512), "tensor-core stage: whole warpgroups");
  constexpr int NRND = (NGRP + NW - 1) / NW;   // column rounds (every warp takes part in each with TC)
  float2* W = reinterpret_cast<float2*>(sraw);
  float2* twT = W + NGRP * B * LP;
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  float2* Tk = d.T + (long long)kx * NCOL * ny;
  TcCtx tc{0u, nullptr, nullptr, 0u, d.err};
  if constexpr (TC) {
    float* Bs = reinterpret_cast<float*>(twT + 32 * M);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(Bs + 4 * kTcB);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 4);
    for (int i = threadIdx.x; i < 4 * kTcB; i += NT) Bs[i] = __ldg(d.tw_tc + i);
    if (threadIdx.x < NW / 4) mbar_init(mbar + threadIdx.x, 1);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    if (warp == 0) tmem_alloc(tslot, 512);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    tc.tbase = *tslot;
    tc.Bs = Bs;
    tc.mbar = mbar;
  }
  // 0. the plane into W (asynchronous copies), the zero rows, L2 prefetch of
  // the kernel rows, the warp twiddles
  if ((ny & 1) == 0) {
    const int q = ny >> 1;                 // 16-byte pieces per column
    const float rq = 1.0f / (float)q;      // e / q by the exact FP32 quotient (e < 2^22)
    for (int e = threadIdx.x; e < NCOL * q; e += NT) {
      const int col = (int)(((float)e + 0.5f) * rq), j = e - col * q;
      const long long ti = (long long)kx * NCOL * ny + (long long)col * ny + 2 * j;
      if (MMP_IN(g, ti + 1, g.lim_T)) cp_async16(W + col * LP + 2 * j, Tk + (long long)col * ny + 2 * j);
    }
  } else {
    const float rny = 1.0f / (float)ny;
    for (int e = threadIdx.x; e < NCOL * ny; e += NT) {
      const int col = (int)(((float)e + 0.5f) * rny), j = e - col * ny;
      if (MMP_IN(g, (long long)kx * NCOL * ny + e, g.lim_T)) cp_async8(W + col * LP + j, Tk + e);
    }
  }
  cp_async_commit();
  if (ny < Ly) {
    const int nz0 = Ly - ny;
    for (int e = threadIdx.x; e < NCOL * nz0; e += NT) {
      const int col = e / nz0, j = ny + e - col * nz0;
      W[col * LP + j] = make_float2(0.0f, 0.0f);
    }
  }
  const float* kbase = d.khat + (long long)kx * g.kyn * g.krow;
  if (threadIdx.x == 0) prefetch_rows_l2(kbase, g, R, r);
  for (int i = threadIdx.x; i < 32 * M; i += NT) twT[i] = __ldg(d.tw_wy + i);
  cp_async_wait_all();
  __syncthreads();
  // 1. forward y transforms: lane l takes y = l + 32 m of each column of its group
  for (int rnd = 0; rnd < NRND; ++rnd) {
    const int grp = warp + rnd * NW;
    const bool valid = grp < NGRP;
    if (!TC && !valid) break;
    float2 v[32];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int col = grp * B + b;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int y = lane + 32 * m;
        float2 x = valid && col < NCOL ? W[col * LP + y] : make_float2(0.0f, 0.0f);
        if (r) x = cmul(x, __ldg(d.tw_y + r * y));
        v[b * M + m] = x;
      }
    }
    __syncwarp();
    // the transpose scratch: this group's own columns of W (B LP >= 1024 float2)
    float2* scr = W + grp * B * LP;
    ytransform<M, false, TC>(v, scr, twT, tc, valid);
    // lane j: column grp B + j / M, ky' = j mod M + M k2
    const int col = grp * B + lane / M, k1 = lane % M;
    if (valid && col < NCOL) {
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) W[col * LP + k1 + M * k2] = v[k2];
    }
    __syncwarp();
  }
  __syncthreads();
  // 2. z stage per ky'.  ky and its mirror Py - ky use the same kernel row
  // (|ky|, the odd components changing sign), so a thread takes such a pair
  // with one row load: kp and Ly - kp in class 0 (kp = 0 and Ly / 2 are
  // their own mirrors), kp and Ly - 1 - kp in class 1.  The first NT pairs
  // go one to a thread, the rest are split into single columns, so that no
  // thread takes more columns than with one column per thread and round.
  // (Loading a pair's row before the forward transforms, to hide its
  // latency, measured slower: its 56 registers spill.)
  {
    const int npair = r ? Ly / 2 : Ly / 2 - 1;
    const int pa = npair < NT ? npair : NT;
    if (threadIdx.x < pa) {
      const int kp = r ? threadIdx.x : threadIdx.x + 1, km = (r ? Ly - 1 : Ly) - kp;
      const int ky = R * kp + r;   // <= Py / 2: its mirror R km + r = Py - ky is above
      const long long ki = ((long long)kx * g.kyn + ky) * g.krow;
      const RowsGlobal<NZ> rows(kbase + (MMP_IN(g, ki + g.krow - 1, g.lim_khat) ? (long long)ky * g.krow : 0));
      zstage_w<NZ>(W, LP, kp, rows, 1.0f);
      zstage_w<NZ>(W, LP, km, rows, -1.0f);
    }
    const int nrest = 2 * (npair - pa) + (r ? 0 : 2);
    for (int v = threadIdx.x; v < nrest; v += NT) {
      int kp;
      if (v < 2 * (npair - pa)) {
        const int u = pa + (v >> 1), k0 = r ? u : u + 1;
        kp = (v & 1) ? (r ? Ly - 1 : Ly) - k0 : k0;
      } else {
        kp = v == 2 * (npair - pa) ? 0 : Ly / 2;
      }
      const int ky = R * kp + r;
      const int iky = ky <= Py / 2 ? ky : Py - ky;
      const long long ki = ((long long)kx * g.kyn + iky) * g.krow;
      const RowsGlobal<NZ> rows(kbase + (MMP_IN(g, ki + g.krow - 1, g.lim_khat) ? (long long)iky * g.krow : 0));
      zstage_w<NZ>(W, LP, kp, rows, ky <= Py / 2 ? 1.0f : -1.0f);
    }
  }
  __syncthreads();
  // 3. inverse y transforms
  for (int rnd = 0; rnd < NRND; ++rnd) {
    const int grp = warp + rnd * NW;
    const bool valid = grp < NGRP;
    if (!TC && !valid) break;
    float2 v[32];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int col = grp * B + b;
#pragma unroll
      for (int m = 0; m < M; ++m)
        v[b * M + m] = valid && col < NCOL ? W[col * LP + lane + 32 * m] : make_float2(0.0f, 0.0f);
    }
    __syncwarp();
    float2* scr = W + grp * B * LP;
    ytransform<M, true, TC>(v, scr, twT, tc, valid);
    const int col = grp * B + lane / M, k1 = lane % M;
    if (valid && col < NCOL) {
      if (R == 1) {
#pragma unroll
        for (int k2 = 0; k2 < 32; ++k2) {
          const int y = k1 + M * k2;
          if (y < ny && MMP_IN(g, (long long)kx * NCOL * ny + (long long)col * ny + y, g.lim_T))
            Tk[(long long)col * ny + y] = v[k2];
        }
      } else {
#pragma unroll
        for (int k2 = 0; k2 < 32; ++k2) {
          const int y = k1 + M * k2;
          float2 h = v[k2];
          if (r) h = cmul(h, cconj(__ldg(d.tw_y + r * y)));
          W[col * LP + y] = h;
        }
      }
    }
    __syncwarp();
  }
  if constexpr (TC) {
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (warp == 0) tmem_free(tc.tbase, 512);
  }
  // 4. R = 2: out[y] = h_0[y] + w^(-y) h_1[y], y < ny; this CTA writes its
  // half of y.  Four pairs of values per thread and step, all loads first.
  if (R == 2) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    const float2* Wo = cl.map_shared_rank(W, r ^ 1);
    const int ylo = (ny * r) >> 1, yhi = (ny * (r + 1)) >> 1, cnt = yhi - ylo;
    if ((ylo & 1) == 0 && (cnt & 1) == 0) {
      const int cp = cnt >> 1;               // pairs per column
      const float rcp = 1.0f / (float)cp;    // exact FP32 quotients (e < 2^22)
      constexpr int U = 4;
      for (int e0 = threadIdx.x; e0 < NCOL * cp; e0 += U * NT) {
        float4 a[U], b[U];
        int off[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = e0 + u * NT;
          const int col = (int)(((float)e + 0.5f) * rcp), y = ylo + 2 * (e - col * cp);
          off[u] = e < NCOL * cp ? col * LP + y : -1;
          if (off[u] >= 0) {
            a[u] = *reinterpret_cast<const float4*>(W + off[u]);
            b[u] = *reinterpret_cast<const float4*>(Wo + off[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (off[u] < 0) continue;
          const int e = e0 + u * NT;
          const int col = (int)(((float)e + 0.5f) * rcp), y = ylo + 2 * (e - col * cp);
          const float4 s4 = make_float4(a[u].x + b[u].x, a[u].y + b[u].y, a[u].z + b[u].z, a[u].w + b[u].w);
          if (!MMP_IN(g, (long long)kx * NCOL * ny + (long long)col * ny + y + 1, g.lim_T)) continue;
          float2* dst = Tk + (long long)col * ny + y;
          if ((ny & 1) == 0) {
            *reinterpret_cast<float4*>(dst) = s4;
          } else {
            dst[0] = make_float2(s4.x, s4.y);
            dst[1] = make_float2(s4.z, s4.w);
          }
        }
      }
    } else {
      const float rcnt = 1.0f / (float)cnt;
      for (int e = threadIdx.x; e < NCOL * cnt; e += NT) {
        const int col = (int)(((float)e + 0.5f) * rcnt), y = ylo + e - col * cnt;
        const float2 a = W[col * LP + y], b = Wo[col * LP + y];
        if (MMP_IN(g, (long long)kx * NCOL * ny + (long long)col * ny + y, g.lim_T)) Tk[(long long)col * ny + y] = cadd(a, b);
      }
    }
    cl.sync();
  }
}

}  // namespace mmp

// ------------------------------------------------------------ kernels ----
namespace mmp {

template <int NZ, int M, bool TC>
__global__ void __launch_bounds__(32 * passb_w_warps(NZ, M), 1) k_passB_w(Grid g, DemagArgs d) {
  extern __shared__ __align__(16) unsigned char sraw[];
  passB_w_plane<NZ, M, passb_w_warps(NZ, M), TC>(sraw, g, d, blockIdx.y, (int)(blockIdx.x % d.R));
}

// One launch over the kx planes: R CTAs per plane (a cluster when R = 2).
template <int NZ, int M, bool TC>
cudaError_t launch_passB_w_t(const Grid& g, const DemagArgs& d, cudaStream_t s) {
  const size_t sm = passb_w_smem(NZ, M, TC);
  cudaError_t e = cudaFuncSetAttribute(k_passB_w<NZ, M, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int threads = 32 * passb_w_warps(NZ, M);
  if (d.R == 1) {
    k_passB_w<NZ, M, TC><<<dim3(1, g.kxn), threads, sm, s>>>(g, d);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(d.R, g.kxn);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = d.R;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_passB_w<NZ, M, TC>, g, d);
}

template <int M>
cudaError_t launch_passB_w_m(const Grid& g, const DemagArgs& d, cudaStream_t s) {
  if (d.engine == 2) {   // the final DFT32 of the y transforms on the tensor cores
    switch (g.nz) {
      case 1: return launch_passB_w_t<1, M, true>(g, d, s);
      case 2: return launch_passB_w_t<2, M, true>(g, d, s);
      case 4: return launch_passB_w_t<4, M, true>(g, d, s);
      case 8: return launch_passB_w_t<8, M, true>(g, d, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (g.nz) {
    case 1: return launch_passB_w_t<1, M, false>(g, d, s);
    case 2: return launch_passB_w_t<2, M, false>(g, d, s);
    case 4: return launch_passB_w_t<4, M, false>(g, d, s);
    case 8: return launch_passB_w_t<8, M, false>(g, d, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mmp

// pass_a.cuh -- device body of pass A of the demag convolution: the
// Dormand-Prince stage assembly fused into the forward FFT along x of
// M = sum_s Ms m_s (two real rows per complex transform; the zero padding
// x >= nx is never loaded).  Used by the per-context kernel (pass_a.cu) and
// the batched stage kernel (batch.cu).
#pragma once
#include "kernels.h"

namespace mmp {

// ------------------------------------------------------------- pass A ----
// Pass A runs two 512-thread blocks per SM (64 registers a thread): its time
// goes to waiting on the stage loads, so twice the warps hide more of it.
// Its FFT therefore holds 16 values per thread (15 with a radix-3 pass),
// half of the other passes' (fft_cap_a on the host).
constexpr int kCapA = 16;
// Shared memory: the row-pair FFT buffer (padded layout) of xb components,
// the length-Px twiddles, and for the renormalised stage 1/|m_i| of every
// tile cell and sublattice.
__host__ __device__ __forceinline__ size_t passa_twiddle_offset(int Px, int ty, int xb) {
  return (size_t)xb * (ty >> 1) * fft_pitch(Px) * sizeof(float2);
}
__host__ __device__ __forceinline__ size_t passa_inv_offset(int Px, int ty, int xb) {
  return passa_twiddle_offset(Px, ty, xb) + (size_t)Px * sizeof(float2);
}

// Stage value of component c of part p at a cell: assembled from y and the
// previous stages (ASSEMBLE) or read from the given stage state.
template <bool ASSEMBLE>
__device__ __forceinline__ float stage_value(const Grid& g, const StageArgs& a, long long n, int p, int c,
                                             long long cell) {
  const long long idx = (long long)(3 * p + c) * n + cell;
  if (!MMP_IN(g, idx, g.lim_state)) return 0.0f;
  if (!ASSEMBLE) return a.stage[idx];
  float acc = a.y[idx];
#pragma unroll
  for (int j = 0; j < 7; ++j)
    if (j < a.nk) acc = fmaf(a.coef[j], a.k[j][idx], acc);
  return acc;
}

// Components c0 .. c0 + nc - 1 of pass A: the stage values are assembled
// straight into the FFT input (and written to the stage state once), M_c is
// packed in row pairs (transform (c - c0) np + p), all nc np transforms are
// done in one block_fft, and the unpacked half spectra are written to T.
// nc = 3 (g.xb) when the block holds all three components, else one call
// per component.
template <int NSUB, bool ASSEMBLE>
__device__ __forceinline__ void passA_components(int c0, int nc, float2* fbuf, const float2* tw, const float* inv,
                                                 const Grid& g, const StageArgs& a, const DemagArgs& d,
                                                 const Coefs& co, int z, int y0) {
  if (nc == 0) return;
  const int nx = g.nx, ny = g.ny, Px = g.Px;
  const int pitch = fft_pitch(Px);
  const int np = g.ty >> 1;
  const long long n = g.n;
  // Groups of FU elements per thread: all loads and sums of a group first,
  // then its stores, so that the loads of the group are in flight together
  // (stores to the stage state would otherwise order every load after the
  // previous element's stores).  Same arithmetic per element.
  constexpr int FU = 2;
  const int total = nc * np * Px;
  // e / Px by the FP32 quotient of e + 1/2: it is at least 1/(2 Px) from an
  // integer and its rounding error (e / Px) 2^-23 is smaller for e < 2^22,
  // so it truncates exactly; np = ty / 2 is a power of two
  const float rPx = 1.0f / (float)Px;
  const int npsh = __ffs(np) - 1;
  for (int e0 = threadIdx.x; e0 < total; e0 += FU * blockDim.x) {
    float mv[FU][2][NSUB];
    long long cl[FU][2];
    int cidx[FU];
#pragma unroll
    for (int u = 0; u < FU; ++u) {
      const int e = e0 + u * blockDim.x;
      const int t = (int)(((float)e + 0.5f) * rPx), x = e - t * Px;
      const int cc = t >> npsh, p = t & (np - 1), c = c0 + cc;
      cidx[u] = c;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int y = y0 + 2 * p + h;
        const bool ok = e < total && x < nx && y < ny;
        cl[u][h] = ok ? x + (long long)nx * (y + (long long)ny * z) : -1;
#pragma unroll
        for (int s = 0; s < NSUB; ++s) mv[u][h][s] = ok ? stage_value<ASSEMBLE>(g, a, n, s, c, cl[u][h]) : 0.0f;
      }
    }
#pragma unroll
    for (int u = 0; u < FU; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e >= total) continue;
      const int t = (int)(((float)e + 0.5f) * rPx), x = e - t * Px;
      const int p = t & (np - 1);
      const int c = cidx[u];
      float v2[2] = {0.0f, 0.0f};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const long long cell = cl[u][h];
        if (cell < 0) continue;
        const int row = 2 * p + h;
        const int reg = co.uniform ? 0 : co.regions[cell];
#pragma unroll
        for (int s = 0; s < NSUB; ++s) {
          float m = mv[u][h][s];
          if (ASSEMBLE) {
            if (a.normalize) m *= inv[(s * g.ty + row) * nx + x];
            if (MMP_IN(g, (long long)(3 * s + c) * n + cell, g.lim_state)) a.stage[(long long)(3 * s + c) * n + cell] = m;
          }
          v2[h] = fmaf(co.reg[s * MMP_MAX_REGIONS + reg].ms, m, v2[h]);
        }
      }
      fbuf[fidx(t, x, pitch)] = make_float2(v2[0], v2[1]);
    }
  }
  __syncthreads();
  block_fft<false, kCapA>(fbuf, d.plan_x, nc * np, tw);
  const int kt = g.kxn * g.ty;
  const float rkt = 1.0f / (float)kt;           // exact quotient as above (e < 2^22)
  const int tysh = __ffs(g.ty) - 1;
  for (int e = threadIdx.x; e < nc * kt; e += blockDim.x) {
    const int cc = (int)(((float)e + 0.5f) * rkt), r = e - cc * kt;
    const int k = r >> tysh, row = r & (g.ty - 1), y = y0 + row;
    if (y >= ny) continue;
    const int t = cc * np + (row >> 1);
    float2 Z = fbuf[fidx(t, k, pitch)];
    float2 Zm = fbuf[fidx(t, k == 0 ? 0 : Px - k, pitch)];
    float2 X;
    if ((row & 1) == 0) X = make_float2(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));
    else X = make_float2(0.5f * (Z.y + Zm.y), -0.5f * (Z.x - Zm.x));
    const long long ti = (((long long)k * 3 + c0 + cc) * g.nz + z) * ny + y;
    if (MMP_IN(g, ti, g.lim_T)) d.T[ti] = X;
  }
  __syncthreads();
}

// Pass A of one tile: rows y0 .. y0 + ty - 1 of plane z.  `sraw` is the
// block's dynamic shared memory.
template <int NSUB, bool ASSEMBLE>
__device__ __forceinline__ void passA_tile(unsigned char* sraw, const Grid& g, const StageArgs& a,
                                           const DemagArgs& d, const Coefs& co, int z, int y0) {
  const int Px = g.Px, nx = g.nx, ny = g.ny;
  float2* fbuf = reinterpret_cast<float2*>(sraw);
  float2* tw = reinterpret_cast<float2*>(sraw + passa_twiddle_offset(Px, g.ty, g.xb));
  float* inv = reinterpret_cast<float*>(sraw + passa_inv_offset(Px, g.ty, g.xb));
  const long long n = g.n;
  for (int i = threadIdx.x; i < Px; i += blockDim.x) tw[i] = __ldg(d.tw_x + i);
  if (ASSEMBLE && (a.normalize || a.nparts > a.nsub)) {
    for (int e = threadIdx.x; e < g.ty * nx; e += blockDim.x) {
      int row = e / nx, x = e - row * nx, y = y0 + row;
      if (y >= ny) continue;
      const long long cell = x + (long long)nx * (y + (long long)ny * z);
      if (a.normalize) {
        // 1/|m_i| of the renormalised stage, per sublattice
        for (int s = 0; s < NSUB; ++s) {
          float v0 = stage_value<true>(g, a, n, s, 0, cell);
          float v1 = stage_value<true>(g, a, n, s, 1, cell);
          float v2 = stage_value<true>(g, a, n, s, 2, cell);
          float nn = v0 * v0 + v1 * v1 + v2 * v2;
          inv[(s * g.ty + row) * nx + x] = nn > 0.0f ? rnorm3df(v0, v1, v2) : 1.0f;
        }
      }
      // elastic parts (u, v): assembled here, not transformed
      for (int p = a.nsub; p < a.nparts; ++p)
        for (int c = 0; c < 3; ++c) {
          const long long idx = (long long)(3 * p + c) * n + cell;
          if (MMP_IN(g, idx, g.lim_state)) a.stage[idx] = stage_value<true>(g, a, n, p, c, cell);
        }
    }
  }
  __syncthreads();
  // straight-line calls (a loop around the FFT body makes the compiler cut
  // the registers and spill); with xb = 3 the first call does all three
  const int rest = g.xb == 3 ? 0 : 1;
  passA_components<NSUB, ASSEMBLE>(0, g.xb == 3 ? 3 : 1, fbuf, tw, inv, g, a, d, co, z, y0);
  passA_components<NSUB, ASSEMBLE>(1, rest, fbuf, tw, inv, g, a, d, co, z, y0);
  passA_components<NSUB, ASSEMBLE>(2, rest, fbuf, tw, inv, g, a, d, co, z, y0);
}

}  // namespace mmp

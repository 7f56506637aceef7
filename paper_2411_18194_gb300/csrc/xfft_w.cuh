// xfft_w.cuh -- passes A and C of the demag convolution on the warp FFT
// engine (wfft.cuh), for grids with Px = 2048 (nx of 769 .. 1024).
//
// A tile is one row pair (rows y0, y0 + 1) of plane z, packed as one
// complex row z[x] = M_a[x] + i M_b[x] (x < nx, zero up to N = Px / 2).  The
// padded length-2N transform splits exactly into its even and odd outputs:
//   Z[2k'] = DFT_N(z)[k'],  Z[2k' + 1] = DFT_N(z[x] w_2N^x)[k'],
//   z[x] = IDFT_N(Z[2k'])[x] + w_2N^(-x) IDFT_N(Z[2k' + 1])[x]   (x < N),
// so six warps, one per (component, parity), do the work of a tile with
// length-N warp transforms.  The row pair is split into the two real rows'
// half spectra (pass A) or rebuilt from them (pass C) with
//   A[k] = (Z[k] + conj Z[2N - k]) / 2,  B[k] = -i (Z[k] - conj Z[2N - k]) / 2,
// where Z[2N - k] has the parity of k, so each warp pairs its own outputs.
//
// Pass A: stage assembly (16-byte loads of 4 cells), M = sum_s Ms m_s into
// shared memory, forward transforms, the half spectra of both rows to T.
// Pass C: the half spectra of both rows gathered into shared memory with
// asynchronous copies, inverse transforms, the demag field of the two rows,
// then the local field and torque of every cell: four cells per item with
// the tile rows of m staged in shared memory (stencil4.cuh), or one cell
// per thread (field_cells) for two sublattices or several regions.
#pragma once
#include "kernels.h"
#include "wfft.cuh"
#include "copy.cuh"
#include "stage.cuh"
#include "pass_a.cuh"
#include "field.cuh"
#include "stencil4.cuh"

namespace mmp {

constexpr int kXwN = 1024;            // transform length N (Px = 2 N)
constexpr int kXwThreads = 192;       // six warps: (component, parity)

// Shared memory of the warp passes A and C (bytes), under 50 KB so that four
// CTAs (24 warps at 80 registers) share an SM; the warp twiddles are read
// from global memory through L1.
//   A: Zin [3][N] float2 (reused as the even warps' scratch), odd scratch
//      [3][N] float2.
//   C: gathered half spectra [3][N + 1] float4 (reused as the six warps'
//      scratch, [6][N] float2).
__host__ __device__ constexpr size_t passa_w_smem() { return (size_t)(6 * kXwN) * sizeof(float2); }
__host__ __device__ constexpr size_t field_w_smem() { return (size_t)3 * (kXwN + 1) * sizeof(float4); }

// ------------------------------------------------------------- pass A ----
// Stage value of part p, component c at 4 consecutive cells (16-byte loads).
template <bool ASSEMBLE>
__device__ __forceinline__ float4 stage_value4(const Grid& g, const StageArgs& a, long long n, int p, int c,
                                               long long cell) {
  const long long idx = (long long)(3 * p + c) * n + cell;
  if (!MMP_IN(g, idx + 3, g.lim_state)) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (!ASSEMBLE) return *reinterpret_cast<const float4*>(a.stage + idx);
  float4 acc = __ldcs(reinterpret_cast<const float4*>(a.y + idx));
#pragma unroll
  for (int j = 0; j < 7; ++j)
    if (j < a.nk) {
      const float4 k = __ldcs(reinterpret_cast<const float4*>(a.k[j] + idx));
      const float cj = a.coef[j];
      acc.x = fmaf(cj, k.x, acc.x);
      acc.y = fmaf(cj, k.y, acc.y);
      acc.z = fmaf(cj, k.z, acc.z);
      acc.w = fmaf(cj, k.w, acc.w);
    }
  return acc;
}

// Assembly of one row (y) of the tile: cells x0 .. x0 + V - 1 (V = 4 with
// 16-byte loads when nx is a multiple of 4, else V = 1), all parts, the
// stage state written once, M_c = sum_s Ms m_s into Zin[c][x].h.
template <int NSUB, bool ASSEMBLE, int V>
__device__ __forceinline__ void passA_w_cells(const Grid& g, const StageArgs& a, const Coefs& co, float2* Zin,
                                              int h, int x0, long long cell0) {
  const long long n = g.n;
  float Mv[3][V];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int i = 0; i < V; ++i) Mv[c][i] = 0.0f;
#pragma unroll
  for (int s = 0; s < NSUB; ++s) {
    float m[3][V];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if constexpr (V == 4) {
        const float4 q = stage_value4<ASSEMBLE>(g, a, n, s, c, cell0);
        m[c][0] = q.x; m[c][1] = q.y; m[c][2] = q.z; m[c][3] = q.w;
      } else {
        m[c][0] = stage_value<ASSEMBLE>(g, a, n, s, c, cell0);
      }
    }
    if (ASSEMBLE && a.normalize) {
#pragma unroll
      for (int i = 0; i < V; ++i) {
        const float nn = m[0][i] * m[0][i] + m[1][i] * m[1][i] + m[2][i] * m[2][i];
        const float r = nn > 0.0f ? rnorm3df(m[0][i], m[1][i], m[2][i]) : 1.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) m[c][i] *= r;
      }
    }
    if (ASSEMBLE) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long idx = (long long)(3 * s + c) * n + cell0;
        if (!MMP_IN(g, idx + V - 1, g.lim_state)) continue;
        float* dst = a.stage + idx;
        if constexpr (V == 4) *reinterpret_cast<float4*>(dst) = make_float4(m[c][0], m[c][1], m[c][2], m[c][3]);
        else dst[0] = m[c][0];
      }
    }
#pragma unroll
    for (int i = 0; i < V; ++i) {
      const int reg = co.uniform ? 0 : co.regions[cell0 + i];
      const float ms = co.reg[s * MMP_MAX_REGIONS + reg].ms;
#pragma unroll
      for (int c = 0; c < 3; ++c) Mv[c][i] = fmaf(ms, m[c][i], Mv[c][i]);
    }
  }
  // elastic parts (u, v): assembled here, not transformed
  if (ASSEMBLE) {
    for (int p = a.nsub; p < a.nparts; ++p)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long idx = (long long)(3 * p + c) * n + cell0;
        if (!MMP_IN(g, idx + V - 1, g.lim_state)) continue;
        float* dst = a.stage + idx;
        if constexpr (V == 4) *reinterpret_cast<float4*>(dst) = stage_value4<true>(g, a, n, p, c, cell0);
        else dst[0] = stage_value<true>(g, a, n, p, c, cell0);
      }
  }
  float* Zf = reinterpret_cast<float*>(Zin);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int i = 0; i < V; ++i) Zf[2 * (c * kXwN + x0 + i) + h] = Mv[c][i];
}

// a.k[j], a.coef[j] for a run-time j by selects (an indexed parameter array
// would be copied to local memory)
__device__ __forceinline__ const float* stage_k(const StageArgs& a, int j) {
  const float* p = a.k[0];
#pragma unroll
  for (int i = 1; i < 7; ++i) p = j == i ? a.k[i] : p;
  return p;
}
__device__ __forceinline__ float stage_coef(const StageArgs& a, int j) {
  float c = a.coef[0];
#pragma unroll
  for (int i = 1; i < 7; ++i) c = j == i ? a.coef[i] : c;
  return c;
}

// Stage assembly of the tile's two rows with the stage vectors streamed
// through shared memory (one sublattice, no elastic parts, nx a multiple of
// 4): y (or the current state) and each previous stage k_j arrive in turn
// by asynchronous 16-byte copies into two alternating 24 KB buffers (the
// transforms' space, free until then), so all of a vector's bytes are in
// flight at once; each thread keeps the sums of its 4-cell items in
// registers.  Then the renormalisation (last stage), the stage state
// written once, and M = Ms m into Zin.
template <bool ASSEMBLE>
__device__ __forceinline__ void passA_w_assemble_async(float* buf0, float* buf1, float2* Zin, const Grid& g,
                                                       const StageArgs& a, const Coefs& co, int z, int y0) {
  constexpr int N = kXwN, IT = 3;   // at most 3 items of 4 cells per thread (2 rows x N / 4 / 192)
  const int nx = g.nx, ny = g.ny, q = nx >> 2;
  const long long n = g.n;
  const int nvec = ASSEMBLE ? 1 + a.nk : 1;
  const bool two = y0 + 1 < ny;
  const long long row0 = (long long)nx * (y0 + (long long)ny * z);   // first cell of row y0
  // copies of vector v: 2 rows x 3 components x q pieces of 16 bytes
  auto issue = [&](int v, float* b) {
    const float* src = v == 0 ? (ASSEMBLE ? a.y : a.stage) : stage_k(a, v - 1);
    const int pieces = (two ? 2 : 1) * 3 * q;
    for (int e = threadIdx.x; e < pieces; e += kXwThreads) {
      const int hc = e / q, j = e - hc * q, h = hc / 3, c = hc - 3 * h;
      const long long si = (long long)c * n + row0 + (long long)h * nx + 4 * j;
      if (MMP_IN(g, si + 3, g.lim_state)) cp_async16(b + (h * 3 + c) * nx + 4 * j, src + si);
    }
    cp_async_commit();
  };
  float acc[IT][3][4];
  issue(0, buf0);
  if (nvec > 1) issue(1, buf1);
  for (int v = 0; v < nvec; ++v) {
    if (v + 1 < nvec) cp_async_wait_one();
    else cp_async_wait_all();
    __syncthreads();
    float* b = (v & 1) ? buf1 : buf0;
    const float cv = v == 0 ? 1.0f : stage_coef(a, v - 1);
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int e = threadIdx.x + it * kXwThreads;
      if (e >= 2 * q) continue;
      const int h = e >= q, x0 = 4 * (e - h * q);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4 w = *reinterpret_cast<const float4*>(b + (h * 3 + c) * nx + x0);
        if (v == 0) {
          acc[it][c][0] = w.x; acc[it][c][1] = w.y; acc[it][c][2] = w.z; acc[it][c][3] = w.w;
        } else {
          acc[it][c][0] = fmaf(cv, w.x, acc[it][c][0]);
          acc[it][c][1] = fmaf(cv, w.y, acc[it][c][1]);
          acc[it][c][2] = fmaf(cv, w.z, acc[it][c][2]);
          acc[it][c][3] = fmaf(cv, w.w, acc[it][c][3]);
        }
      }
    }
    __syncthreads();   // the buffer is read: it takes vector v + 2
    if (v + 2 < nvec) issue(v + 2, b);
  }
  const float ms_uni = co.uniform ? co.reg[0].ms : 0.0f;
  float* Zf = reinterpret_cast<float*>(Zin);
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int e = threadIdx.x + it * kXwThreads;
    if (e >= 2 * q) continue;
    const int h = e >= q, x0 = 4 * (e - h * q);
    if (h == 1 && !two) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i) Zf[2 * (c * N + x0 + i) + h] = 0.0f;
      continue;
    }
    const long long cell0 = row0 + (long long)h * nx + x0;
    if (ASSEMBLE && a.normalize) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float m0 = acc[it][0][i], m1 = acc[it][1][i], m2 = acc[it][2][i];
        const float nn = m0 * m0 + m1 * m1 + m2 * m2;
        const float r = nn > 0.0f ? rnorm3df(m0, m1, m2) : 1.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[it][c][i] *= r;
      }
    }
    if (ASSEMBLE) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (MMP_IN(g, (long long)c * n + cell0 + 3, g.lim_state))
          *reinterpret_cast<float4*>(a.stage + (long long)c * n + cell0) =
              make_float4(acc[it][c][0], acc[it][c][1], acc[it][c][2], acc[it][c][3]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float ms = co.uniform ? ms_uni : co.reg[co.regions[cell0 + i]].ms;
#pragma unroll
      for (int c = 0; c < 3; ++c) Zf[2 * (c * N + x0 + i) + h] = ms * acc[it][c][i];
    }
  }
}

template <int NSUB, bool ASSEMBLE>
__device__ __forceinline__ void passA_w_tile(unsigned char* sraw, const Grid& g, const StageArgs& a,
                                             const DemagArgs& d, const Coefs& co, int z, int y0) {
  constexpr int N = kXwN;
  const int nx = g.nx, ny = g.ny;
  float2* Zin = reinterpret_cast<float2*>(sraw);   // [3][N]; even warps' scratch afterwards
  float2* Sodd = Zin + 3 * N;                      // [3][N] odd warps' scratch
  const float2* twT = d.tw_wx;                     // [N], global (L1)
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  // 1. stage assembly of both rows into Zin (zero for x >= nx and a row y >= ny)
  if (NSUB == 1 && (nx & 3) == 0 && a.nparts == a.nsub) {
    passA_w_assemble_async<ASSEMBLE>(reinterpret_cast<float*>(Zin), reinterpret_cast<float*>(Sodd), Zin, g, a, co,
                                     z, y0);
  } else if ((nx & 3) == 0) {
    const int q = nx >> 2;
    for (int e = threadIdx.x; e < 2 * q; e += kXwThreads) {
      const int h = e >= q, x0 = 4 * (e - h * q), y = y0 + h;
      if (y < ny) {
        passA_w_cells<NSUB, ASSEMBLE, 4>(g, a, co, Zin, h, x0, x0 + (long long)nx * (y + (long long)ny * z));
      } else {
        float* Zf = reinterpret_cast<float*>(Zin);
        for (int c = 0; c < 3; ++c)
          for (int i = 0; i < 4; ++i) Zf[2 * (c * N + x0 + i) + h] = 0.0f;
      }
    }
  } else {
    for (int e = threadIdx.x; e < 2 * nx; e += kXwThreads) {
      const int h = e >= nx, x0 = e - h * nx, y = y0 + h;
      if (y < ny) {
        passA_w_cells<NSUB, ASSEMBLE, 1>(g, a, co, Zin, h, x0, x0 + (long long)nx * (y + (long long)ny * z));
      } else {
        float* Zf = reinterpret_cast<float*>(Zin);
        for (int c = 0; c < 3; ++c) Zf[2 * (c * N + x0) + h] = 0.0f;
      }
    }
  }
  for (int i = threadIdx.x; i < 3 * (N - nx); i += kXwThreads) {
    const int c = i / (N - nx), x = nx + i - c * (N - nx);
    Zin[c * N + x] = make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  // 2. forward transforms: warp (c, par), lane l takes x = l + 32 m
  const int c = warp >> 1, par = warp & 1;
  float2 v[32];
#pragma unroll
  for (int m = 0; m < 32; ++m) {
    const int x = lane + 32 * m;
    float2 zv = Zin[c * N + x];
    if (par) zv = cmul(zv, __ldg(d.tw_wx2 + x));
    v[m] = zv;
  }
  __syncthreads();   // every warp holds its input: Zin becomes the even warps' scratch
  float2* scr = par ? Sodd + c * N : Zin + c * N;
  wfft<32, false, true>(v, scr, twT);
  // lane j: v[k2] = Z[2 k' + par], k' = j + 32 k2; natural order into the scratch
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) scr[lane + 32 * k2] = v[k2];
  __syncwarp();
  // 3. the two rows' half spectra: k = 2 k' + par <= N
  const int kmax = par ? N / 2 - 1 : N / 2;
  const bool two = y0 + 1 < ny;
  for (int kp = lane; kp <= kmax; kp += 32) {
    const int kq = par ? N - 1 - kp : (N - kp) & (N - 1);   // Z[2N - k]
    const float2 Z = scr[kp], Zm = scr[kq];
    const float2 A = make_float2(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));
    const float2 Bv = make_float2(0.5f * (Z.y + Zm.y), -0.5f * (Z.x - Zm.x));
    const int k = 2 * kp + par;
    const long long ti = (((long long)k * 3 + c) * g.nz + z) * ny + y0;
    if (!MMP_IN(g, ti + (two ? 1 : 0), g.lim_T)) continue;
    float2* dst = d.T + ti;
    if (two && (ny & 1) == 0) {
      *reinterpret_cast<float4*>(dst) = make_float4(A.x, A.y, Bv.x, Bv.y);
    } else {
      dst[0] = A;
      if (two) dst[1] = Bv;
    }
  }
}

// ------------------------------------------------------------- pass C ----
template <int NSUB, bool UNI>
__device__ __forceinline__ void field_w_tile(unsigned char* sraw, const Grid& g, const DemagArgs& d,
                                             const Coefs& co, const FieldArgs& f, int z, int y0) {
  constexpr int N = kXwN;
  const int ny = g.ny;
  float4* G = reinterpret_cast<float4*>(sraw);          // [3][N + 1]: (X_a, X_b) of the two rows
  float2* S = reinterpret_cast<float2*>(sraw);          // afterwards [6][N] warp scratch
  const float2* twT = d.tw_wx;                          // [N], global (L1)
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  // 1. gather T[k][c][z][y0 .. y0 + 1], k <= N
  const bool two = y0 + 1 < ny;
  const float2* T0 = d.T + (long long)z * ny + y0;
  const long long kstride = (long long)3 * g.nz * ny, cstride = (long long)g.nz * ny;
  if (two && (ny & 1) == 0) {
    for (int e = threadIdx.x; e < 3 * (N + 1); e += kXwThreads) {
      const int c = e / (N + 1), k = e - c * (N + 1);
      const long long ti = (long long)z * ny + y0 + k * kstride + c * cstride;
      if (MMP_IN(g, ti + 1, g.lim_T)) cp_async16(G + e, T0 + k * kstride + c * cstride);
    }
  } else {
    for (int e = threadIdx.x; e < 3 * (N + 1); e += kXwThreads) {
      const int c = e / (N + 1), k = e - c * (N + 1);
      const float2* src = T0 + k * kstride + c * cstride;
      const long long ti = (long long)z * ny + y0 + k * kstride + c * cstride;
      if (!MMP_IN(g, ti + (two ? 1 : 0), g.lim_T)) continue;
      cp_async8(reinterpret_cast<float2*>(G + e), src);
      if (two) cp_async8(reinterpret_cast<float2*>(G + e) + 1, src + 1);
      else reinterpret_cast<float2*>(G + e)[1] = make_float2(0.0f, 0.0f);
    }
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  // 2. inverse transforms: warp (c, par) takes Z[2 k' + par], k' = l + 32 m,
  // Z[k] = X_a[k] + i X_b[k] (k <= N) and conj X_a[2N - k] + i conj X_b[2N - k] above
  const int c = warp >> 1, par = warp & 1;
  float2 v[32];
#pragma unroll
  for (int m = 0; m < 32; ++m) {
    const int k = 2 * (lane + 32 * m) + par;
    const bool lo = k <= N;
    const float4 q = G[c * (N + 1) + (lo ? k : 2 * N - k)];
    v[m] = lo ? make_float2(q.x - q.w, q.y + q.z) : make_float2(q.x + q.w, q.z - q.y);
  }
  __syncthreads();   // every warp holds its input: G becomes the warps' scratch
  float2* scr = S + warp * N;
  wfft<32, true, true>(v, scr, twT);
  // lane j: v[k2] = IDFT_N(Z[2 k' + par])[x], x = j + 32 k2
  if (par) {
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
      const int x = lane + 32 * k2;
      scr[x] = cmul(v[k2], cconj(__ldg(d.tw_wx2 + x)));
    }
  }
  __syncthreads();
  if (!par) {
    const float2* odd = S + (warp + 1) * N;
    float* bd = reinterpret_cast<float*>(scr);        // rows y0, y0 + 1 of component c: [2][N]
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
      const int x = lane + 32 * k2;
      const float2 o = odd[x];
      bd[x] = v[k2].x + o.x;
      bd[N + x] = v[k2].y + o.y;
    }
  }
  __syncthreads();
  // 3. local field and torque of the two rows.  One sublattice of uniform
  // material with nx a multiple of 4: the tile rows of m into the odd
  // warps' scratch (free now; component c at floats 4 c N + 2 N) by 16-byte
  // asynchronous copies, then four cells per item (stencil4.cuh).
  if (NSUB == 1 && UNI && (g.nx & 3) == 0) {
    float* Sf = reinterpret_cast<float*>(S);
    const int nx = g.nx, q = nx >> 2, nrows = two ? 2 : 1;
    const long long n = g.n, row0 = (long long)nx * (y0 + (long long)ny * z);
    for (int e = threadIdx.x; e < 3 * nrows * q; e += kXwThreads) {
      const int c = e / (nrows * q), rem = e - c * nrows * q, h = rem / q, j = rem - h * q;
      const long long si = c * n + row0 + (long long)h * nx + 4 * j;
      if (MMP_IN(g, si + 3, g.lim_state)) cp_async16(Sf + c * 4 * N + 2 * N + h * N + 4 * j, f.stage + si);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    field_cells4<true>(Sf + 2 * N, Sf, 4 * N, N, nrows, g, co, f, z, y0);
  } else {
    field_cells<NSUB, true, UNI>(reinterpret_cast<const float*>(S), 4 * N, N, 2, g, co, f, z, y0);
  }
}

// ------------------------------------------------------------ kernels ----
template <int NSUB, bool ASSEMBLE>
__global__ void __launch_bounds__(kXwThreads, 4) k_passA_w(Grid g, StageArgs a, DemagArgs d, Coefs co) {
  extern __shared__ __align__(16) unsigned char sraw[];
  passA_w_tile<NSUB, ASSEMBLE>(sraw, g, a, d, co, blockIdx.y, 2 * blockIdx.x);
}

template <int NSUB, bool UNI>
__global__ void __launch_bounds__(kXwThreads, 4) k_field_w(Grid g, DemagArgs d, Coefs co, FieldArgs f) {
  extern __shared__ __align__(16) unsigned char sraw[];
  field_w_tile<NSUB, UNI>(sraw, g, d, co, f, blockIdx.y, 2 * blockIdx.x);
}

}  // namespace mmp

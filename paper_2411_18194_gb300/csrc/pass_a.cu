// pass_a.cu -- Dormand-Prince stage assembly and pass A of the demag
// convolution: forward FFT along x of M = sum_s Ms m_s (two real rows per
// complex transform; the zero padding x >= nx is never loaded).
#include <cooperative_groups.h>
#include "kernels.h"
#include "launch.cuh"
#include "stage.cuh"

namespace cg = cooperative_groups;

namespace mmp {

__global__ void k_assemble(Grid g, StageArgs a) {
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < g.n;
       cell += (long long)gridDim.x * blockDim.x)
    assemble_cell(a, g.n, cell);
}

__global__ void k_normalize(float* m, long long n) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    float x = m[c], y = m[n + c], z = m[2 * n + c];
    if (x * x + y * y + z * z > 0.0f) {
      float r = rnorm3df(x, y, z);
      m[c] = x * r; m[n + c] = y * r; m[2 * n + c] = z * r;
    }
  }
}

// ------------------------------------------------------------- pass A ----
// Shared memory: the row-pair FFT buffer (padded layout), the length-Px
// twiddles, and for the renormalised stage 1/|m_i| of every tile cell and
// sublattice.
__host__ __device__ __forceinline__ size_t passa_twiddle_offset(int Px, int ty) {
  return (size_t)(ty >> 1) * fft_pitch(Px) * sizeof(float2);
}
__host__ __device__ __forceinline__ size_t passa_inv_offset(int Px, int ty) {
  return passa_twiddle_offset(Px, ty) + (size_t)Px * sizeof(float2);
}

// Stage value of component c of part p at a cell: assembled from y and the
// previous stages (ASSEMBLE) or read from the given stage state.
template <bool ASSEMBLE>
__device__ __forceinline__ float stage_value(const StageArgs& a, long long n, int p, int c, long long cell) {
  const long long idx = (long long)(3 * p + c) * n + cell;
  if (!ASSEMBLE) return a.stage[idx];
  float acc = a.y[idx];
#pragma unroll
  for (int j = 0; j < 7; ++j)
    if (j < a.nk) acc = fmaf(a.coef[j], a.k[j][idx], acc);
  return acc;
}

// One component of pass A: the stage values of component c are assembled
// straight into the FFT input (and written to the stage state once), M_c is
// packed in row pairs, transformed, and the unpacked half spectra are
// written to T.  Called three times in straight-line code (a loop over c
// made the compiler keep the FFT pass registers in local memory).
template <int NSUB, bool ASSEMBLE>
__device__ __forceinline__ void passA_component(int c, float2* fbuf, const float2* tw, const float* inv,
                                                const Grid& g, const StageArgs& a, const DemagArgs& d,
                                                const Coefs& co, int z, int y0) {
  const int nx = g.nx, ny = g.ny, Px = g.Px;
  const int pitch = fft_pitch(Px);
  const long long n = g.n;
  for (int e = threadIdx.x; e < (g.ty >> 1) * Px; e += blockDim.x) {
    int p = e / Px, x = e - p * Px;
    float v2[2] = {0.0f, 0.0f};
    if (x < nx) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = 2 * p + h, y = y0 + row;
        if (y >= ny) continue;
        const long long cell = x + (long long)nx * (y + (long long)ny * z);
        const int reg = co.uniform ? 0 : co.regions[cell];
#pragma unroll
        for (int s = 0; s < NSUB; ++s) {
          float m = stage_value<ASSEMBLE>(a, n, s, c, cell);
          if (ASSEMBLE) {
            if (a.normalize) m *= inv[(s * g.ty + row) * nx + x];
            a.stage[(long long)(3 * s + c) * n + cell] = m;
          }
          v2[h] = fmaf(co.reg[s * MMP_MAX_REGIONS + reg].ms, m, v2[h]);
        }
      }
    }
    fbuf[fidx(p, x, pitch)] = make_float2(v2[0], v2[1]);
  }
  __syncthreads();
  block_fft<false>(fbuf, d.plan_x, (g.ty >> 1), tw);
  for (int e = threadIdx.x; e < g.kxn * g.ty; e += blockDim.x) {
    int k = e / g.ty, row = e - k * g.ty, y = y0 + row;
    if (y >= ny) continue;
    int p = row >> 1;
    float2 Z = fbuf[fidx(p, k, pitch)];
    float2 Zm = fbuf[fidx(p, k == 0 ? 0 : Px - k, pitch)];
    float2 X;
    if ((row & 1) == 0) X = make_float2(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));
    else X = make_float2(0.5f * (Z.y + Zm.y), -0.5f * (Z.x - Zm.x));
    d.T[(((long long)k * 3 + c) * g.nz + z) * ny + y] = X;
  }
  __syncthreads();
}

template <int NSUB, bool ASSEMBLE>
__global__ void __launch_bounds__(512) k_passA(Grid g, StageArgs a, DemagArgs d, Coefs co) {
  extern __shared__ __align__(16) unsigned char sraw[];
  const int Px = g.Px, nx = g.nx, ny = g.ny;
  float2* fbuf = reinterpret_cast<float2*>(sraw);
  float2* tw = reinterpret_cast<float2*>(sraw + passa_twiddle_offset(Px, g.ty));
  float* inv = reinterpret_cast<float*>(sraw + passa_inv_offset(Px, g.ty));
  const int z = blockIdx.y, y0 = blockIdx.x * g.ty;
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
          float v0 = stage_value<true>(a, n, s, 0, cell);
          float v1 = stage_value<true>(a, n, s, 1, cell);
          float v2 = stage_value<true>(a, n, s, 2, cell);
          float nn = v0 * v0 + v1 * v1 + v2 * v2;
          inv[(s * g.ty + row) * nx + x] = nn > 0.0f ? rnorm3df(v0, v1, v2) : 1.0f;
        }
      }
      // elastic parts (u, v): assembled here, not transformed
      for (int p = a.nsub; p < a.nparts; ++p)
        for (int c = 0; c < 3; ++c) a.stage[(long long)(3 * p + c) * n + cell] = stage_value<true>(a, n, p, c, cell);
    }
  }
  __syncthreads();
  passA_component<NSUB, ASSEMBLE>(0, fbuf, tw, inv, g, a, d, co, z, y0);
  passA_component<NSUB, ASSEMBLE>(1, fbuf, tw, inv, g, a, d, co, z, y0);
  passA_component<NSUB, ASSEMBLE>(2, fbuf, tw, inv, g, a, d, co, z, y0);
}

size_t smem_passA(const Grid& g) { return passa_inv_offset(g.Px, g.ty); }
static size_t smem_passA_launch(const Grid& g, const StageArgs& a) {
  return passa_inv_offset(g.Px, g.ty) + (a.normalize ? (size_t)a.nsub * g.ty * g.nx * sizeof(float) : 0);
}

cudaError_t launch_assemble(const Grid& g, const StageArgs& a, cudaStream_t s) {
  k_assemble<<<grid_for(g.n, 256), 256, 0, s>>>(g, a);
  return cudaGetLastError();
}

cudaError_t launch_normalize(float* m, long long n, cudaStream_t s) {
  k_normalize<<<grid_for(n, 256), 256, 0, s>>>(m, n);
  return cudaGetLastError();
}

cudaError_t launch_passA(const Grid& g, const StageArgs& a, const DemagArgs& d, const Coefs& c, int threads,
                         cudaStream_t s) {
  dim3 grid((g.ny + g.ty - 1) / g.ty, g.nz);
  size_t sm = smem_passA_launch(g, a);
  bool assemble = a.stage != nullptr && a.y != nullptr;
  cudaError_t e;
#define MMP_PA(NS, AS)                                                      \
  do {                                                                      \
    if ((e = set_smem(k_passA<NS, AS>, smem_passA(g) + 2 * g.ty * g.nx * sizeof(float))) != cudaSuccess) \
      return e;                                                             \
    k_passA<NS, AS><<<grid, threads, sm, s>>>(g, a, d, c);                 \
  } while (0)
  if (a.nsub == 1) { if (assemble) MMP_PA(1, true); else MMP_PA(1, false); }
  else { if (assemble) MMP_PA(2, true); else MMP_PA(2, false); }
#undef MMP_PA
  return cudaGetLastError();
}

}  // namespace mmp

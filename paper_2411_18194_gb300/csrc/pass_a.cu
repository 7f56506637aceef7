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
// One component of pass A: M_c of the tile, packed row pairs, forward FFT,
// unpacked half spectra written to T.  Called three times in straight-line
// code (a loop over c made the compiler keep the FFT pass registers in
// local memory).
template <int NSUB>
__device__ __forceinline__ void passA_component(int c, float2* fbuf, const Grid& g, const StageArgs& a,
                                                const DemagArgs& d, const Coefs& co, int z, int y0) {
  const int nx = g.nx, ny = g.ny, Px = g.Px;
  const int pitch = fft_pitch(Px);
  const long long n = g.n;
  for (int e = threadIdx.x; e < MMP_NP * Px; e += blockDim.x) {
    int p = e / Px, x = e - p * Px;
    int ya = y0 + 2 * p, yb = ya + 1;
    float va = 0.0f, vb = 0.0f;
    if (x < nx) {
#pragma unroll
      for (int s = 0; s < NSUB; ++s) {
        const float* ms = a.stage + ((long long)(3 * s + c)) * n;
        if (ya < ny) {
          long long cell = x + (long long)nx * (ya + (long long)ny * z);
          int r = co.uniform ? 0 : co.regions[cell];
          va = fmaf(co.reg[s * MMP_MAX_REGIONS + r].ms, ms[cell], va);
        }
        if (yb < ny) {
          long long cell = x + (long long)nx * (yb + (long long)ny * z);
          int r = co.uniform ? 0 : co.regions[cell];
          vb = fmaf(co.reg[s * MMP_MAX_REGIONS + r].ms, ms[cell], vb);
        }
      }
    }
    fbuf[fidx(p, x, pitch)] = make_float2(va, vb);
  }
  __syncthreads();
  block_fft<false>(fbuf, d.plan_x, MMP_NP, d.tw_x);
  for (int e = threadIdx.x; e < g.kxn * MMP_TY; e += blockDim.x) {
    int k = e / MMP_TY, row = e - k * MMP_TY, y = y0 + row;
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
  extern __shared__ float2 fbuf[];   // [MMP_NP][Px]
  const int z = blockIdx.y, y0 = blockIdx.x * MMP_TY;
  const int nx = g.nx, ny = g.ny;
  if (ASSEMBLE) {
    for (int e = threadIdx.x; e < MMP_TY * nx; e += blockDim.x) {
      int row = e / nx, x = e - row * nx, y = y0 + row;
      if (y < ny) assemble_cell(a, g.n, x + (long long)nx * (y + (long long)ny * z));
    }
    __syncthreads();
  }
  passA_component<NSUB>(0, fbuf, g, a, d, co, z, y0);
  passA_component<NSUB>(1, fbuf, g, a, d, co, z, y0);
  passA_component<NSUB>(2, fbuf, g, a, d, co, z, y0);
}

size_t smem_passA(const Grid& g) { return (size_t)MMP_NP * fft_pitch(g.Px) * sizeof(float2); }
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
  dim3 grid((g.ny + MMP_TY - 1) / MMP_TY, g.nz);
  size_t sm = smem_passA(g);
  bool assemble = a.stage != nullptr && a.y != nullptr;
  cudaError_t e;
#define MMP_PA(NS, AS)                                        \
  do {                                                        \
    if ((e = set_smem(k_passA<NS, AS>, sm)) != cudaSuccess) return e; \
    k_passA<NS, AS><<<grid, threads, sm, s>>>(g, a, d, c);   \
  } while (0)
  if (a.nsub == 1) { if (assemble) MMP_PA(1, true); else MMP_PA(1, false); }
  else { if (assemble) MMP_PA(2, true); else MMP_PA(2, false); }
#undef MMP_PA
  return cudaGetLastError();
}

}  // namespace mmp

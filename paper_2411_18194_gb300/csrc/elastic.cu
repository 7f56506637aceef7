// elastic.cu -- strain/stress and elastic force (4th-order stencils in the
// bulk, divergence = -G^T of the gradient G) plus the magnetoelastic force.
#include <cooperative_groups.h>
#include "kernels.h"
#include "launch.cuh"
#include "stage.cuh"

namespace cg = cooperative_groups;

namespace mmp {

// ---------------------------------------------------------- elastic -------
// Gradient operator G along an axis of n cells (rows: one-sided 2nd order at
// an edge, central 2nd order one cell in, central 4th order in the bulk;
// (f1 - f0)/h for n = 2); the divergence is -G^T.
__device__ __forceinline__ float gcoef(int i, int j, int n, float ih) {
  if (n == 1) return 0.0f;
  if (n == 2) return j == 0 ? -ih : (j == 1 ? ih : 0.0f);
  int dj = j - i;
  if (i == 0) return dj == 0 ? -1.5f * ih : dj == 1 ? 2.0f * ih : dj == 2 ? -0.5f * ih : 0.0f;
  if (i == n - 1) return dj == -2 ? 0.5f * ih : dj == -1 ? -2.0f * ih : dj == 0 ? 1.5f * ih : 0.0f;
  if (i == 1 || i == n - 2) return dj == -1 ? -0.5f * ih : dj == 1 ? 0.5f * ih : 0.0f;
  const float c = ih * (1.0f / 12.0f);
  return dj == -2 ? c : dj == -1 ? -8.0f * c : dj == 1 ? 8.0f * c : dj == 2 ? -c : 0.0f;
}

// (G f)(cell) along an axis: row `i` of G applied to f.
__device__ __forceinline__ float grad_at(const float* __restrict__ f, long long cell, int i, int n,
                                         long long stride, float ih) {
  float acc = 0.0f;
  int lo = i - 2 < 0 ? 0 : i - 2, hi = i + 2 > n - 1 ? n - 1 : i + 2;
  for (int j = lo; j <= hi; ++j) {
    float c = gcoef(i, j, n, ih);
    if (c != 0.0f) acc = fmaf(c, f[cell + (long long)(j - i) * stride], acc);
  }
  return acc;
}

// (G^T s)(cell) along an axis: sum_i G[i][j] s_i, j the cell's index.
__device__ __forceinline__ float gradT_at(const float* __restrict__ s, long long cell, int j, int n,
                                          long long stride, float ih) {
  float acc = 0.0f;
  int lo = j - 2 < 0 ? 0 : j - 2, hi = j + 2 > n - 1 ? n - 1 : j + 2;
  for (int i = lo; i <= hi; ++i) {
    float c = gcoef(i, j, n, ih);
    if (c != 0.0f) acc = fmaf(c, s[cell + (long long)(i - j) * stride], acc);
  }
  return acc;
}

// Bulk rows of G (4th-order central) and of G^T, with the coefficients and
// the order of the multiply-adds of grad_at / gradT_at, so a bulk cell gets
// bitwise the same value without the per-term coefficient selection.
__device__ __forceinline__ float grad_bulk(const float* __restrict__ f, long long cell, long long st, float ih) {
  const float c = ih * (1.0f / 12.0f);
  float acc = fmaf(c, f[cell - 2 * st], 0.0f);
  acc = fmaf(-8.0f * c, f[cell - st], acc);
  acc = fmaf(8.0f * c, f[cell + st], acc);
  return fmaf(-c, f[cell + 2 * st], acc);
}
__device__ __forceinline__ float gradT_bulk(const float* __restrict__ s, long long cell, long long st, float ih) {
  const float c = ih * (1.0f / 12.0f);
  float acc = fmaf(-c, s[cell - 2 * st], 0.0f);
  acc = fmaf(8.0f * c, s[cell - st], acc);
  acc = fmaf(-8.0f * c, s[cell + st], acc);
  return fmaf(c, s[cell + 2 * st], acc);
}
// Whether every axis of more than one cell has index i with all the rows the
// operator needs in the 4th-order bulk: G: 2 <= i <= n - 3; G^T: 4 <= i <= n - 5.
__device__ __forceinline__ bool in_bulk(const int (&idx)[3], const int (&ext)[3], int margin) {
  bool b = true;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (ext[a] > 1) b = b && idx[a] >= margin && idx[a] <= ext[a] - 1 - margin;
  return b;
}

__global__ void k_strain(Grid g, ElasticArgs e, int nsub) {
  const long long n = g.n;
  const float* u = e.stage + (long long)3 * nsub * n;
  const float* v = u + 3 * n;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n;
       cell += (long long)gridDim.x * blockDim.x) {
    int x = cell % g.nx, y = (cell / g.nx) % g.ny, z = cell / ((long long)g.nx * g.ny);
    const int idx[3] = {x, y, z}, ext[3] = {g.nx, g.ny, g.nz};
    const long long st[3] = {1, g.nx, (long long)g.nx * g.ny};
    float G[3][3], Gv[3][3];
    if (in_bulk(idx, ext, 2)) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          G[a][j] = ext[a] > 1 ? grad_bulk(u + j * n, cell, st[a], g.ih[a]) : 0.0f;
          Gv[a][j] = e.eta != 0.0f && ext[a] > 1 ? grad_bulk(v + j * n, cell, st[a], g.ih[a]) : 0.0f;
        }
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          G[a][j] = grad_at(u + j * n, cell, idx[a], ext[a], st[a], g.ih[a]);
          Gv[a][j] = e.eta != 0.0f ? grad_at(v + j * n, cell, idx[a], ext[a], st[a], g.ih[a]) : 0.0f;
        }
    }
    float eps[6] = {G[0][0], G[1][1], G[2][2], 0.5f * (G[0][1] + G[1][0]), 0.5f * (G[0][2] + G[2][0]),
                    0.5f * (G[1][2] + G[2][1])};
    float epv[6] = {Gv[0][0], Gv[1][1], Gv[2][2], 0.5f * (Gv[0][1] + Gv[1][0]), 0.5f * (Gv[0][2] + Gv[2][0]),
                    0.5f * (Gv[1][2] + Gv[2][1])};
#pragma unroll
    for (int c = 0; c < 6; ++c) e.eps[c * n + cell] = eps[c];
    float sig[6];
    sig[0] = e.c11 * eps[0] + e.c12 * (eps[1] + eps[2]);
    sig[1] = e.c11 * eps[1] + e.c12 * (eps[0] + eps[2]);
    sig[2] = e.c11 * eps[2] + e.c12 * (eps[0] + eps[1]);
    sig[3] = 2.0f * e.c44 * eps[3];
    sig[4] = 2.0f * e.c44 * eps[4];
    sig[5] = 2.0f * e.c44 * eps[5];
    if (e.eta != 0.0f) {
      sig[0] += e.eta * (e.c11 * epv[0] + e.c12 * (epv[1] + epv[2]));
      sig[1] += e.eta * (e.c11 * epv[1] + e.c12 * (epv[0] + epv[2]));
      sig[2] += e.eta * (e.c11 * epv[2] + e.c12 * (epv[0] + epv[1]));
      sig[3] += e.eta * 2.0f * e.c44 * epv[3];
      sig[4] += e.eta * 2.0f * e.c44 * epv[4];
      sig[5] += e.eta * 2.0f * e.c44 * epv[5];
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) e.sig[c * n + cell] = sig[c];
  }
}

template <bool UNI>
__global__ void k_elastic_rhs(Grid g, ElasticArgs e, Coefs co, int nsub) {
  const long long n = g.n;
  const float* u = e.stage + (long long)3 * nsub * n;
  const float* v = u + 3 * n;
  float* ku = e.kout + (long long)3 * nsub * n;
  float* kv = ku + 3 * n;
  // sigma_ab as component index into sig[6]
  const int sidx[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n;
       cell += (long long)gridDim.x * blockDim.x) {
    int x = cell % g.nx, y = (cell / g.nx) % g.ny, z = cell / ((long long)g.nx * g.ny);
    const int idx[3] = {x, y, z}, ext[3] = {g.nx, g.ny, g.nz};
    const long long st[3] = {1, g.nx, (long long)g.nx * g.ny};
    float f[3] = {0.0f, 0.0f, 0.0f};
    const bool bulkT = in_bulk(idx, ext, 4), bulk = in_bulk(idx, ext, 2);
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a)
        f[b] -= bulkT ? (ext[a] > 1 ? gradT_bulk(e.sig + sidx[a][b] * n, cell, st[a], g.ih[a]) : 0.0f)
                      : gradT_at(e.sig + sidx[a][b] * n, cell, idx[a], ext[a], st[a], g.ih[a]);
    if (e.terms & 64u) {
      int reg = UNI ? 0 : co.regions[cell];
      for (int s = 0; s < nsub; ++s) {
        const float* m = e.stage + (long long)3 * s * n;
        const RegionCoef& R = co.reg[s * MMP_MAX_REGIONS + reg];
        float G[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int j = 0; j < 3; ++j)
            G[a][j] = bulk ? (ext[a] > 1 ? grad_bulk(m + j * n, cell, st[a], g.ih[a]) : 0.0f)
                           : grad_at(m + j * n, cell, idx[a], ext[a], st[a], g.ih[a]);
        float mx = m[cell], my = m[n + cell], mz = m[2 * n + cell];
        float B1 = R.b1, B2 = R.b2;
        f[0] += 2.0f * B1 * mx * G[0][0] + B2 * (mx * (G[1][1] + G[2][2]) + my * G[1][0] + mz * G[2][0]);
        f[1] += 2.0f * B1 * my * G[1][1] + B2 * (my * (G[0][0] + G[2][2]) + mx * G[0][1] + mz * G[2][1]);
        f[2] += 2.0f * B1 * mz * G[2][2] + B2 * (mz * (G[0][0] + G[1][1]) + mx * G[0][2] + my * G[1][2]);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ku[c * n + cell] = v[c * n + cell];
      kv[c * n + cell] = f[c] * e.inv_rho;
    }
  }
}

cudaError_t launch_strain(const Grid& g, const ElasticArgs& e, int nsub, cudaStream_t s) {
  k_strain<<<grid_for(g.n, 256), 256, 0, s>>>(g, e, nsub);
  return cudaGetLastError();
}

cudaError_t launch_elastic_rhs(const Grid& g, const ElasticArgs& e, const Coefs& c, int nsub, cudaStream_t s) {
  if (c.uniform) k_elastic_rhs<true><<<grid_for(g.n, 256), 256, 0, s>>>(g, e, c, nsub);
  else k_elastic_rhs<false><<<grid_for(g.n, 256), 256, 0, s>>>(g, e, c, nsub);
  return cudaGetLastError();
}

}  // namespace mmp

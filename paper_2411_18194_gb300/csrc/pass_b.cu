// pass_b.cu -- pass B of the demag convolution, per kx plane: the ky
// residue class r (mod R) of the zero-padded y transform as a folded
// length-Py/R FFT, the z transform + 3x3 symmetric demag-kernel multiply +
// inverse z transform in registers, the inverse y FFT, and the
// recombination of the R classes through distributed shared memory of an
// R-CTA thread-block cluster (only y < ny is formed).
#include <cooperative_groups.h>
#include "kernels.h"
#include "launch.cuh"
#include "stage.cuh"

namespace cg = cooperative_groups;

namespace mmp {

// ------------------------------------------------------------- pass B ----
// 3x3 symmetric kernel times a complex 3-vector.  K points at the six
// components (xx, yy, zz, xy, xz, yz) of octant entry (|ky|, |kz|); sy, sz
// flip the components odd in ky, kz.
__device__ __forceinline__ void kmul(const float* __restrict__ K, float sy, float sz, float2& a, float2& b,
                                     float2& c) {
  float2 k01 = __ldg(reinterpret_cast<const float2*>(K));
  float2 k23 = __ldg(reinterpret_cast<const float2*>(K + 2));
  float2 k45 = __ldg(reinterpret_cast<const float2*>(K + 4));
  float xx = k01.x, yy = k01.y, zz = k23.x, xy = k23.y * sy, xz = k45.x * sz, yz = k45.y * sy * sz;
  float2 ha = make_float2(xx * a.x + xy * b.x + xz * c.x, xx * a.y + xy * b.y + xz * c.y);
  float2 hb = make_float2(xy * a.x + yy * b.x + yz * c.x, xy * a.y + yy * b.y + yz * c.y);
  float2 hc = make_float2(xz * a.x + yz * b.x + zz * c.x, xz * a.y + yz * b.y + zz * c.y);
  a = ha; b = hb; c = hc;
}

// z transform (nz = NZ cells, padded Pz = 2 NZ), kernel multiply, inverse z
// transform for column kp of W (row pitch `pitch`), as two length-NZ DFTs per
// parity of kz.
template <int NZ>
__device__ __forceinline__ void zkz_fixed(float2* W, int kp, int pitch, const float* __restrict__ Kc, float sy,
                                          const float2* __restrict__ twz) {
  if constexpr (NZ == 1) {
    float2 a = W[fidx(0, kp, pitch)], b = W[fidx(1, kp, pitch)], c = W[fidx(2, kp, pitch)];
    kmul(Kc, sy, 1.0f, a, b, c);
    W[fidx(0, kp, pitch)] = a; W[fidx(1, kp, pitch)] = b; W[fidx(2, kp, pitch)] = c;
  } else {
    float2 out[3][NZ];
#pragma unroll
    for (int par = 1; par >= 0; --par) {
      float2 f[3][NZ];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int zz = 0; zz < NZ; ++zz) {
          float2 v = W[fidx(c * NZ + zz, kp, pitch)];
          f[c][zz] = par ? cmul(v, __ldg(twz + zz)) : v;
        }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if constexpr (NZ == 2) dft2<false>(f[c][0], f[c][1]);
        else if constexpr (NZ == 4) dft4<false>(f[c][0], f[c][1], f[c][2], f[c][3]);
        else dft8<false>(f[c]);
      }
#pragma unroll
      for (int q = 0; q < NZ; ++q) {
        int kz = 2 * q + par;
        int ikz = kz <= NZ ? kz : 2 * NZ - kz;
        float sz = kz <= NZ ? 1.0f : -1.0f;
        kmul(Kc + ikz * 6, sy, sz, f[0][q], f[1][q], f[2][q]);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if constexpr (NZ == 2) dft2<true>(f[c][0], f[c][1]);
        else if constexpr (NZ == 4) dft4<true>(f[c][0], f[c][1], f[c][2], f[c][3]);
        else dft8<true>(f[c]);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int zz = 0; zz < NZ; ++zz) {
          if (par) out[c][zz] = cmul(f[c][zz], cconj(__ldg(twz + zz)));
          else out[c][zz] = cadd(out[c][zz], f[c][zz]);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int zz = 0; zz < NZ; ++zz) W[fidx(c * NZ + zz, kp, pitch)] = out[c][zz];
  }
}

// Any nz <= 16: direct DFT over the padded length Pz.
__device__ void zkz_generic(float2* W, int kp, int pitch, int nz, int Pz, const float* __restrict__ Kc, float sy,
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
    kmul(Kc + ikz * 6, sy, sz, F[0], F[1], F[2]);
    for (int zz = 0; zz < nz; ++zz) {
      float2 w = cconj(__ldg(twz + (kz * zz) % Pz));
      for (int c = 0; c < 3; ++c) out[c][zz] = cadd(out[c][zz], cmul(F[c], w));
    }
  }
  for (int c = 0; c < 3; ++c)
    for (int zz = 0; zz < nz; ++zz) W[fidx(c * nz + zz, kp, pitch)] = out[c][zz];
}

constexpr int kMaxCluster = 8;

template <int NZ>
__global__ void __launch_bounds__(512) k_passB(Grid g, DemagArgs d) {
  extern __shared__ float2 W[];    // [3 nz][Ly]
  const int RCL = d.R;              // cluster size = residue classes of ky
  const int r = (int)(blockIdx.x % RCL);
  const int kx = blockIdx.y;
  const int ny = g.ny, nz = g.nz, Py = g.Py;
  const int Ly = Py / RCL;
  const int pitch = fft_pitch(Ly);
  const int ncol = 3 * nz;
  float2* Tk = d.T + (long long)kx * ncol * ny;
  // 1. fold the ky residue class r: g_r[j] = sum_q T[j + q Ly] w^(r (j + q Ly))
  for (int e = threadIdx.x; e < ncol * Ly; e += blockDim.x) {
    int col = e / Ly, j = e - col * Ly;
    float2 acc = make_float2(0.0f, 0.0f);
    int ti = r * j;   // r*y mod Py, advanced by r*Ly per fold
    for (int y = j; y < ny; y += Ly) {
      float2 v = Tk[(long long)col * ny + y];
      if (r > 0) {
        while (ti >= Py) ti -= Py;
        v = cmul(v, __ldg(d.tw_y + ti));
        ti += r * Ly;
      }
      acc = cadd(acc, v);
    }
    W[fidx(col, j, pitch)] = acc;
  }
  __syncthreads();
  block_fft<false>(W, d.plan_ly, ncol, d.tw_ly);
  // 2. z transform + kernel multiply + inverse z transform per ky column
  for (int kp = threadIdx.x; kp < Ly; kp += blockDim.x) {
    int ky = RCL * kp + r;
    int iky = ky <= Py / 2 ? ky : Py - ky;
    float sy = ky <= Py / 2 ? 1.0f : -1.0f;
    const float* Kc = d.khat + ((long long)kx * g.kyn + iky) * g.kzn * 6;
    if constexpr (NZ > 0) zkz_fixed<NZ>(W, kp, pitch, Kc, sy, d.tw_z);
    else zkz_generic(W, kp, pitch, nz, g.Pz, Kc, sy, d.tw_z);
  }
  __syncthreads();
  block_fft<true>(W, d.plan_ly, ncol, d.tw_ly);
  // 3. recombine: out[y] = sum_r w^(-r y) h_r[y mod Ly], y < ny
  if (RCL == 1) {
    for (int e = threadIdx.x; e < ncol * ny; e += blockDim.x) {
      int col = e / ny, y = e - col * ny;
      Tk[e] = W[fidx(col, y, pitch)];
    }
  } else {
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    const int ylo = (int)((long long)ny * r / RCL), yhi = (int)((long long)ny * (r + 1) / RCL);
    const int cnt = yhi - ylo;
    float2* Wq[kMaxCluster];
    for (int q = 0; q < RCL; ++q) Wq[q] = cl.map_shared_rank(W, q);
    for (int e = threadIdx.x; e < ncol * cnt; e += blockDim.x) {
      int col = e / cnt, y = ylo + (e - col * cnt);
      int j = y;
      while (j >= Ly) j -= Ly;
      const int at = fidx(col, j, pitch);
      float2 acc = Wq[0][at];
      int ti = 0;
      for (int q = 1; q < RCL; ++q) {
        ti += y;   // q*y mod Py
        while (ti >= Py) ti -= Py;
        acc = cadd(acc, cmul(Wq[q][at], cconj(__ldg(d.tw_y + ti))));
      }
      Tk[(long long)col * ny + y] = acc;
    }
    cl.sync();
  }
}

size_t smem_passB(const Grid& g, int R) { return (size_t)3 * g.nz * fft_pitch(g.Py / R) * sizeof(float2); }
template <int NZ>
static cudaError_t launch_passB_t(const Grid& g, const DemagArgs& d, int threads, cudaStream_t s) {
  size_t sm = smem_passB(g, d.R);
  cudaError_t e = set_smem(k_passB<NZ>, sm);
  if (e != cudaSuccess) return e;
  if (d.R == 1) {
    k_passB<NZ><<<dim3(1, g.kxn), threads, sm, s>>>(g, d);
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
  return cudaLaunchKernelEx(&cfg, k_passB<NZ>, g, d);
}

cudaError_t launch_passB(const Grid& g, const DemagArgs& d, int threads, cudaStream_t s) {
  switch (g.nz) {
    case 1: return launch_passB_t<1>(g, d, threads, s);
    case 2: return launch_passB_t<2>(g, d, threads, s);
    case 4: return launch_passB_t<4>(g, d, threads, s);
    case 8: return launch_passB_t<8>(g, d, threads, s);
    default: return launch_passB_t<0>(g, d, threads, s);
  }
}

}  // namespace mmp

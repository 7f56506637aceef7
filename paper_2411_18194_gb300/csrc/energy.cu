// energy.cu -- energy of every field term (mmp_energy): one pass over the
// cells, energy densities in FP64 from the FP32 state, block sums and one
// FP64 atomic per block and term.
//
// The energies are the ones whose negative gradients the field terms are
// (Methods, Micromagnetism): exchange and DMI over the pairs of
// neighbouring magnetic cells (the boundary ghosts are the natural boundary
// condition of these energies, not energy terms), the demag energy
// -1/2 sum M . B_demag dV, the local anisotropy, cubic, Zeeman and
// magnetoelastic densities, the intersublattice exchange, and the elastic
// strain and kinetic energy.
#include "kernels.h"
#include "launch.cuh"

namespace mmp {

namespace {

constexpr int kTerms = 9;

__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

}  // namespace

template <bool UNI>
__global__ void __launch_bounds__(256) k_energy(Grid g, Coefs co, EnergyArgs a) {
  double e[kTerms];
#pragma unroll
  for (int t = 0; t < kTerms; ++t) e[t] = 0.0;
  const long long n = g.n;
  const int ext[3] = {g.nx, g.ny, g.nz};
  const long long stride[3] = {1, g.nx, (long long)g.nx * g.ny};
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n;
       cell += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(cell % g.nx), y = (int)((cell / g.nx) % g.ny), z = (int)(cell / ((long long)g.nx * g.ny));
    const int coord[3] = {x, y, z};
    const int reg = UNI ? 0 : co.regions[cell];
    for (int s = 0; s < a.nsub; ++s) {
      const RegionCoef& R = co.reg[s * MMP_MAX_REGIONS + reg];
      if (R.ms == 0.0f) continue;
      const float* ms = a.m + (long long)3 * s * n;
      const double Ms = R.ms;
      const double m[3] = {ms[cell], ms[n + cell], ms[2 * n + cell]};
      if ((a.terms & 1u) && a.Bd) {
        const float* B = a.Bd + (long long)3 * s * n;
        const double b[3] = {B[cell], B[n + cell], B[2 * n + cell]};
        e[0] += -0.5 * Ms * dot3(m, b);
      }
      if (a.terms & (2u | 8u)) {
        for (int ax = 0; ax < 3; ++ax) {
          if (coord[ax] + 1 >= ext[ax]) continue;
          const long long nc = cell + stride[ax];
          const int rn = UNI ? 0 : co.regions[nc];
          const RegionCoef& Rn = co.reg[s * MMP_MAX_REGIONS + rn];
          if (Rn.ms == 0.0f) continue;
          const double v[3] = {ms[nc], ms[n + nc], ms[2 * n + nc]};
          const double ih = g.ih[ax];
          if (a.terms & 2u) {
            double A;
            if (UNI) {
              A = R.aex;
            } else {
              const float2 h = co.hA[((long long)s * MMP_MAX_REGIONS + reg) * MMP_MAX_REGIONS + rn];
              A = (double)h.x + (double)h.y;
            }
            const double d0 = v[0] - m[0], d1 = v[1] - m[1], d2 = v[2] - m[2];
            e[1] += A * (d0 * d0 + d1 * d1 + d2 * d2) * ih * ih;
          }
          if ((a.terms & 8u) && ax < 2) {
            const double D = 0.5 * ((double)R.dind + (double)Rn.dind);
            e[3] += D * (m[2] * v[ax] - m[ax] * v[2]) * ih;
          }
        }
      }
      if (a.terms & 4u) {
        const double u[3] = {R.u[0], R.u[1], R.u[2]}, ub[3] = {R.ub[0], R.ub[1], R.ub[2]};
        const double mu = dot3(m, u), mub = dot3(m, ub);
        // ku1 = 2 Ku1 / Ms, ku2 = 4 Ku2 / Ms, kb1 = 2 Kb1 / Ms
        e[2] += -0.5 * R.ku1 * Ms * mu * mu - 0.25 * R.ku2 * Ms * mu * mu * mu * mu - 0.5 * R.kb1 * Ms * mub * mub;
      }
      if (a.terms & 256u) {
        const double c1[3] = {R.c1[0], R.c1[1], R.c1[2]}, c2[3] = {R.c2[0], R.c2[1], R.c2[2]},
                     c3[3] = {R.c3[0], R.c3[1], R.c3[2]};
        const double p = dot3(m, c1), q = dot3(m, c2), r = dot3(m, c3);
        e[8] += 0.5 * R.kc1 * Ms * (p * p * q * q + p * p * r * r + q * q * r * r);   // kc1 = 2 Kc1 / Ms
      }
      if (a.terms & 16u) {
        const double b[3] = {R.bext[0], R.bext[1], R.bext[2]};
        e[4] += -Ms * dot3(m, b);
      }
      if ((a.terms & 64u) && a.eps) {
        const float* E = a.eps;
        const double exx = E[cell], eyy = E[n + cell], ezz = E[2 * n + cell];
        const double exy = E[3 * n + cell], exz = E[4 * n + cell], eyz = E[5 * n + cell];
        e[6] += (double)R.b1 * (exx * m[0] * m[0] + eyy * m[1] * m[1] + ezz * m[2] * m[2]) +
                2.0 * (double)R.b2 * (exy * m[0] * m[1] + exz * m[0] * m[2] + eyz * m[1] * m[2]);
      }
    }
    if ((a.terms & 32u) && a.nsub == 2) {
      const RegionCoef& R1 = co.reg[reg];
      const RegionCoef& R2 = co.reg[MMP_MAX_REGIONS + reg];
      if (R1.ms > 0.0f && R2.ms > 0.0f) {
        const float* m1 = a.m;
        const float* m2 = a.m + 3 * n;
        const double p1[3] = {m1[cell], m1[n + cell], m1[2 * n + cell]};
        const double p2[3] = {m2[cell], m2[n + cell], m2[2 * n + cell]};
        for (int ax = 0; ax < 3; ++ax) {
          if (coord[ax] + 1 >= ext[ax]) continue;
          const long long nc = cell + stride[ax];
          const int rn = UNI ? 0 : co.regions[nc];
          if (co.reg[rn].ms == 0.0f || co.reg[MMP_MAX_REGIONS + rn].ms == 0.0f) continue;
          const double ih = g.ih[ax];
          double acc = 0.0;
          for (int i = 0; i < 3; ++i) acc += ((double)m1[i * n + nc] - p1[i]) * ((double)m2[i * n + nc] - p2[i]);
          e[5] += a.a12 * acc * ih * ih;
        }
        e[5] -= a.a0c * dot3(p1, p2);
      }
    }
    if ((a.terms & 128u) && a.sig) {
      const float* S = a.sig;
      const float* E = a.eps;
      double w = 0.0;
      for (int i = 0; i < 3; ++i) w += (double)S[i * n + cell] * E[i * n + cell];
      for (int i = 3; i < 6; ++i) w += 2.0 * (double)S[i * n + cell] * E[i * n + cell];
      double v2 = 0.0;
      for (int i = 0; i < 3; ++i) v2 += (double)a.vel[i * n + cell] * a.vel[i * n + cell];
      e[7] += 0.5 * w + 0.5 * a.rho * v2;
    }
  }
  // block sums, one atomic per term
  __shared__ double red[kTerms][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < kTerms; ++t) {
    double v = e[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[t][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < kTerms && ((a.terms >> threadIdx.x) & 1u)) {
    double v = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) v += red[threadIdx.x][i];
    atomicAdd(a.out + threadIdx.x, v * a.dV);
  }
}

cudaError_t launch_energy(const Grid& g, const Coefs& co, const EnergyArgs& a, cudaStream_t s) {
  const int blocks = grid_for(g.n, 256);
  if (co.uniform) k_energy<true><<<blocks, 256, 0, s>>>(g, co, a);
  else k_energy<false><<<blocks, 256, 0, s>>>(g, co, a);
  return cudaGetLastError();
}

}  // namespace mmp

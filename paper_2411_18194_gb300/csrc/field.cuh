// field.cuh -- device body of pass C: inverse x FFT of the demag field
// (x < nx only), then per cell the local field (exchange, interfacial DMI
// with its boundary ghosts, anisotropy, Zeeman, intersublattice exchange,
// magnetoelastic field) and the LLG torque, written as the Runge-Kutta
// stage derivative; for the 5th-order stage also the error estimate
// max |sum_j (b_j - b*_j) k_j| (warp-shuffle max, one atomic per block).
// Used by the per-context kernel (field.cu) and the batched stage kernel
// (batch.cu).
#pragma once
#include "kernels.h"

namespace mmp {

// ------------------------------------------------------------ helpers ----
__device__ __forceinline__ void atomic_max_pos(unsigned* addr, float v) {
  // non-negative floats (and +NaN) order like their bit patterns
  atomicMax(addr, __float_as_uint(v));
}

__device__ __forceinline__ float block_max(float v) {
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  // fmaxf drops NaN: keep it visible
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? red[lane] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;  // valid in thread 0
}

// ------------------------------------------------------ local field ------
struct CellOut { float B[3]; float tau[3]; float mxb; };

template <bool UNI>
__device__ __forceinline__ const RegionCoef& coef_at(const Coefs& co, int s, int reg) {
  return co.reg[s * MMP_MAX_REGIONS + (UNI ? 0 : reg)];
}

// Field and torque of sublattice s at one cell.  `bd` is the demag field.
template <bool UNI, int NSUB>
__device__ __forceinline__ CellOut cell_field(const Grid& g, const Coefs& co, const FieldArgs& f, int s, int x,
                                              int y, int z, long long cell, int reg, const float* bd) {
  CellOut o;
  const long long n = g.n;
  const float* ms = f.stage + (long long)3 * s * n;
  const RegionCoef& R = coef_at<UNI>(co, s, reg);
  if (R.ms == 0.0f || !MMP_IN(g, (long long)(3 * s + 2) * n + cell, g.lim_state)) {
    for (int i = 0; i < 3; ++i) { o.B[i] = 0.0f; o.tau[i] = 0.0f; }
    o.mxb = 0.0f;
    return o;
  }
  const float m[3] = {ms[cell], ms[n + cell], ms[2 * n + cell]};
  const unsigned terms = f.terms;
  const bool EX = terms & 2u, DM = terms & 8u, OPEN = terms & kTermOpenBC;
  df acc[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
  float sm[3] = {bd[0], bd[1], bd[2]};
  float dmi[3] = {0.0f, 0.0f, 0.0f};
  const int coord[3] = {x, y, z};
  const int ext[3] = {g.nx, g.ny, g.nz};
  const long long stride[3] = {1, g.nx, (long long)g.nx * g.ny};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int d = -1; d <= 1; d += 2) {
      const bool inside = (unsigned)(coord[a] + d) < (unsigned)ext[a] && MMP_IN(g, cell + d * stride[a], n);
      const long long nc = cell + d * stride[a];
      int rn = reg;
      bool present = inside;
      if (!UNI && inside) {
        rn = co.regions[nc];
        present = co.reg[s * MMP_MAX_REGIONS + rn].ms > 0.0f;
      }
      float v[3];
      float dpair = 0.0f;
      if (present) {
        v[0] = ms[nc]; v[1] = ms[n + nc]; v[2] = ms[2 * n + nc];
        if (EX) {
          df c;
          if (UNI) c = df{R.exch[a].x, R.exch[a].y};
          else {
            float2 h = co.hA[((long long)s * MMP_MAX_REGIONS + reg) * MMP_MAX_REGIONS + rn];
            c = df_mul(df{h.x, h.y}, df{R.two_over_ms_h2_df[a].x, R.two_over_ms_h2_df[a].y});
          }
#pragma unroll
          for (int i = 0; i < 3; ++i) acc[i] = df_add(acc[i], df_mul(c, two_sum(v[i], -m[i])));
        }
        if (DM && a < 2)
          dpair = UNI ? R.dmi[a]
                      : 0.5f * (R.dind + co.reg[s * MMP_MAX_REGIONS + rn].dind) * R.inv_ms * g.ih[a];
      } else if (DM && a < 2 && !OPEN) {
        // boundary ghost m + h d_n m, d_n m = -(D/2A) (z x n) x m = -(D/2A) d w
        float w[3];
        if (a == 0) { w[0] = m[2]; w[1] = 0.0f; w[2] = -m[0]; }
        else { w[0] = 0.0f; w[1] = m[2]; w[2] = -m[1]; }
        const float gf = d * R.ghost[a];
#pragma unroll
        for (int i = 0; i < 3; ++i) v[i] = m[i] - gf * w[i];
        if (EX) {
          const float eb = -d * R.exbc[a];
#pragma unroll
          for (int i = 0; i < 3; ++i) sm[i] = fmaf(eb, w[i], sm[i]);
        }
        dpair = R.dmi[a];
      } else {
        // no DMI (the ghost is m: zero-Neumann) or an open boundary (dpair
        // stays 0: the missing pair adds nothing)
        v[0] = m[0]; v[1] = m[1]; v[2] = m[2];
      }
      if (DM && a < 2) {
        dmi[a] = fmaf(d * dpair, v[2], dmi[a]);
        dmi[2] = fmaf(-d * dpair, v[a], dmi[2]);
      }
    }
  }
  if (terms & 4u) {   // anisotropy
    float mu = m[0] * R.u[0] + m[1] * R.u[1] + m[2] * R.u[2];
    float mub = m[0] * R.ub[0] + m[1] * R.ub[1] + m[2] * R.ub[2];
    float c1 = fmaf(R.ku2 * mu, mu * mu, R.ku1 * mu);
    float c2 = R.kb1 * mub;
#pragma unroll
    for (int i = 0; i < 3; ++i) sm[i] = fmaf(c1, R.u[i], fmaf(c2, R.ub[i], sm[i]));
  }
  if (terms & 256u) {   // cubic anisotropy: -(2 Kc1/Ms) [a (b^2 + c^2) c1 + b (a^2 + c^2) c2 + c (a^2 + b^2) c3]
    const float ca = m[0] * R.c1[0] + m[1] * R.c1[1] + m[2] * R.c1[2];
    const float cb = m[0] * R.c2[0] + m[1] * R.c2[1] + m[2] * R.c2[2];
    const float cc = m[0] * R.c3[0] + m[1] * R.c3[1] + m[2] * R.c3[2];
    const float fa = -R.kc1 * ca * fmaf(cb, cb, cc * cc);
    const float fb = -R.kc1 * cb * fmaf(ca, ca, cc * cc);
    const float fc = -R.kc1 * cc * fmaf(ca, ca, cb * cb);
#pragma unroll
    for (int i = 0; i < 3; ++i) sm[i] = fmaf(fa, R.c1[i], fmaf(fb, R.c2[i], fmaf(fc, R.c3[i], sm[i])));
  }
  if (terms & 16u) {  // Zeeman
#pragma unroll
    for (int i = 0; i < 3; ++i) sm[i] += R.bext[i];
  }
  if (NSUB == 2 && (terms & 32u)) {   // intersublattice exchange
    const int so = 1 - s;
    const float* mo = f.stage + (long long)3 * so * n;
    const RegionCoef& Ro = coef_at<UNI>(co, so, reg);
    if (Ro.ms > 0.0f) {
      const float mc[3] = {mo[cell], mo[n + cell], mo[2 * n + cell]};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int d = -1; d <= 1; d += 2) {
          const bool inside = (unsigned)(coord[a] + d) < (unsigned)ext[a] && MMP_IN(g, cell + d * stride[a], n);
          if (!inside) continue;
          const long long nc = cell + d * stride[a];
          if (!UNI && co.reg[so * MMP_MAX_REGIONS + co.regions[nc]].ms == 0.0f) continue;
#pragma unroll
          for (int i = 0; i < 3; ++i) sm[i] = fmaf(R.afm12[a], mo[i * n + nc] - mc[i], sm[i]);
        }
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) acc[i] = df_add(acc[i], df_mul_f(df{R.afm0.x, R.afm0.y}, mc[i]));
    }
  }
  if (terms & 64u) {   // magnetoelastic field
    const float* e = f.eps;
    float exx = e[cell], eyy = e[n + cell], ezz = e[2 * n + cell];
    float exy = e[3 * n + cell], exz = e[4 * n + cell], eyz = e[5 * n + cell];
    sm[0] += R.mel1 * exx * m[0] + R.mel2 * (exy * m[1] + exz * m[2]);
    sm[1] += R.mel1 * eyy * m[1] + R.mel2 * (exy * m[0] + eyz * m[2]);
    sm[2] += R.mel1 * ezz * m[2] + R.mel2 * (exz * m[0] + eyz * m[1]);
  }
  float B[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) B[i] = df_round(df_add_f(acc[i], sm[i] + dmi[i]));
  float mxB[3] = {m[1] * B[2] - m[2] * B[1], m[2] * B[0] - m[0] * B[2], m[0] * B[1] - m[1] * B[0]};
  float mmB[3] = {m[1] * mxB[2] - m[2] * mxB[1], m[2] * mxB[0] - m[0] * mxB[2], m[0] * mxB[1] - m[1] * mxB[0]};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    o.B[i] = B[i];
    o.tau[i] = f.relax ? R.tq * R.alpha * mmB[i] : R.tq * fmaf(R.alpha, mmB[i], mxB[i]);
  }
  o.mxb = sqrtf(mxB[0] * mxB[0] + mxB[1] * mxB[1] + mxB[2] * mxB[2]);
  return o;
}

// Pass C has its own tile height (Grid.tyc, tuned with the shape).  Unlike
// pass A it stays at 128 registers (one 512-thread block per SM): at two
// blocks of 64 registers it measured no faster (its time goes to the local
// field arithmetic, not to waiting), so its FFT holds 32 values a thread.
constexpr int kCapC = 32;

// Components c0 .. c0 + nc - 1 of the inverse x transform of pass C:
// Hermitian-extended row pairs from T (transform (c - c0) np + p), one
// inverse block_fft, the x < nx outputs into bd[c][row][x].
__device__ __forceinline__ void inverse_x_components(int c0, int nc, float2* fbuf, const float2* tw, float* bd,
                                                     const Grid& g, const DemagArgs& d, int z, int y0) {
  if (nc == 0) return;
  const int nx = g.nx, ny = g.ny, Px = g.Px;
  const int pitch = fft_pitch(Px);
  const int np = g.tyc >> 1;
  // groups of FU elements per thread: all loads first, then the stores
  constexpr int FU = 4;
  const int total = nc * np * Px;
  // e / (np Px) by the FP32 quotient of e + 1/2, exact for e < 2^22 (its
  // error (e / d) 2^-23 is below its 1/(2d) distance to an integer); np is
  // a power of two
  const float rnp = 1.0f / (float)(np * Px);
  const int npsh = __ffs(np) - 1;
  for (int e0 = threadIdx.x; e0 < total; e0 += FU * blockDim.x) {
    float2 va[FU], vb[FU];
#pragma unroll
    for (int u = 0; u < FU; ++u) {
      const int e = e0 + u * blockDim.x;
      const int cc = (int)(((float)e + 0.5f) * rnp), r = e - cc * (np * Px);
      const int k = r >> npsh, p = r & (np - 1);
      const int kk = k <= Px / 2 ? k : Px - k;
      const int ya = y0 + 2 * p, yb = ya + 1;
      const long long tb = (((long long)kk * 3 + c0 + cc) * g.nz + z) * ny;
      const float2* Tc = d.T + tb;
      const bool ok = e < total;
      va[u] = ok && ya < ny && MMP_IN(g, tb + ya, g.lim_T) ? __ldcg(Tc + ya) : make_float2(0.0f, 0.0f);
      vb[u] = ok && yb < ny && MMP_IN(g, tb + yb, g.lim_T) ? __ldcg(Tc + yb) : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int u = 0; u < FU; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e >= total) continue;
      const int cc = (int)(((float)e + 0.5f) * rnp), r = e - cc * (np * Px);
      const int k = r >> npsh, p = r & (np - 1);
      float2 xa = va[u], xb = vb[u];
      if (k > Px / 2) { xa.y = -xa.y; xb.y = -xb.y; }
      fbuf[fidx(cc * np + p, k, pitch)] = make_float2(xa.x - xb.y, xa.y + xb.x);
    }
  }
  __syncthreads();
  block_fft<true, kCapC>(fbuf, d.plan_x, nc * np, tw);
  const float rtn = 1.0f / (float)(g.tyc * nx), rnx = 1.0f / (float)nx;   // exact quotients (e < 2^22)
  for (int e = threadIdx.x; e < nc * g.tyc * nx; e += blockDim.x) {
    const int cc = (int)(((float)e + 0.5f) * rtn), r = e - cc * (g.tyc * nx);
    const int row = (int)(((float)r + 0.5f) * rnx), x = r - row * nx;
    float2 v = fbuf[fidx(cc * np + (row >> 1), x, pitch)];
    bd[((c0 + cc) * g.tyc + row) * nx + x] = (row & 1) ? v.y : v.x;
  }
  __syncthreads();
}

// Local field, torque and the reductions of rows y0 .. y0 + nrows - 1 of
// plane z (one tile): bd is the demag field of the tile, component c, row
// `row`, cell x at bd[c * cstride + row * rstride + x].
template <int NSUB, bool DEMAG, bool UNI>
__device__ __forceinline__ void field_cells(const float* bd, int cstride, int rstride, int nrows, const Grid& g,
                                            const Coefs& co, const FieldArgs& f, int z, int y0) {
  const int nx = g.nx, ny = g.ny;
  float emax = 0.0f, tmax = 0.0f;
  const long long n = g.n;
  for (int e = threadIdx.x; e < nrows * nx; e += blockDim.x) {
    int row = e / nx, x = e - row * nx, y = y0 + row;
    if (y >= ny) continue;
    long long cell = x + (long long)nx * (y + (long long)ny * z);
    if (!MMP_IN(g, cell, g.n)) continue;
    int reg = UNI ? 0 : co.regions[cell];
    float b3[3] = {0.0f, 0.0f, 0.0f};
    if (DEMAG) {
#pragma unroll
      for (int c = 0; c < 3; ++c) b3[c] = bd[c * cstride + row * rstride + x];
    }
#pragma unroll
    for (int s = 0; s < NSUB; ++s) {
      CellOut o = cell_field<UNI, NSUB>(g, co, f, s, x, y, z, cell, reg, b3);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        long long idx = (long long)(3 * s + i) * n + cell;
        if (!MMP_IN(g, idx, g.lim_B)) continue;
        f.kout[idx] = o.tau[i];
        if (f.Bout) f.Bout[idx] = o.B[i];
        if (f.err) {
          float ev = f.ecoef[6] * o.tau[i];
#pragma unroll
          for (int j = 0; j < 6; ++j)
            if (f.ecoef[j] != 0.0f) ev = fmaf(f.ecoef[j], f.ek[j][idx], ev);
          ev = fabsf(ev);
          emax = isnan(ev) || ev > emax ? ev : emax;
        }
      }
      tmax = isnan(o.mxb) || o.mxb > tmax ? o.mxb : tmax;
    }
  }
  if (f.err) {
    float v = block_max(isnan(emax) ? __int_as_float(0x7f800000) : emax);
    if (threadIdx.x == 0) atomic_max_pos(f.err, v);
  }
  if (f.torque_max) {
    float v = block_max(isnan(tmax) ? __int_as_float(0x7f800000) : tmax);
    if (threadIdx.x == 0) atomic_max_pos(f.torque_max, v);
  }
}

// Pass C of one tile: rows y0 .. y0 + ty - 1 of plane z.  `smem` is the
// block's dynamic shared memory.
template <int NSUB, bool DEMAG, bool UNI>
__device__ __forceinline__ void field_tile(float* smem, const Grid& g, const DemagArgs& d, const Coefs& co,
                                           const FieldArgs& f, int z, int y0) {
  const int nx = g.nx, ny = g.ny, Px = g.Px;
  float* bd = smem;                                                     // [3][TY][nx]
  float2* fbuf = reinterpret_cast<float2*>(smem + ((3 * g.tyc * nx + 3) & ~3));   // [NP][Px]
  if (DEMAG) {
    float2* tw = fbuf + g.xbc * (g.tyc >> 1) * fft_pitch(Px);
    for (int i = threadIdx.x; i < Px; i += blockDim.x) tw[i] = __ldg(d.tw_x + i);
    // straight-line calls, as in pass A; with xb = 3 the first does all three
    const int rest = g.xbc == 3 ? 0 : 1;
    inverse_x_components(0, g.xbc == 3 ? 3 : 1, fbuf, tw, bd, g, d, z, y0);
    inverse_x_components(1, rest, fbuf, tw, bd, g, d, z, y0);
    inverse_x_components(2, rest, fbuf, tw, bd, g, d, z, y0);
  }
  field_cells<NSUB, DEMAG, UNI>(bd, g.tyc * nx, nx, g.tyc, g, co, f, z, y0);
}

}  // namespace mmp

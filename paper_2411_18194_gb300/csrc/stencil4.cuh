// stencil4.cuh -- local field and LLG torque of one sublattice of uniform
// material on items of four consecutive cells (x0 .. x0 + 3 of one row),
// for the warp pass C (xfft_w.cuh).
//
// Data: the tile's own rows of m arrive in shared memory by 16-byte
// asynchronous copies (the caller stages them); every cell then reads its
// centre, its x neighbours and the other tile row from shared memory, and
// the y-halo row and the z-neighbour planes as 16-byte read-only loads.
//
// Arithmetic (same sums as cell_field in field.cuh, regrouped):
//   exchange  sum_a c_a ((m(+a) + m(-a)) - 2 m), c_a = 2 A / (Ms h_a^2),
//             each axis formed exactly with TwoSum, multiplied once by the
//             double-float c_a (FMA TwoProduct), the three products added
//             with TwoSum: one rounding at the end, as in cell_field;
//   iDMI      (D / (Ms h_a)) (m_z(+a) - m_z(-a)) on B_a, a = x, y, and
//             -(D / (Ms h_a)) (m_a(+a) - m_a(-a)) on B_z;
//   anisotropy, cubic anisotropy, Zeeman, magnetoelastic: per cell;
//   torque    tau = tq (m x B + alpha m x (m x B)) (relax: damping only).
// Boundaries as in cell_field: a missing neighbour adds nothing to the
// exchange sum (the zero-Neumann ghost, m itself); with DMI and a closed
// boundary, a missing x or y neighbour is the ghost m - d (h_a D / 2A)
// (z x n) x m, whose exchange term -d (D / (Ms h_a)) w is added on its own
// and whose value enters the DMI sum; at an open boundary it drops out of
// the DMI sum.
#pragma once
#include "kernels.h"
#include "field.cuh"

namespace mmp {

// ((a + b) - 2 m) with two roundings kept: (hi, lo) exact up to the final
// addition of the two rounding errors
__device__ __forceinline__ df st4_qsum(float a, float b, float m) {
  const df s = two_sum(a, b);
  const df t = two_sum(s.hi, -2.0f * m);
  return {t.hi, s.lo + t.lo};
}
// c * q, unnormalised (hi, lo)
__device__ __forceinline__ df st4_prod(float2 c, df q) {
  const float p = c.x * q.hi;
  float e = fmaf(c.x, q.hi, -p);
  e = fmaf(c.x, q.lo, fmaf(c.y, q.hi, e));
  return {p, e};
}
// sum over the three axes of c_a ((m(+a) + m(-a)) - 2 m), (hi, lo)
__device__ __forceinline__ df st4_exch(const RegionCoef& R, float xm, float xp, float ym, float yp, float zm,
                                       float zp, float m) {
  const df px = st4_prod(R.exch[0], st4_qsum(xm, xp, m));
  const df py = st4_prod(R.exch[1], st4_qsum(ym, yp, m));
  const df pz = st4_prod(R.exch[2], st4_qsum(zm, zp, m));
  const df t = two_sum(px.hi, py.hi);
  const df u = two_sum(t.hi, pz.hi);
  return {u.hi, (px.lo + py.lo + pz.lo) + (t.lo + u.lo)};
}
// hi + lo + F rounded once
__device__ __forceinline__ float st4_fin(df a, float F) {
  const df w = two_sum(a.hi, F);
  return w.hi + (a.lo + w.lo);
}
__device__ __forceinline__ void st4_put(float (&d)[4], float4 q) {
  d[0] = q.x; d[1] = q.y; d[2] = q.z; d[3] = q.w;
}
__device__ __forceinline__ float4 st4_get(const float (&d)[4]) { return make_float4(d[0], d[1], d[2], d[3]); }

// Outputs of one cell: the stage derivative, B (optional), the error
// estimate of the 5th-order stage and the torque maximum (both NaN-keeping).
__device__ __forceinline__ void st4_errmax(const FieldArgs& f, long long idx, float tau, float& emax) {
  float ev = f.ecoef[6] * tau;
#pragma unroll
  for (int j = 0; j < 6; ++j)
    if (f.ecoef[j] != 0.0f) ev = fmaf(f.ecoef[j], f.ek[j][idx], ev);
  ev = fabsf(ev);
  emax = isnan(ev) || ev > emax ? ev : emax;
}

// Value of component i of the ghost cell beyond a missing neighbour in
// direction d along axis a (x: 0, y: 1) with the DMI boundary condition:
// m - d (h_a D / 2A) w, w = (m_z, 0, -m_x) for x and (0, m_z, -m_y) for y.
__device__ __forceinline__ float st4_ghost(int i, int a, float d, float g, float mx, float my, float mz) {
  if (a == 0) return i == 0 ? mx - d * g * mz : i == 1 ? my : mz + d * g * mx;
  return i == 0 ? mx : i == 1 ? my - d * g * mz : mz + d * g * my;
}

// One item: cells x0 .. x0 + 3 of tile row h (y = y0 + h) of plane z.
// msm, bd: m and the demag field of the tile rows in shared memory,
// component c, row h, cell x at [c * cs + h * rs + x]; `two`: the tile has
// its second row.
template <bool DEMAG>
__device__ __forceinline__ void st4_item(const float* msm, const float* bd, int cs, int rs, int h, int x0, bool two,
                                         const Grid& g, const RegionCoef& R, const FieldArgs& f, int z, int y,
                                         long long cell0, float& emax, float& tmax) {
  const int nx = g.nx, ny = g.ny;
  const long long n = g.n, pl = (long long)nx * ny;
  const unsigned terms = f.terms;
  const bool EX = terms & 2u, DM = terms & 8u, OPEN = terms & kTermOpenBC;
  if (R.ms == 0.0f) {   // empty material: no field, no torque
    if (!MMP_IN(g, cell0 + 3, n)) return;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const long long idx = (long long)i * n + cell0;
      *reinterpret_cast<float4*>(f.kout + idx) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (f.Bout) *reinterpret_cast<float4*>(f.Bout + idx) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (f.err) {
#pragma unroll
        for (int j = 0; j < 4; ++j) st4_errmax(f, idx + j, 0.0f, emax);
      }
    }
    return;
  }
  const bool hasL = x0 > 0, hasR = x0 + 4 < nx, hasYm = y > 0, hasYp = y + 1 < ny;
  const bool hasZm = z > 0, hasZp = z + 1 < g.nz;
  if (!MMP_IN(g, cell0 + 3, n) || (hasYm && !MMP_IN(g, cell0 - nx, n)) || (hasYp && !MMP_IN(g, cell0 + nx + 3, n)) ||
      (hasZm && !MMP_IN(g, cell0 - pl, n)) || (hasZp && !MMP_IN(g, cell0 + pl + 3, n)))
    return;
  // a missing x or y neighbour: the ghost (DMI, closed boundary) or m itself
  // (no DMI, or open boundary, where it also drops out of the DMI sum)
  const bool GH = DM && !OPEN;
  const float* st = f.stage;
  float m[3][4];
#pragma unroll
  for (int c = 0; c < 3; ++c) st4_put(m[c], *reinterpret_cast<const float4*>(msm + c * cs + h * rs + x0));
  // F_c: every single-precision term of B_c (demag added at the end)
  float F[3][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float mx = m[0][j], my = m[1][j], mz = m[2][j];
    float s[3] = {0.0f, 0.0f, 0.0f};
    if (GH && EX) {   // the exchange term of the ghosts, c_a (ghost - m) = -d (D / (Ms h_a)) w
      const bool lx = j == 0 && !hasL, rx = j == 3 && !hasR;
      const float ex = (lx ? R.exbc[0] : 0.0f) - (rx ? R.exbc[0] : 0.0f);
      const float ey = (!hasYm ? R.exbc[1] : 0.0f) - (!hasYp ? R.exbc[1] : 0.0f);
      s[0] = ex * mz;
      s[1] = ey * mz;
      s[2] = -(ex * mx) - ey * my;
    }
    if (terms & 4u) {   // uniaxial anisotropy
      const float mu = mx * R.u[0] + my * R.u[1] + mz * R.u[2];
      const float mub = mx * R.ub[0] + my * R.ub[1] + mz * R.ub[2];
      const float c1 = fmaf(R.ku2 * mu, mu * mu, R.ku1 * mu), c2 = R.kb1 * mub;
#pragma unroll
      for (int i = 0; i < 3; ++i) s[i] = fmaf(c1, R.u[i], fmaf(c2, R.ub[i], s[i]));
    }
    if (terms & 256u) {   // cubic anisotropy
      const float ca = mx * R.c1[0] + my * R.c1[1] + mz * R.c1[2];
      const float cb = mx * R.c2[0] + my * R.c2[1] + mz * R.c2[2];
      const float cc = mx * R.c3[0] + my * R.c3[1] + mz * R.c3[2];
      const float fa = -R.kc1 * ca * fmaf(cb, cb, cc * cc);
      const float fb = -R.kc1 * cb * fmaf(ca, ca, cc * cc);
      const float fc = -R.kc1 * cc * fmaf(ca, ca, cb * cb);
#pragma unroll
      for (int i = 0; i < 3; ++i) s[i] = fmaf(fa, R.c1[i], fmaf(fb, R.c2[i], fmaf(fc, R.c3[i], s[i])));
    }
    if (terms & 16u) {   // Zeeman
#pragma unroll
      for (int i = 0; i < 3; ++i) s[i] += R.bext[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) F[i][j] = s[i];
  }
  if (terms & 64u) {   // magnetoelastic field
    const float* e = f.eps + cell0;
    float exx[4], eyy[4], ezz[4], exy[4], exz[4], eyz[4];
    st4_put(exx, __ldg(reinterpret_cast<const float4*>(e)));
    st4_put(eyy, __ldg(reinterpret_cast<const float4*>(e + n)));
    st4_put(ezz, __ldg(reinterpret_cast<const float4*>(e + 2 * n)));
    st4_put(exy, __ldg(reinterpret_cast<const float4*>(e + 3 * n)));
    st4_put(exz, __ldg(reinterpret_cast<const float4*>(e + 4 * n)));
    st4_put(eyz, __ldg(reinterpret_cast<const float4*>(e + 5 * n)));
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      F[0][j] += R.mel1 * exx[j] * m[0][j] + R.mel2 * (exy[j] * m[1][j] + exz[j] * m[2][j]);
      F[1][j] += R.mel1 * eyy[j] * m[1][j] + R.mel2 * (exy[j] * m[0][j] + eyz[j] * m[2][j]);
      F[2][j] += R.mel1 * ezz[j] * m[2][j] + R.mel2 * (exz[j] * m[0][j] + eyz[j] * m[1][j]);
    }
  }
  // neighbours of component i: xl, xr the cells left of x0 and right of
  // x0 + 3; ym, yp, zm, zp the 4 cells one row / plane away (a missing z
  // neighbour is m itself: the zero-Neumann ghost)
  float B[3][4];
  df exz[4];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int i = k == 0 ? 2 : k - 1;   // z first: its neighbours carry the DMI of B_x and B_y
    const float* srow = msm + i * cs + h * rs;
    const float* grow = st + (long long)i * n + cell0;
    const float xl = hasL ? srow[x0 - 1] : m[i][0];
    const float xr = hasR ? srow[x0 + 4] : m[i][3];
    float ym[4], yp[4], zm[4], zp[4];
    if (h == 0) {
      if (hasYm) st4_put(ym, __ldg(reinterpret_cast<const float4*>(grow - nx)));
      else st4_put(ym, st4_get(m[i]));
      if (two) st4_put(yp, *reinterpret_cast<const float4*>(srow + rs + x0));
      else st4_put(yp, st4_get(m[i]));   // y + 1 = ny
    } else {
      st4_put(ym, *reinterpret_cast<const float4*>(srow - rs + x0));
      if (hasYp) st4_put(yp, __ldg(reinterpret_cast<const float4*>(grow + nx)));
      else st4_put(yp, st4_get(m[i]));
    }
    if (hasZm) st4_put(zm, __ldg(reinterpret_cast<const float4*>(grow - pl)));
    else st4_put(zm, st4_get(m[i]));
    if (hasZp) st4_put(zp, __ldg(reinterpret_cast<const float4*>(grow + pl)));
    else st4_put(zp, st4_get(m[i]));
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float xm = j == 0 ? xl : m[i][j - 1];
      const float xp = j == 3 ? xr : m[i][j + 1];
      df ex = {0.0f, 0.0f};
      if (EX) ex = st4_exch(R, xm, xp, ym[j], yp[j], zm[j], zp[j], m[i][j]);
      if (DM) {
        // DMI neighbour values: the ghost beyond a missing neighbour (closed
        // boundary) or nothing (open boundary: it drops out of the sum)
        const float dxm = j > 0 || hasL ? xm : GH ? st4_ghost(i, 0, -1.0f, R.ghost[0], m[0][0], m[1][0], m[2][0]) : 0.0f;
        const float dxp = j < 3 || hasR ? xp : GH ? st4_ghost(i, 0, 1.0f, R.ghost[0], m[0][3], m[1][3], m[2][3]) : 0.0f;
        if (i == 2) {
          F[0][j] = fmaf(R.dmi[0], dxp - dxm, F[0][j]);
        } else if (i == 0) {
          F[2][j] = fmaf(-R.dmi[0], dxp - dxm, F[2][j]);
        }
        if (i != 0) {
          const float dym = hasYm ? ym[j] : GH ? st4_ghost(i, 1, -1.0f, R.ghost[1], m[0][j], m[1][j], m[2][j]) : 0.0f;
          const float dyp = hasYp ? yp[j] : GH ? st4_ghost(i, 1, 1.0f, R.ghost[1], m[0][j], m[1][j], m[2][j]) : 0.0f;
          if (i == 2) F[1][j] = fmaf(R.dmi[1], dyp - dym, F[1][j]);
          else F[2][j] = fmaf(-R.dmi[1], dyp - dym, F[2][j]);
        }
      }
      if (i == 2) {
        exz[j] = ex;
      } else {
        const float b = DEMAG ? bd[i * cs + h * rs + x0 + j] : 0.0f;
        B[i][j] = st4_fin(ex, F[i][j] + b);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float b = DEMAG ? bd[2 * cs + h * rs + x0 + j] : 0.0f;
    B[2][j] = st4_fin(exz[j], F[2][j] + b);
  }
  // torque
  float tau[3][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float mx = m[0][j], my = m[1][j], mz = m[2][j];
    const float bx = B[0][j], by = B[1][j], bz = B[2][j];
    const float mxB[3] = {my * bz - mz * by, mz * bx - mx * bz, mx * by - my * bx};
    const float mmB[3] = {my * mxB[2] - mz * mxB[1], mz * mxB[0] - mx * mxB[2], mx * mxB[1] - my * mxB[0]};
#pragma unroll
    for (int i = 0; i < 3; ++i) tau[i][j] = f.relax ? R.tq * R.alpha * mmB[i] : R.tq * fmaf(R.alpha, mmB[i], mxB[i]);
    const float mxb = sqrtf(mxB[0] * mxB[0] + mxB[1] * mxB[1] + mxB[2] * mxB[2]);
    tmax = isnan(mxb) || mxb > tmax ? mxb : tmax;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const long long idx = (long long)i * n + cell0;
    *reinterpret_cast<float4*>(f.kout + idx) = st4_get(tau[i]);
    if (f.Bout) *reinterpret_cast<float4*>(f.Bout + idx) = st4_get(B[i]);
    if (f.err) {
#pragma unroll
      for (int j = 0; j < 4; ++j) st4_errmax(f, idx + j, tau[i][j], emax);
    }
  }
}

// Local field and torque of the tile rows y0 .. y0 + nrows - 1 (nrows = 1
// or 2) of plane z, four cells per item (nx a multiple of 4, uniform
// material, one sublattice), then the block reductions as in field_cells.
template <bool DEMAG>
__device__ __forceinline__ void field_cells4(const float* msm, const float* bd, int cs, int rs, int nrows,
                                             const Grid& g, const Coefs& co, const FieldArgs& f, int z, int y0) {
  const int nx = g.nx, q = nx >> 2;
  // the material's coefficients in shared memory: read there, they are not
  // reloaded from global memory after every store of the outputs
  __shared__ RegionCoef sR;
  {
    const int* src = reinterpret_cast<const int*>(co.reg);
    int* dst = reinterpret_cast<int*>(&sR);
    for (int i = threadIdx.x; i < (int)(sizeof(RegionCoef) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  float emax = 0.0f, tmax = 0.0f;
  for (int e = threadIdx.x; e < nrows * q; e += blockDim.x) {
    const int h = e >= q, x0 = 4 * (e - h * q), y = y0 + h;
    const long long cell0 = x0 + (long long)nx * (y + (long long)g.ny * z);
    st4_item<DEMAG>(msm, bd, cs, rs, h, x0, nrows == 2, g, sR, f, z, y, cell0, emax, tmax);
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

}  // namespace mmp

// mmp.cu -- the C-ABI (include/mmp.h): context, parameters, set-up of the
// demag kernel spectrum, evaluation sequencing and the Dormand-Prince RK45
// controller (FP64 time, step size and error control on the host).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "ctx.h"
#include "dp45.h"
#include "kernels.h"
#include "mmp.h"
#include "plan.h"

using namespace mmp;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

const double kRc = 10.0;   // Newell below 10 max(cell), asymptotic above

float2 split(double v) {
  float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

}  // namespace

namespace {

void* dalloc(mmp_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (c->ualloc) {
    p = c->ualloc(bytes, c->uuser);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}

void dfree(mmp_ctx* c, void* p) {
  if (!p) return;
  if (c->ufree) c->ufree(p, c->uuser);
  else cudaFree(p);
}

template <typename T>
int alloc_into(mmp_ctx* c, T*& p, size_t bytes) {
  dfree(c, p);
  p = static_cast<T*>(dalloc(c, bytes));
  if (!p) return fail(MMP_E_OOM, "device allocation of %zu bytes failed", bytes);
  return MMP_OK;
}

int cuda_check(mmp_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MMP_OK;
  c->poisoned = true;
  return fail(MMP_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(expr, what)                                   \
  do {                                                   \
    int _rc = cuda_check(ctx, (expr), what);             \
    if (_rc != MMP_OK) return _rc;                       \
  } while (0)
#define TRY(expr)                                        \
  do {                                                   \
    int _rc = (expr);                                    \
    if (_rc != MMP_OK) return _rc;                       \
  } while (0)

// A device-side wait that ran past its limit (the tensor-core stage) sets
// ctx->d_flag; read it at a point that synchronises anyway.
// The device flag word: bit 0 set by a device-side wait that ran past its
// limit (tensor-core stage), bit 1 by an index check of the bounds-checked
// build (MMP_CHECK_BOUNDS).
int check_flag(mmp_ctx* ctx) {
#ifdef MMP_CHECK_BOUNDS
  if (!ctx->d_flag) return MMP_OK;
#else
  if (!(ctx->engine & MMP_ENGINE_TC_Y) || !ctx->d_flag) return MMP_OK;
#endif
  unsigned f = 0;
  CK(cudaMemcpyAsync(&f, ctx->d_flag, sizeof f, cudaMemcpyDeviceToHost, ctx->stream), "read device flag");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  if (f & 2u) {
    ctx->poisoned = true;
    return fail(MMP_E_BOUNDS, "bounds-checked build: a kernel index fell outside its buffer (the access was skipped)");
  }
  if (f) {
    ctx->poisoned = true;
    return fail(MMP_E_TIMEOUT, "a device-side wait of the tensor-core stage ran past its limit");
  }
  return MMP_OK;
}

int check_ctx(mmp_ctx* ctx) {
  if (!ctx) return fail(MMP_E_INVAL, "null context");
  if (ctx->poisoned) return fail(MMP_E_STATE, "context poisoned by an earlier CUDA error");
  return MMP_OK;
}

bool has(const mmp_ctx* c, unsigned t) { return (c->terms & t) != 0; }

int wanted_parts(const mmp_ctx* c) { return c->nsub + (has(c, MMP_T_ELASTIC) ? 2 : 0); }

// (Re)allocate the state-sized buffers when the number of parts changes,
// keeping the magnetisation (and u, v when they exist in both layouts).
int ensure_state(mmp_ctx* ctx) {
  int want = wanted_parts(ctx);
  if (want == ctx->nparts && ctx->d_y) return MMP_OK;
  long long n = ctx->g.n;
  long long nstate = 3LL * want * n;
  float* ny = static_cast<float*>(dalloc(ctx, nstate * sizeof(float)));
  if (!ny) return fail(MMP_E_OOM, "state allocation failed");
  CK(cudaMemsetAsync(ny, 0, nstate * sizeof(float), ctx->stream), "memset state");
  if (ctx->d_y) {
    int keep = std::min(ctx->nparts, want);
    CK(cudaMemcpyAsync(ny, ctx->d_y, 3LL * keep * n * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream),
       "copy state");
  }
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  dfree(ctx, ctx->d_y);
  ctx->d_y = ny;
  ctx->nparts = want;
  ctx->nstate = nstate;
  ctx->g.lim_state = nstate;
  TRY(alloc_into(ctx, ctx->d_stage, nstate * sizeof(float)));
  for (int i = 0; i < 7; ++i) TRY(alloc_into(ctx, ctx->d_k[i], nstate * sizeof(float)));
  ctx->k1_valid = false;
  return MMP_OK;
}

int upload_coefs(mmp_ctx* ctx) {
  if (!ctx->coef_dirty) return MMP_OK;
  std::vector<RegionCoef> rc(2 * MMP_MAX_REGIONS);
  const double* h = ctx->cell;
  const double A0 = ctx->glob[MMP_A0], A12 = ctx->glob[MMP_A12], alat = ctx->glob[MMP_LATTICE_A];
  for (int s = 0; s < 2; ++s)
    for (int r = 0; r < MMP_MAX_REGIONS; ++r) {
      RegionCoef& c = rc[s * MMP_MAX_REGIONS + r];
      memset(&c, 0, sizeof c);
      if (s >= ctx->nsub) continue;
      double Ms = ctx->scal[MMP_MS][s][r], A = ctx->scal[MMP_AEX][s][r], al = ctx->scal[MMP_ALPHA][s][r];
      double D = ctx->scal[MMP_DIND][s][r];
      c.ms = (float)Ms;
      c.alpha = (float)al;
      c.tq = (float)(-kGamma / (1.0 + al * al));
      c.aex = (float)A;
      c.dind = (float)D;
      if (Ms <= 0.0) { c.ms = 0.0f; continue; }
      double im = 1.0 / Ms;
      c.inv_ms = (float)im;
      for (int a = 0; a < 3; ++a) {
        c.exch[a] = split(2.0 * A * im / (h[a] * h[a]));
        c.two_over_ms_h2[a] = (float)(2.0 * im / (h[a] * h[a]));
        c.two_over_ms_h2_df[a] = split(2.0 * im / (h[a] * h[a]));
        c.dmi[a] = (float)(D * im / h[a]);
        c.ghost[a] = A > 0 ? (float)(h[a] * D / (2.0 * A)) : 0.0f;
        c.exbc[a] = A > 0 ? (float)(D * im / h[a]) : 0.0f;
        c.afm12[a] = (float)(A12 * im / (h[a] * h[a]));
      }
      c.ku1 = (float)(2.0 * ctx->scal[MMP_KU1][s][r] * im);
      c.ku2 = (float)(4.0 * ctx->scal[MMP_KU2][s][r] * im);
      c.kb1 = (float)(2.0 * ctx->scal[MMP_KB1][s][r] * im);
      // cubic axes: c1 normalised, c2 made orthogonal to it (Gram-Schmidt), c3 = c1 x c2
      {
        const double* a1 = ctx->vec[MMP_ANIS_C1][s][r];
        const double* a2 = ctx->vec[MMP_ANIS_C2][s][r];
        double n1 = sqrt(a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2]);
        double e1[3] = {0, 0, 0}, e2[3] = {0, 0, 0};
        if (n1 > 0)
          for (int i = 0; i < 3; ++i) e1[i] = a1[i] / n1;
        double d12 = a2[0] * e1[0] + a2[1] * e1[1] + a2[2] * e1[2];
        double v2[3] = {a2[0] - d12 * e1[0], a2[1] - d12 * e1[1], a2[2] - d12 * e1[2]};
        double n2 = sqrt(v2[0] * v2[0] + v2[1] * v2[1] + v2[2] * v2[2]);
        if (n2 > 0)
          for (int i = 0; i < 3; ++i) e2[i] = v2[i] / n2;
        double e3[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        for (int i = 0; i < 3; ++i) {
          c.c1[i] = (float)e1[i];
          c.c2[i] = (float)e2[i];
          c.c3[i] = (float)e3[i];
        }
        c.kc1 = (float)(2.0 * ctx->scal[MMP_KC1][s][r] * im);
      }
      const double* u = ctx->vec[MMP_ANIS_U][s][r];
      const double* ub = ctx->vec[MMP_ANIS_UB][s][r];
      double nu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      double nub = sqrt(ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
      for (int i = 0; i < 3; ++i) {
        c.u[i] = nu > 0 ? (float)(u[i] / nu) : 0.0f;
        c.ub[i] = nub > 0 ? (float)(ub[i] / nub) : 0.0f;
        c.bext[i] = (float)ctx->vec[MMP_B_EXT][s][r][i];
      }
      c.afm0 = alat > 0 ? split(4.0 * A0 * im / (alat * alat)) : make_float2(0.0f, 0.0f);
      c.mel1 = (float)(-2.0 * ctx->scal[MMP_B1][s][r] * im);
      c.mel2 = (float)(-2.0 * ctx->scal[MMP_B2][s][r] * im);
      c.b1 = (float)ctx->scal[MMP_B1][s][r];
      c.b2 = (float)ctx->scal[MMP_B2][s][r];
    }
  CK(cudaMemcpyAsync(ctx->d_coef, rc.data(), rc.size() * sizeof(RegionCoef), cudaMemcpyHostToDevice,
                     ctx->stream),
     "upload coefficients");
  if (!ctx->uniform) {
    if (!ctx->d_hA) TRY(alloc_into(ctx, ctx->d_hA, (size_t)2 * MMP_MAX_REGIONS * MMP_MAX_REGIONS * sizeof(float2)));
    std::vector<float2> hA((size_t)2 * MMP_MAX_REGIONS * MMP_MAX_REGIONS);
    for (int s = 0; s < 2; ++s)
      for (int a = 0; a < MMP_MAX_REGIONS; ++a)
        for (int b = 0; b < MMP_MAX_REGIONS; ++b) {
          double A1 = s < ctx->nsub ? ctx->scal[MMP_AEX][s][a] : 0.0;
          double A2 = s < ctx->nsub ? ctx->scal[MMP_AEX][s][b] : 0.0;
          double hm = (A1 + A2) != 0.0 ? 2.0 * A1 * A2 / (A1 + A2) : 0.0;
          hA[((size_t)s * MMP_MAX_REGIONS + a) * MMP_MAX_REGIONS + b] = split(hm);
        }
    CK(cudaMemcpyAsync(ctx->d_hA, hA.data(), hA.size() * sizeof(float2), cudaMemcpyHostToDevice, ctx->stream),
       "upload hA");
  }
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  ctx->coef_dirty = false;
  return MMP_OK;
}

// Resident demag kernel spectra, shared by every context of the process
// with the same extents and cell size on the same device (reference
// counted; library-owned cudaMalloc memory).
struct KhatEntry {
  float* ptr = nullptr;
  int refs = 0;
};
using KhatKey = std::tuple<int, int, int, int, double, double, double>;
std::mutex g_khat_mu;
std::map<KhatKey, KhatEntry> g_khat;

KhatKey khat_key(const mmp_ctx* ctx) {
  int dev = 0;
  cudaGetDevice(&dev);
  return KhatKey(dev, ctx->g.nx, ctx->g.ny, ctx->g.nz, ctx->cell[0], ctx->cell[1], ctx->cell[2]);
}

void release_khat(mmp_ctx* ctx) {
  if (!ctx->d_khat) return;
  std::lock_guard<std::mutex> lk(g_khat_mu);
  auto it = g_khat.find(ctx->khat_key);
  if (it != g_khat.end() && it->second.ptr == ctx->d_khat && --it->second.refs == 0) {
    cudaFree(it->second.ptr);
    g_khat.erase(it);
  }
  ctx->d_khat = nullptr;
}

int build_khat(mmp_ctx* ctx) {
  if (!ctx->khat_dirty) return MMP_OK;
  const Grid& g = ctx->g;
  const KhatKey key = khat_key(ctx);
  std::lock_guard<std::mutex> lk(g_khat_mu);
  {
    auto it = g_khat.find(key);
    if (it != g_khat.end()) {
      it->second.refs++;
      ctx->d_khat = it->second.ptr;
      ctx->khat_key = key;
      ctx->khat_dirty = false;
      return MMP_OK;
    }
  }
  size_t nk = (size_t)g.kxn * g.kyn * g.kzn;
  float* khat = nullptr;
  if (cudaMalloc(&khat, (size_t)g.kxn * g.kyn * g.krow * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return fail(MMP_E_OOM, "allocation of the demag kernel spectrum failed");
  }
  long long ext = std::max<long long>({(long long)g.nx * g.ny * g.nz, (long long)g.kxn * g.ny * g.nz,
                                       (long long)g.kxn * g.kyn * g.nz, (long long)nk});
  double* b0 = nullptr;
  double* b1 = nullptr;
  double2* trig[3] = {nullptr, nullptr, nullptr};
  int rc = MMP_OK;
  rc = alloc_into(ctx, b0, (size_t)ext * 6 * sizeof(double));
  if (rc == MMP_OK) rc = alloc_into(ctx, b1, (size_t)ext * 6 * sizeof(double));
  const int P[3] = {g.Px, g.Py, g.Pz};
  std::vector<double2> host[3];
  for (int a = 0; a < 3 && rc == MMP_OK; ++a) {
    host[a].resize(P[a]);
    for (int t = 0; t < P[a]; ++t) {
      double ang = 2.0 * 3.14159265358979323846 * (double)t / (double)P[a];
      host[a][t] = make_double2(cos(ang), sin(ang));
    }
    rc = alloc_into(ctx, trig[a], P[a] * sizeof(double2));
    if (rc == MMP_OK && cudaMemcpyAsync(trig[a], host[a].data(), P[a] * sizeof(double2),
                                        cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
      rc = cuda_check(ctx, cudaGetLastError(), "upload trig");
  }
  if (rc == MMP_OK) {
    KernelBuild kb;
    kb.n[0] = g.nx; kb.n[1] = g.ny; kb.n[2] = g.nz;
    kb.P[0] = g.Px; kb.P[1] = g.Py; kb.P[2] = g.Pz;
    for (int a = 0; a < 3; ++a) { kb.cell[a] = ctx->cell[a]; kb.trig[a] = trig[a]; }
    kb.rc = kRc;
    kb.buf0 = b0;
    kb.buf1 = b1;
    kb.out = khat;
    kb.krow = g.krow;
    rc = cuda_check(ctx, build_kernel_spectrum(kb, ctx->stream), "demag kernel build");
    if (rc == MMP_OK) rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "demag kernel build (sync)");
  }
  dfree(ctx, b0);
  dfree(ctx, b1);
  for (int a = 0; a < 3; ++a) dfree(ctx, trig[a]);
  if (rc != MMP_OK) {
    cudaFree(khat);
    return rc;
  }
  KhatEntry e;
  e.ptr = khat;
  e.refs = 1;
  g_khat[key] = e;
  ctx->d_khat = khat;
  ctx->khat_key = key;
  ctx->khat_dirty = false;
  return MMP_OK;
}

int validate_terms(mmp_ctx* ctx) {
  if (ctx->nsub == 2 && has(ctx, MMP_T_DMI))
    return fail(MMP_E_INVAL, "DMI with two sublattices is not supported (its boundary condition couples them)");
  if (has(ctx, MMP_T_MEL) && !has(ctx, MMP_T_ELASTIC))
    return fail(MMP_E_INVAL, "the magnetoelastic term needs the elastic term (its strain comes from u)");
  if (has(ctx, MMP_T_MEL) || has(ctx, MMP_T_ELASTIC)) {
    // empty cells would need free elastic surfaces inside the grid
    for (int s = 0; s < ctx->nsub; ++s)
      for (int r = 0; r < MMP_MAX_REGIONS; ++r)
        if (ctx->used[r] && ctx->scal[MMP_MS][s][r] == 0.0)
          return fail(MMP_E_INVAL, "magnetoelastic/elastic terms need every cell magnetic (region %d has Ms = 0)", r);
  }
  if (has(ctx, MMP_T_DEMAG)) {
    const Grid& g = ctx->g;
    if (g.Px > 4096 || g.Py > 4096 || g.Pz > 32)
      return fail(MMP_E_INVAL, "demag: padded lengths must be <= 4096 (x, y) and nz <= 16");
  }
  if (has(ctx, MMP_T_ELASTIC) && ctx->glob[MMP_RHO] <= 0.0)
    return fail(MMP_E_INVAL, "elastic term needs a positive mass density");
  if (has(ctx, MMP_T_AFM) && ctx->nsub != 2) return fail(MMP_E_INVAL, "AFM term needs two sublattices");
  if (has(ctx, MMP_T_AFM) && ctx->glob[MMP_LATTICE_A] <= 0.0)
    return fail(MMP_E_INVAL, "AFM term needs a positive lattice parameter");
  return MMP_OK;
}

int prepare(mmp_ctx* ctx) {
  TRY(validate_terms(ctx));
  TRY(ensure_state(ctx));
  TRY(upload_coefs(ctx));
  if (has(ctx, MMP_T_DEMAG)) {
    TRY(build_khat(ctx));
    if (!ctx->d_T)
      TRY(alloc_into(ctx, ctx->d_T, (size_t)ctx->g.kxn * 3 * ctx->g.nz * ctx->g.ny * sizeof(float2)));
  }
  if ((has(ctx, MMP_T_MEL) || has(ctx, MMP_T_ELASTIC)) && !ctx->d_eps) {
    TRY(alloc_into(ctx, ctx->d_eps, (size_t)6 * ctx->g.n * sizeof(float)));
    TRY(alloc_into(ctx, ctx->d_sig, (size_t)6 * ctx->g.n * sizeof(float)));
  }
  return MMP_OK;
}

int upload_table(mmp_ctx* ctx, float2*& dst, const std::vector<float2>& w) {
  TRY(alloc_into(ctx, dst, w.size() * sizeof(float2)));
  CK(cudaMemcpy(dst, w.data(), w.size() * sizeof(float2), cudaMemcpyHostToDevice), "upload twiddles");
  return MMP_OK;
}

// Whether a launch shape is valid for the context's grid; message in `why`.
bool shape_ok(const mmp_ctx* ctx, const mmp_shape& s, const char** why) {
  const Grid& g = ctx->g;
  FftPlan px, py;
  if (s.ty != 2 && s.ty != 4 && s.ty != 8) { *why = "ty must be 2, 4 or 8"; return false; }
  if (s.R != 1 && s.R != 2 && s.R != 4 && s.R != 8) { *why = "R must be 1, 2, 4 or 8"; return false; }
  if (g.Py % s.R != 0 || (s.R > 1 && g.Py / s.R < 2)) { *why = "R must divide the padded y length"; return false; }
  if (!make_plan(g.Px, px, s.radix_x) || !make_plan(g.Py / s.R, py, s.radix_y)) {
    *why = "unsupported FFT plan";
    return false;
  }
  if ((long long)(s.ty / 2) * g.Px > (long long)fft_cap_a(px) * 512) {
    *why = "pass A row pairs above the FFT capacity of a 512-thread block";
    return false;
  }
  if (s.tyc != 0 && s.tyc != 2 && s.tyc != 4 && s.tyc != 8) { *why = "tyc must be 0, 2, 4 or 8"; return false; }
  const int tyc = s.tyc ? s.tyc : pick_tile_rows_c(s.ty, g.Px);
  if ((long long)(tyc / 2) * g.Px > (long long)fft_cap(px) * 512) {
    *why = "pass C row pairs above the FFT capacity of a 512-thread block";
    return false;
  }
  Grid gs = g;   // shared memory of passes A and C at this shape (one component per call)
  gs.ty = s.ty;
  gs.xb = 1;
  gs.tyc = tyc;
  gs.xbc = 1;
  if (smem_passA(gs) + (size_t)ctx->nsub * s.ty * g.nx * sizeof(float) > 227 * 1024 ||
      smem_field(gs, true) > 227 * 1024) {
    *why = "pass A or C shared memory above 227 KB";
    return false;
  }
  if (s.engine & ~(MMP_ENGINE_WARP_B | MMP_ENGINE_WARP_X | MMP_ENGINE_TC_Y)) { *why = "unknown engine bits"; return false; }
  if ((s.engine & MMP_ENGINE_TC_Y) && !((s.engine & MMP_ENGINE_WARP_B) && passb_tc_supported(g, s.R))) {
    *why = "the tensor-core stage needs the warp pass B";
    return false;
  }
  if ((s.engine & MMP_ENGINE_WARP_X) && !xw_supported(g)) {
    *why = "the warp passes A and C need Px = 2048 (nx of 769 .. 1024)";
    return false;
  }
  if (s.engine & MMP_ENGINE_WARP_B) {
    if (!passb_w_supported(g, s.R)) {
      *why = "the warp pass B needs Py/R of 256, 512 or 1024, ny <= Py/R, R of 1 or 2 and nz of 1, 2, 4 or 8";
      return false;
    }
    return true;
  }
  if (passb_smem(g.ny, g.nz, g.Py, g.kzn, s.R, s.stage_kernel != 0).total > 227 * 1024) {
    *why = "pass B shared memory above 227 KB";
    return false;
  }
  if ((long long)3 * g.nz * (g.Py / s.R) > 2LL * fft_cap(py) * 512) {
    *why = "pass B plane above two chunks of the FFT capacity of a 512-thread block";
    return false;
  }
  return true;
}

// Set the launch shape: FFT plans, their twiddle tables, tile rows, cluster
// size and block sizes.  The cached first stage is dropped (the FP32
// rounding order changes).
int apply_shape(mmp_ctx* ctx, const mmp_shape& s) {
  const char* why = "";
  if (!shape_ok(ctx, s, &why)) return fail(MMP_E_INVAL, "bad shape: %s", why);
  Grid& g = ctx->g;
  make_plan(g.Px, ctx->plan_x, s.radix_x);
  make_plan(g.Py / s.R, ctx->plan_ly, s.radix_y);
  TRY(upload_table(ctx, ctx->d_tw_x, pass_twiddles(ctx->plan_x)));
  TRY(upload_table(ctx, ctx->d_tw_ly, pass_twiddles(ctx->plan_ly)));
  if (s.engine & MMP_ENGINE_WARP_B) TRY(upload_table(ctx, ctx->d_tw_wy, warp_twiddles(g.Py / s.R)));
  if ((s.engine & MMP_ENGINE_TC_Y) && !ctx->d_tw_tc) {
    const std::vector<float> t = tc_dft32_table();
    TRY(alloc_into(ctx, ctx->d_tw_tc, t.size() * sizeof(float)));
    CK(cudaMemcpy(ctx->d_tw_tc, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice), "upload tensor-core table");
  }
  if (s.engine & MMP_ENGINE_WARP_X) {
    TRY(upload_table(ctx, ctx->d_tw_wx, warp_twiddles(g.Px / 2)));
    std::vector<float2> w = roots(g.Px);
    w.resize(g.Px / 2);
    TRY(upload_table(ctx, ctx->d_tw_wx2, w));
  }
  g.ty = s.ty;
  g.tyc = s.tyc ? s.tyc : pick_tile_rows_c(s.ty, g.Px);
  // all three components in one x-FFT call when a 512-thread block holds
  // them and the pass's shared memory fits (pass A and pass C separately)
  g.xb = 3;
  if ((long long)3 * (g.ty / 2) * g.Px > (long long)fft_cap_a(ctx->plan_x) * 512 ||
      smem_passA(g) + (size_t)ctx->nsub * g.ty * g.nx * sizeof(float) > 227 * 1024)
    g.xb = 1;
  g.xbc = 3;
  if ((long long)3 * (g.tyc / 2) * g.Px > (long long)fft_cap(ctx->plan_x) * 512 || smem_field(g, true) > 227 * 1024)
    g.xbc = 1;
  ctx->R = s.R;
  ctx->ks = s.stage_kernel != 0;
  ctx->radix_x = s.radix_x;
  ctx->radix_y = s.radix_y;
  ctx->engine = s.engine;
  launch_threads(g, ctx->R, &ctx->thrA, &ctx->thrB, &ctx->thrC);
  ctx->k1_valid = false;
  ctx->config_gen++;
  return MMP_OK;
}

mmp_shape current_shape(const mmp_ctx* ctx) {
  mmp_shape s;
  s.ty = ctx->g.ty;
  s.tyc = ctx->g.tyc;
  s.radix_x = ctx->radix_x;
  s.radix_y = ctx->radix_y;
  s.R = ctx->R;
  s.stage_kernel = ctx->ks;
  s.engine = ctx->engine;
  return s;
}

DemagArgs demag_args(mmp_ctx* ctx) {
  DemagArgs d;
  d.T = ctx->d_T;
  d.khat = ctx->d_khat;
  d.tw_x = ctx->d_tw_x;
  d.tw_y = ctx->d_tw_y;
  d.tw_ly = ctx->d_tw_ly;
  d.tw_z = ctx->d_tw_z;
  d.plan_x = ctx->plan_x;
  d.plan_ly = ctx->plan_ly;
  d.R = ctx->R;
  d.ks = ctx->ks;
  d.tw_wy = ctx->d_tw_wy;
  d.tw_wx = ctx->d_tw_wx;
  d.tw_wx2 = ctx->d_tw_wx2;
  d.tw_tc = ctx->d_tw_tc;
  d.err = ctx->d_flag;
  d.engine = (ctx->engine & MMP_ENGINE_WARP_B) ? ((ctx->engine & MMP_ENGINE_TC_Y) ? 2 : 1) : 0;
  return d;
}

Coefs coefs(mmp_ctx* ctx) {
  Coefs c;
  c.reg = ctx->d_coef;
  c.regions = ctx->d_regions;
  c.hA = ctx->d_hA;
  c.uniform = ctx->uniform ? 1 : 0;
  return c;
}

// Bracket one launch with events when tracing is on.
struct Traced {
  mmp_ctx* ctx;
  int k;
  cudaEvent_t stop = nullptr;
  Traced(mmp_ctx* c, int kernel) : ctx(c), k(kernel) {
    if (!ctx->prof) return;
    auto& v = ctx->prof_events[k];
    if (ctx->prof_used[k] == v.size()) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      v.push_back({a, b});
    }
    auto& pr = v[ctx->prof_used[k]++];
    cudaEventRecord(pr.first, ctx->stream);
    stop = pr.second;
  }
  ~Traced() {
    if (stop) cudaEventRecord(stop, ctx->stream);
  }
};

// One field evaluation.  With `sa.y` set the stage is assembled from it
// into ctx->d_stage; otherwise `src` (the current state) is evaluated.
int evaluate(mmp_ctx* ctx, StageArgs sa, const float* src, float* kout, float* Bout, unsigned* err,
             const float* ecoef, const float* const* ek, int relax, unsigned* tmax) {
  const Grid& g = ctx->g;
  const bool demag = has(ctx, MMP_T_DEMAG);
  const bool elastic = has(ctx, MMP_T_ELASTIC);
  const bool strain = elastic || has(ctx, MMP_T_MEL);
  DemagArgs d = demag_args(ctx);
  Coefs co = coefs(ctx);
  sa.stage = sa.y ? ctx->d_stage : const_cast<float*>(src);
  sa.nparts = ctx->nparts;
  sa.nsub = ctx->nsub;
  const float* stage = sa.stage;
  const bool wx = demag && (ctx->engine & MMP_ENGINE_WARP_X);
  if (demag) {
    {
      Traced t(ctx, MMP_K_PASS_A);
      CK(wx ? launch_passA_w(g, sa, d, co, ctx->stream) : launch_passA(g, sa, d, co, ctx->thrA, ctx->stream),
         "pass A");
    }
    { Traced t(ctx, MMP_K_PASS_B); CK(launch_passB(g, d, ctx->thrB, ctx->stream), "pass B"); }
  } else if (sa.y) {
    Traced t(ctx, MMP_K_ASSEMBLE);
    CK(launch_assemble(g, sa, ctx->stream), "assemble");
  }
  ElasticArgs ea;
  ea.stage = stage;
  ea.kout = kout;
  ea.eps = ctx->d_eps;
  ea.sig = ctx->d_sig;
  ea.c11 = (float)ctx->glob[MMP_C11];
  ea.c12 = (float)ctx->glob[MMP_C12];
  ea.c44 = (float)ctx->glob[MMP_C44];
  ea.eta = (float)ctx->glob[MMP_ETA];
  ea.inv_rho = ctx->glob[MMP_RHO] > 0 ? (float)(1.0 / ctx->glob[MMP_RHO]) : 0.0f;
  ea.terms = ctx->terms;
  if (strain) { Traced t(ctx, MMP_K_STRAIN); CK(launch_strain(g, ea, ctx->nsub, ctx->stream), "strain"); }
  FieldArgs f;
  memset(&f, 0, sizeof f);
  f.stage = stage;
  f.kout = kout;
  f.Bout = Bout;
  f.eps = ctx->d_eps;
  f.terms = kernel_terms(ctx);
  f.err = err;
  if (err) {
    for (int j = 0; j < 7; ++j) f.ecoef[j] = ecoef[j];
    for (int j = 0; j < 6; ++j) f.ek[j] = ek[j];
  }
  f.relax = relax;
  f.torque_max = tmax;
  {
    Traced t(ctx, MMP_K_FIELD);
    CK(wx ? launch_field_w(g, d, co, f, ctx->nsub, ctx->stream)
          : launch_field(g, d, co, f, ctx->nsub, demag, ctx->thrC, ctx->stream),
       "field");
  }
  if (elastic) {
    Traced t(ctx, MMP_K_ELASTIC);
    CK(launch_elastic_rhs(g, ea, co, ctx->nsub, ctx->stream), "elastic");
  }
  ctx->evals++;
  return MMP_OK;
}

int ensure_k1(mmp_ctx* ctx, int relax) {
  if (ctx->k1_valid && ctx->k1_relax == relax) return MMP_OK;
  StageArgs sa;
  memset(&sa, 0, sizeof sa);
  TRY(evaluate(ctx, sa, ctx->d_y, ctx->d_k[0], nullptr, nullptr, nullptr, nullptr, relax, nullptr));
  ctx->k1_valid = true;
  ctx->k1_relax = relax;
  return MMP_OK;
}

// One attempt of size h of the context's method: stages 1..S, the last at
// the renormalised solution (whose k is the next step's k1).  With want_err
// the error estimate (and the torque maximum at the new state) are read
// back (one synchronisation).
int attempt(mmp_ctx* ctx, double h, bool want_err, int relax, double* err_out, double* tmax_out) {
  TRY(ensure_k1(ctx, relax));
  if (want_err) CK(cudaMemsetAsync(ctx->d_red, 0, 2 * sizeof(unsigned), ctx->stream), "reset error");
  const Tableau& T = tableau(ctx->method);
  float ecoef[7];
  error_coefs(T, h, ecoef);
  const float* ek[6];
  for (int j = 0; j < 6; ++j) ek[j] = j < T.S ? ctx->d_k[j] : nullptr;
  for (int i = 1; i <= T.S; ++i) {
    StageArgs sa;
    memset(&sa, 0, sizeof sa);
    sa.y = ctx->d_y;
    sa.nk = i;
    for (int j = 0; j < i; ++j) sa.k[j] = ctx->d_k[j];
    stage_coefs(T, h, i, sa.coef);
    sa.normalize = (i == T.S);
    bool last = (i == T.S);
    TRY(evaluate(ctx, sa, nullptr, ctx->d_k[i], nullptr, last && want_err ? ctx->d_red : nullptr, ecoef, ek,
                 relax, last && want_err ? ctx->d_red + 1 : nullptr));
  }
  if (want_err) {
    CK(cudaMemcpyAsync(ctx->h_red, ctx->d_red, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream),
       "read error");
    CK(cudaStreamSynchronize(ctx->stream), "sync");
    float e, tm;
    memcpy(&e, &ctx->h_red[0], 4);
    memcpy(&tm, &ctx->h_red[1], 4);
    *err_out = e;
    if (tmax_out) *tmax_out = tm;
  }
  return MMP_OK;
}

void accept(mmp_ctx* ctx, double h) {
  std::swap(ctx->d_y, ctx->d_stage);
  std::swap(ctx->d_k[0], ctx->d_k[tableau(ctx->method).S]);
  ctx->k1_valid = true;
  ctx->t += h;
  ctx->steps++;
}

// Advance: nsteps attempts-limited loop.  `until` < 0: count accepted steps.
// Fixed-step pairs from a CUDA graph: two steps (12 evaluations and the
// buffer swaps) captured once on the context's private stream; after two
// accepted steps the y/stage and k1/k7 buffers are back in place, so the
// graph replays.  Re-captured when the buffers, the step or the method
// differ from those of the capture.  Ordered after earlier work of the
// context's stream and before later work by events.
int replay_pairs(mmp_ctx* ctx, long long pairs) {
  const Tableau& T = tableau(ctx->method);
  const bool same = ctx->gexec && ctx->g_y == ctx->d_y && ctx->g_k0 == ctx->d_k[0] && ctx->g_dt == ctx->dt &&
                    ctx->g_method == ctx->method && ctx->g_config_gen == ctx->config_gen && ctx->g_ks == T.S;
  if (!ctx->gstream) {
    CK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking), "graph stream");
    CK(cudaEventCreateWithFlags(&ctx->gev[0], cudaEventDisableTiming), "graph event");
    CK(cudaEventCreateWithFlags(&ctx->gev[1], cudaEventDisableTiming), "graph event");
  }
  if (!same) {
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
    cudaStream_t user = ctx->stream;
    ctx->stream = ctx->gstream;
    ctx->g_y = ctx->d_y;
    ctx->g_k0 = ctx->d_k[0];
    CK(cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeRelaxed), "begin capture");
    int rc = MMP_OK;
    double err = 0.0;
    for (int s = 0; s < 2 && rc == MMP_OK; ++s) {
      rc = attempt(ctx, ctx->dt, false, 0, &err, nullptr);
      std::swap(ctx->d_y, ctx->d_stage);
      std::swap(ctx->d_k[0], ctx->d_k[T.S]);
    }
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->gstream, &gr);
    ctx->stream = user;
    ctx->evals -= 2 * T.S;   // captured, not run
    TRY(rc);
    CK(e, "end capture");
    e = cudaGraphInstantiate(&ctx->gexec, gr, 0);
    cudaGraphDestroy(gr);
    CK(e, "instantiate");
    ctx->g_dt = ctx->dt;
    ctx->g_method = ctx->method;
    ctx->g_config_gen = ctx->config_gen;
    ctx->g_ks = T.S;
  }
  CK(cudaEventRecord(ctx->gev[0], ctx->stream), "graph event");
  CK(cudaStreamWaitEvent(ctx->gstream, ctx->gev[0], 0), "graph wait");
  for (long long i = 0; i < pairs; ++i) CK(cudaGraphLaunch(ctx->gexec, ctx->gstream), "graph launch");
  CK(cudaEventRecord(ctx->gev[1], ctx->gstream), "graph event");
  CK(cudaStreamWaitEvent(ctx->stream, ctx->gev[1], 0), "graph wait");
  for (long long i = 0; i < 2 * pairs; ++i) {
    ctx->t += ctx->dt;
    ctx->steps++;
  }
  ctx->evals += 2 * pairs * T.S;
  return MMP_OK;
}

int advance(mmp_ctx* ctx, long long nsteps, double until, int relax, double torque_tol, double timeout_s,
            bool* converged) {
  TRY(prepare(ctx));
  auto t0 = std::chrono::steady_clock::now();
  long long done = 0;
  const bool adaptive = ctx->adaptive || relax;
  // fixed steps without a time limit or tracing: pairs of steps from a graph
  if (!adaptive && until < 0.0 && !ctx->prof && nsteps - done >= 2) {
    TRY(ensure_k1(ctx, 0));
    const long long pairs = (nsteps - done) / 2;
    TRY(replay_pairs(ctx, pairs));
    done += 2 * pairs;
  }
  while (true) {
    if (until >= 0.0) {
      if (ctx->t >= until * (1.0 - 1e-15)) break;
    } else if (done >= nsteps) {
      break;
    }
    double h = ctx->dt;
    if (until >= 0.0 && ctx->t + h > until) h = until - ctx->t;
    if (!adaptive) {
      double err = 0.0;
      TRY(attempt(ctx, h, false, relax, &err, nullptr));
      accept(ctx, h);
      ++done;
      continue;
    }
    double err = 0.0, tm = 0.0;
    TRY(attempt(ctx, h, true, relax, &err, &tm));
    if (!std::isfinite(err)) {
      ctx->k1_valid = true;   // state and k1 untouched
      return fail(MMP_E_NONFINITE, "non-finite error estimate at t = %g s (dt = %g s)", ctx->t, h);
    }
    bool ok = err <= ctx->tol || h <= ctx->dt_min;
    double fac = grow(err, ctx->tol, tableau(ctx->method).exponent);
    if (ok) {
      accept(ctx, h);
      ++done;
    } else {
      ctx->rejected++;
    }
    ctx->dt = std::min(std::max(h * fac, ctx->dt_min), ctx->dt_max);
    if (relax && ok && tm <= torque_tol) {
      if (converged) *converged = true;
      break;
    }
    if (timeout_s > 0) {
      double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > timeout_s) return fail(MMP_E_TIMEOUT, "relax did not converge within %g s", timeout_s);
    }
  }
  if (!adaptive) CK(cudaStreamSynchronize(ctx->stream), "sync");
  return check_flag(ctx);
}

// Device time per pass (ms) of `reps` field evaluations of the current
// state, from the tracing events (one warm-up evaluation first).
int time_passes(mmp_ctx* ctx, int reps, double* ta, double* tb, double* tc) {
  StageArgs sa;
  memset(&sa, 0, sizeof sa);
  TRY(evaluate(ctx, sa, ctx->d_y, ctx->d_k[0], nullptr, nullptr, nullptr, nullptr, 0, nullptr));
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  const bool was = ctx->prof;
  for (int k = 0; k < MMP_NKERNEL; ++k) ctx->prof_used[k] = 0;
  ctx->prof = true;
  int rc = MMP_OK;
  for (int r = 0; r < reps && rc == MMP_OK; ++r)
    rc = evaluate(ctx, sa, ctx->d_y, ctx->d_k[0], nullptr, nullptr, nullptr, nullptr, 0, nullptr);
  ctx->prof = was;
  TRY(rc);
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  double t[3] = {0, 0, 0};
  const int ks[3] = {MMP_K_PASS_A, MMP_K_PASS_B, MMP_K_FIELD};
  for (int i = 0; i < 3; ++i) {
    for (size_t j = 0; j < ctx->prof_used[ks[i]]; ++j) {
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, ctx->prof_events[ks[i]][j].first, ctx->prof_events[ks[i]][j].second),
         "event time");
      t[i] += ms;
    }
    t[i] /= reps;
  }
  for (int k = 0; k < MMP_NKERNEL; ++k) ctx->prof_used[k] = 0;
  *ta = t[0];
  *tb = t[1];
  *tc = t[2];
  return MMP_OK;
}

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, mmp_shape> g_tuned;

}  // namespace

namespace mmp {
int report_error(int code, const char* msg) { return fail(code, "%s", msg); }
int ctx_prepare(mmp_ctx* ctx) { return prepare(ctx); }
}  // namespace mmp

// ============================================================== C-ABI =====
extern "C" {

int mmp_version(void) { return MMP_VERSION; }

const char* mmp_last_error(void) { return g_err.c_str(); }

int mmp_create(mmp_ctx** out, int nx, int ny, int nz, double cx, double cy, double cz, int nsub,
               void* stream, mmp_alloc_fn alloc, mmp_free_fn dealloc, void* user) {
  g_err.clear();
  if (!out) return fail(MMP_E_INVAL, "out is null");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return fail(MMP_E_INVAL, "grid extents must be >= 1");
  if (!(cx > 0) || !(cy > 0) || !(cz > 0)) return fail(MMP_E_INVAL, "cell sizes must be > 0");
  if (nsub != 1 && nsub != 2) return fail(MMP_E_INVAL, "n_sublattices must be 1 or 2");
  if ((alloc == nullptr) != (dealloc == nullptr)) return fail(MMP_E_INVAL, "give both allocator functions or none");
  long long n = (long long)nx * ny * nz;
  if (n > (1LL << 31)) return fail(MMP_E_INVAL, "grid too large");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MMP_E_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
  }
  mmp_ctx* ctx = new mmp_ctx();
  ctx->stream = static_cast<cudaStream_t>(stream);
  ctx->ualloc = alloc;
  ctx->ufree = dealloc;
  ctx->uuser = user;
  ctx->nsub = nsub;
  ctx->cell[0] = cx; ctx->cell[1] = cy; ctx->cell[2] = cz;
  memset(ctx->scal, 0, sizeof ctx->scal);
  memset(ctx->vec, 0, sizeof ctx->vec);
  memset(ctx->glob, 0, sizeof ctx->glob);
  for (int s = 0; s < 2; ++s)
    for (int r = 0; r < MMP_MAX_REGIONS; ++r) {
      ctx->vec[MMP_ANIS_U][s][r][2] = 1.0;
      ctx->vec[MMP_ANIS_UB][s][r][0] = 1.0;
      ctx->vec[MMP_ANIS_C1][s][r][0] = 1.0;
      ctx->vec[MMP_ANIS_C2][s][r][1] = 1.0;
    }
  Grid& g = ctx->g;
  g.nx = nx; g.ny = ny; g.nz = nz; g.n = n;
  g.Px = nice_length(nx); g.Py = nice_length(ny); g.Pz = nice_length(nz);
  g.kxn = g.Px / 2 + 1; g.kyn = g.Py / 2 + 1; g.kzn = g.Pz / 2 + 1;
  g.krow = (6 * g.kzn + 3) & ~3;
  g.ty = pick_tile_rows(g.ny, g.nz, g.Px);
  g.xb = 1;
  g.tyc = pick_tile_rows_c(g.ty, g.Px);
  g.xbc = 1;
  for (int a = 0; a < 3; ++a) {
    g.h[a] = (float)ctx->cell[a];
    g.ih[a] = (float)(1.0 / ctx->cell[a]);
  }
  int rc = MMP_OK;
#define CR(x) do { if (rc == MMP_OK) rc = (x); } while (0)
  CR(alloc_into(ctx, ctx->d_coef, 2 * MMP_MAX_REGIONS * sizeof(RegionCoef)));
  CR(alloc_into(ctx, ctx->d_red, 2 * sizeof(unsigned)));
  CR(alloc_into(ctx, ctx->d_flag, sizeof(unsigned)));
  if (rc == MMP_OK && cudaMemset(ctx->d_flag, 0, sizeof(unsigned)) != cudaSuccess)
    rc = cuda_check(ctx, cudaGetLastError(), "clear device flag");
  // sizes the index checks of the bounds-checked build compare against
  g.chk = ctx->d_flag;
  g.lim_state = 3LL * nsub * n;
  g.lim_B = 3LL * nsub * n;
  g.lim_T = (long long)g.kxn * 3 * g.nz * g.ny;
  g.lim_khat = (long long)g.kxn * g.kyn * g.krow;
  if (rc == MMP_OK && cudaMallocHost(&ctx->h_red, 2 * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    rc = fail(MMP_E_OOM, "pinned allocation failed");
  }
  CR(upload_table(ctx, ctx->d_tw_y, roots(g.Py)));
  CR(upload_table(ctx, ctx->d_tw_z, roots(g.Pz)));
  if (rc == MMP_OK) {
    mmp_shape sh;
    sh.ty = pick_tile_rows(g.ny, g.nz, g.Px);
    sh.tyc = 0;
    sh.radix_x = 0;
    sh.radix_y = 0;
    sh.R = pick_residues(g);
    sh.stage_kernel = 1;
    sh.engine = 0;
    // the warp pass B where it applies: one CTA per plane up to Py = 1024,
    // a two-CTA cluster at Py = 2048
    const int Rw = g.Py > 1024 ? 2 : 1;
    if (passb_w_supported(g, Rw)) {
      sh.R = Rw;
      sh.stage_kernel = 0;
      sh.engine = MMP_ENGINE_WARP_B;
    }
    if (xw_supported(g)) sh.engine |= MMP_ENGINE_WARP_X;
    if (sh.R == 0) rc = fail(MMP_E_INVAL, "y-z plane of %d x %d too large for pass B", ny, nz);
    else rc = apply_shape(ctx, sh);
  }
#undef CR
  if (rc == MMP_OK) rc = ensure_state(ctx);
  if (rc != MMP_OK) {
    std::string msg = g_err;
    mmp_destroy(ctx);
    g_err = msg;
    return rc;
  }
  *out = ctx;
  return MMP_OK;
}

int mmp_destroy(mmp_ctx* ctx) {
  if (!ctx) return MMP_OK;
  cudaStreamSynchronize(ctx->stream);
  release_khat(ctx);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
  for (cudaEvent_t ev : ctx->gev)
    if (ev) cudaEventDestroy(ev);
  void* bufs[] = {ctx->d_regions, ctx->d_coef, ctx->d_hA, ctx->d_y, ctx->d_stage, ctx->d_B, ctx->d_eps,
                  ctx->d_sig, ctx->d_T, ctx->d_tw_x, ctx->d_tw_y, ctx->d_tw_ly, ctx->d_tw_z, ctx->d_red,
                  ctx->d_energy, ctx->d_tw_wy, ctx->d_tw_wx, ctx->d_tw_wx2, ctx->d_tw_tc, ctx->d_flag};
  for (void* p : bufs) dfree(ctx, p);
  for (int i = 0; i < 7; ++i) dfree(ctx, ctx->d_k[i]);
  if (ctx->h_red) cudaFreeHost(ctx->h_red);
  for (int k = 0; k < MMP_NKERNEL; ++k)
    for (auto& pr : ctx->prof_events[k]) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  delete ctx;
  return MMP_OK;
}

int mmp_set_region_map(mmp_ctx* ctx, const uint8_t* regions) {
  TRY(check_ctx(ctx));
  if (!regions) return fail(MMP_E_INVAL, "regions is null");
  const long long n = ctx->g.n;
  std::vector<uint8_t> host(n);
  CK(cudaMemcpyAsync(host.data(), regions, n, cudaMemcpyDefault, ctx->stream), "copy regions");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  bool uni = std::all_of(host.begin(), host.end(), [](uint8_t r) { return r == 0; });
  for (int r = 0; r < MMP_MAX_REGIONS; ++r) ctx->used[r] = false;
  for (uint8_t r : host) ctx->used[r] = true;
  if (!ctx->d_regions) TRY(alloc_into(ctx, ctx->d_regions, n));
  CK(cudaMemcpyAsync(ctx->d_regions, host.data(), n, cudaMemcpyHostToDevice, ctx->stream), "upload regions");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  ctx->uniform = uni;
  ctx->coef_dirty = true;
  ctx->k1_valid = false;
  ctx->config_gen++;
  return MMP_OK;
}

int mmp_set_param(mmp_ctx* ctx, int sub, int param, int region, double value) {
  TRY(check_ctx(ctx));
  if (param < 0 || param >= MMP_NPARAM) return fail(MMP_E_INVAL, "unknown parameter %d", param);
  if (sub < -1 || sub >= ctx->nsub) return fail(MMP_E_INVAL, "bad sublattice %d", sub);
  if (region < -1 || region >= MMP_MAX_REGIONS) return fail(MMP_E_INVAL, "bad region %d", region);
  if (!std::isfinite(value)) return fail(MMP_E_INVAL, "non-finite value");
  if (param == MMP_MS && value < 0) return fail(MMP_E_INVAL, "Ms must be >= 0");
  for (int s = 0; s < ctx->nsub; ++s) {
    if (sub >= 0 && s != sub) continue;
    for (int r = 0; r < MMP_MAX_REGIONS; ++r)
      if (region < 0 || r == region) ctx->scal[param][s][r] = value;
  }
  ctx->coef_dirty = true;
  ctx->k1_valid = false;
  return MMP_OK;
}

int mmp_set_param3(mmp_ctx* ctx, int sub, int param, int region, double x, double y, double z) {
  TRY(check_ctx(ctx));
  if (param < 0 || param >= MMP_NPARAM3) return fail(MMP_E_INVAL, "unknown vector parameter %d", param);
  if (sub < -1 || sub >= ctx->nsub) return fail(MMP_E_INVAL, "bad sublattice %d", sub);
  if (region < -1 || region >= MMP_MAX_REGIONS) return fail(MMP_E_INVAL, "bad region %d", region);
  if (!std::isfinite(x) || !std::isfinite(y) || !std::isfinite(z)) return fail(MMP_E_INVAL, "non-finite value");
  for (int s = 0; s < ctx->nsub; ++s) {
    if (sub >= 0 && s != sub) continue;
    for (int r = 0; r < MMP_MAX_REGIONS; ++r)
      if (region < 0 || r == region) {
        ctx->vec[param][s][r][0] = x;
        ctx->vec[param][s][r][1] = y;
        ctx->vec[param][s][r][2] = z;
      }
  }
  ctx->coef_dirty = true;
  ctx->k1_valid = false;
  return MMP_OK;
}

int mmp_set_global(mmp_ctx* ctx, int param, double value) {
  TRY(check_ctx(ctx));
  if (param < 0 || param >= MMP_NGLOBAL) return fail(MMP_E_INVAL, "unknown global %d", param);
  if (!std::isfinite(value)) return fail(MMP_E_INVAL, "non-finite value");
  ctx->glob[param] = value;
  ctx->coef_dirty = true;
  ctx->k1_valid = false;
  ctx->config_gen++;
  return MMP_OK;
}

int mmp_set_boundary(mmp_ctx* ctx, int bc) {
  TRY(check_ctx(ctx));
  if (bc != MMP_BC_NEUMANN && bc != MMP_BC_OPEN) return fail(MMP_E_INVAL, "unsupported boundary condition %d", bc);
  ctx->bc = bc;
  ctx->k1_valid = false;
  ctx->config_gen++;
  return MMP_OK;
}

int mmp_enable_terms(mmp_ctx* ctx, unsigned terms) {
  TRY(check_ctx(ctx));
  if (terms & ~511u) return fail(MMP_E_INVAL, "unknown term bits 0x%x", terms);
  ctx->terms = terms;
  ctx->k1_valid = false;
  ctx->config_gen++;
  return ensure_state(ctx);
}

int mmp_set_m(mmp_ctx* ctx, int sub, const float* m, int normalize) {
  TRY(check_ctx(ctx));
  if (sub < 0 || sub >= ctx->nsub) return fail(MMP_E_INVAL, "bad sublattice %d", sub);
  if (!m) return fail(MMP_E_INVAL, "m is null");
  TRY(ensure_state(ctx));
  float* dst = ctx->d_y + 3LL * sub * ctx->g.n;
  CK(cudaMemcpyAsync(dst, m, 3LL * ctx->g.n * sizeof(float), cudaMemcpyDefault, ctx->stream), "copy m");
  if (normalize) CK(launch_normalize(dst, ctx->g.n, ctx->stream), "normalize");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  ctx->k1_valid = false;
  return MMP_OK;
}

int mmp_get_m(mmp_ctx* ctx, int sub, float* m) {
  TRY(check_ctx(ctx));
  if (sub < 0 || sub >= ctx->nsub) return fail(MMP_E_INVAL, "bad sublattice %d", sub);
  if (!m) return fail(MMP_E_INVAL, "m is null");
  CK(cudaMemcpyAsync(m, ctx->d_y + 3LL * sub * ctx->g.n, 3LL * ctx->g.n * sizeof(float), cudaMemcpyDefault,
                     ctx->stream),
     "copy m");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  return MMP_OK;
}

int mmp_set_elastic(mmp_ctx* ctx, const float* u, const float* v) {
  TRY(check_ctx(ctx));
  if (!has(ctx, MMP_T_ELASTIC)) return fail(MMP_E_STATE, "enable MMP_T_ELASTIC first");
  TRY(ensure_state(ctx));
  const long long n3 = 3LL * ctx->g.n;
  float* base = ctx->d_y + 3LL * ctx->nsub * ctx->g.n;
  if (u) CK(cudaMemcpyAsync(base, u, n3 * sizeof(float), cudaMemcpyDefault, ctx->stream), "copy u");
  if (v) CK(cudaMemcpyAsync(base + n3, v, n3 * sizeof(float), cudaMemcpyDefault, ctx->stream), "copy v");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  ctx->k1_valid = false;
  return MMP_OK;
}

int mmp_get_elastic(mmp_ctx* ctx, float* u, float* v) {
  TRY(check_ctx(ctx));
  if (!has(ctx, MMP_T_ELASTIC)) return fail(MMP_E_STATE, "elastic term is off");
  const long long n3 = 3LL * ctx->g.n;
  const float* base = ctx->d_y + 3LL * ctx->nsub * ctx->g.n;
  if (u) CK(cudaMemcpyAsync(u, base, n3 * sizeof(float), cudaMemcpyDefault, ctx->stream), "copy u");
  if (v) CK(cudaMemcpyAsync(v, base + n3, n3 * sizeof(float), cudaMemcpyDefault, ctx->stream), "copy v");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  return MMP_OK;
}

int mmp_set_solver(mmp_ctx* ctx, int method, int adaptive, double dt, double tol, double dt_min, double dt_max) {
  TRY(check_ctx(ctx));
  if (method < MMP_DP45 || method > MMP_RKF45) return fail(MMP_E_INVAL, "unknown method %d", method);
  if (!(dt > 0) || !(dt_min > 0) || !(dt_max >= dt_min) || (adaptive && !(tol > 0)))
    return fail(MMP_E_INVAL, "bad solver settings");
  if (method != ctx->method) ctx->k1_valid = false;
  ctx->method = method;
  ctx->adaptive = adaptive ? 1 : 0;
  ctx->dt = dt;
  ctx->tol = tol;
  ctx->dt_min = dt_min;
  ctx->dt_max = dt_max;
  return MMP_OK;
}

int mmp_eval_field(mmp_ctx* ctx, int sub, float* B, float* tau) {
  TRY(check_ctx(ctx));
  if (sub < 0 || sub >= ctx->nsub) return fail(MMP_E_INVAL, "bad sublattice %d", sub);
  TRY(prepare(ctx));
  if (B && !ctx->d_B) TRY(alloc_into(ctx, ctx->d_B, 3LL * ctx->nsub * ctx->g.n * sizeof(float)));
  StageArgs sa;
  memset(&sa, 0, sizeof sa);
  TRY(evaluate(ctx, sa, ctx->d_y, ctx->d_k[0], B ? ctx->d_B : nullptr, nullptr, nullptr, nullptr, 0, nullptr));
  ctx->k1_valid = true;
  ctx->k1_relax = 0;
  const long long n3 = 3LL * ctx->g.n;
  if (B) CK(cudaMemcpyAsync(B, ctx->d_B + sub * n3, n3 * sizeof(float), cudaMemcpyDefault, ctx->stream), "copy B");
  if (tau)
    CK(cudaMemcpyAsync(tau, ctx->d_k[0] + sub * n3, n3 * sizeof(float), cudaMemcpyDefault, ctx->stream),
       "copy tau");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  return check_flag(ctx);
}

int mmp_step(mmp_ctx* ctx, int nsteps) {
  TRY(check_ctx(ctx));
  if (nsteps < 0) return fail(MMP_E_INVAL, "nsteps < 0");
  return advance(ctx, nsteps, -1.0, 0, 0.0, 0.0, nullptr);
}

int mmp_run(mmp_ctx* ctx, double duration) {
  TRY(check_ctx(ctx));
  if (!(duration >= 0)) return fail(MMP_E_INVAL, "duration must be >= 0");
  return advance(ctx, 0, ctx->t + duration, 0, 0.0, 0.0, nullptr);
}

int mmp_relax(mmp_ctx* ctx, double torque_tol, double max_time, double timeout_s) {
  TRY(check_ctx(ctx));
  if (!(torque_tol > 0) || !(max_time > 0)) return fail(MMP_E_INVAL, "bad relax settings");
  bool conv = false;
  int rc = advance(ctx, 0, ctx->t + max_time, 1, torque_tol, timeout_s, &conv);
  ctx->k1_valid = false;   // k1 holds the damping-only torque
  return rc;
}

int mmp_get_time(mmp_ctx* ctx, double* t, double* dt, long long* steps, long long* rejected, long long* evals) {
  TRY(check_ctx(ctx));
  if (t) *t = ctx->t;
  if (dt) *dt = ctx->dt;
  if (steps) *steps = ctx->steps;
  if (rejected) *rejected = ctx->rejected;
  if (evals) *evals = ctx->evals;
  return MMP_OK;
}

namespace {
struct BlobHeader {
  char magic[8];
  int version, nsub, nparts, pad;
  long long n, steps, rejected, evals;
  double t, dt;
};
}  // namespace

int mmp_get_state(mmp_ctx* ctx, void* blob, size_t* size) {
  TRY(check_ctx(ctx));
  if (!size) return fail(MMP_E_INVAL, "size is null");
  TRY(ensure_state(ctx));
  size_t need = sizeof(BlobHeader) + ctx->nstate * sizeof(float);
  if (!blob) { *size = need; return MMP_OK; }
  if (*size < need) return fail(MMP_E_INVAL, "blob too small (%zu < %zu)", *size, need);
  BlobHeader h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, "MMPSTATE", 8);
  h.version = MMP_VERSION;
  h.nsub = ctx->nsub;
  h.nparts = ctx->nparts;
  h.n = ctx->g.n;
  h.steps = ctx->steps;
  h.rejected = ctx->rejected;
  h.evals = ctx->evals;
  h.t = ctx->t;
  h.dt = ctx->dt;
  memcpy(blob, &h, sizeof h);
  CK(cudaMemcpyAsync(static_cast<char*>(blob) + sizeof h, ctx->d_y, ctx->nstate * sizeof(float),
                     cudaMemcpyDeviceToHost, ctx->stream),
     "copy state");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  *size = need;
  return MMP_OK;
}

int mmp_set_state(mmp_ctx* ctx, const void* blob, size_t size) {
  TRY(check_ctx(ctx));
  if (!blob || size < sizeof(BlobHeader)) return fail(MMP_E_INVAL, "blob too small");
  BlobHeader h;
  memcpy(&h, blob, sizeof h);
  if (memcmp(h.magic, "MMPSTATE", 8) != 0 || h.version != MMP_VERSION) return fail(MMP_E_INVAL, "not a state blob");
  TRY(ensure_state(ctx));
  if (h.nsub != ctx->nsub || h.nparts != ctx->nparts || h.n != ctx->g.n)
    return fail(MMP_E_INVAL, "state blob does not match the context");
  if (size < sizeof h + ctx->nstate * sizeof(float)) return fail(MMP_E_INVAL, "blob truncated");
  CK(cudaMemcpyAsync(ctx->d_y, static_cast<const char*>(blob) + sizeof h, ctx->nstate * sizeof(float),
                     cudaMemcpyHostToDevice, ctx->stream),
     "copy state");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  ctx->t = h.t;
  ctx->dt = h.dt;
  ctx->steps = h.steps;
  ctx->rejected = h.rejected;
  ctx->evals = h.evals;
  ctx->k1_valid = false;
  return MMP_OK;
}

int mmp_profile(mmp_ctx* ctx, int enable) {
  TRY(check_ctx(ctx));
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  for (int k = 0; k < MMP_NKERNEL; ++k) ctx->prof_used[k] = 0;
  ctx->prof = enable != 0;
  return MMP_OK;
}

int mmp_profile_read(mmp_ctx* ctx, int kernel, long long* launches, double* total_ms) {
  TRY(check_ctx(ctx));
  if (kernel < 0 || kernel >= MMP_NKERNEL) return fail(MMP_E_INVAL, "unknown kernel %d", kernel);
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  double tot = 0.0;
  for (size_t i = 0; i < ctx->prof_used[kernel]; ++i) {
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, ctx->prof_events[kernel][i].first, ctx->prof_events[kernel][i].second),
       "event time");
    tot += ms;
  }
  if (launches) *launches = (long long)ctx->prof_used[kernel];
  if (total_ms) *total_ms = tot;
  return MMP_OK;
}

int mmp_energy(mmp_ctx* ctx, double* e_terms) {
  TRY(check_ctx(ctx));
  if (!e_terms) return fail(MMP_E_INVAL, "e_terms is null");
  TRY(prepare(ctx));
  const long long n = ctx->g.n;
  if (!ctx->d_energy) TRY(alloc_into(ctx, ctx->d_energy, MMP_NTERMS * sizeof(double)));
  CK(cudaMemsetAsync(ctx->d_energy, 0, MMP_NTERMS * sizeof(double), ctx->stream), "reset energy");
  const unsigned terms = ctx->terms;
  if (terms & MMP_T_DEMAG) {
    // B_demag of every sublattice: an evaluation with the demag term alone
    // (torque into the stage buffer, which holds nothing between steps)
    if (!ctx->d_B) TRY(alloc_into(ctx, ctx->d_B, 3LL * ctx->nsub * n * sizeof(float)));
    const long long evals = ctx->evals;
    ctx->terms = MMP_T_DEMAG;
    StageArgs sa;
    memset(&sa, 0, sizeof sa);
    int rc = evaluate(ctx, sa, ctx->d_y, ctx->d_stage, ctx->d_B, nullptr, nullptr, nullptr, 0, nullptr);
    ctx->terms = terms;
    ctx->evals = evals;
    TRY(rc);
  }
  const bool strain = (terms & (MMP_T_MEL | MMP_T_ELASTIC)) != 0;
  if (strain) {
    ElasticArgs ea;
    memset(&ea, 0, sizeof ea);
    ea.stage = ctx->d_y;
    ea.eps = ctx->d_eps;
    ea.sig = ctx->d_sig;
    ea.c11 = (float)ctx->glob[MMP_C11];
    ea.c12 = (float)ctx->glob[MMP_C12];
    ea.c44 = (float)ctx->glob[MMP_C44];
    ea.terms = terms;
    CK(launch_strain(ctx->g, ea, ctx->nsub, ctx->stream), "strain");
  }
  EnergyArgs a;
  memset(&a, 0, sizeof a);
  a.m = ctx->d_y;
  a.Bd = (terms & MMP_T_DEMAG) ? ctx->d_B : nullptr;
  a.eps = strain ? ctx->d_eps : nullptr;
  a.sig = (terms & MMP_T_ELASTIC) ? ctx->d_sig : nullptr;
  a.vel = (terms & MMP_T_ELASTIC) ? ctx->d_y + 3LL * (ctx->nsub + 1) * n : nullptr;
  a.out = ctx->d_energy;
  a.terms = terms;
  a.nsub = ctx->nsub;
  a.dV = ctx->cell[0] * ctx->cell[1] * ctx->cell[2];
  a.a12 = ctx->glob[MMP_A12];
  a.a0c = ctx->glob[MMP_LATTICE_A] > 0 ? 4.0 * ctx->glob[MMP_A0] / (ctx->glob[MMP_LATTICE_A] * ctx->glob[MMP_LATTICE_A]) : 0.0;
  a.rho = ctx->glob[MMP_RHO];
  CK(launch_energy(ctx->g, coefs(ctx), a, ctx->stream), "energy");
  CK(cudaMemcpyAsync(e_terms, ctx->d_energy, MMP_NTERMS * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
     "read energy");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  return MMP_OK;
}

int mmp_get_shape(mmp_ctx* ctx, mmp_shape* out) {
  TRY(check_ctx(ctx));
  if (!out) return fail(MMP_E_INVAL, "out is null");
  *out = current_shape(ctx);
  return MMP_OK;
}

int mmp_set_shape(mmp_ctx* ctx, const mmp_shape* shape) {
  TRY(check_ctx(ctx));
  if (!shape) return fail(MMP_E_INVAL, "shape is null");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  return apply_shape(ctx, *shape);
}

int mmp_autotune(mmp_ctx* ctx, int flags, mmp_shape* chosen, double* eval_ms) {
  TRY(check_ctx(ctx));
  if (flags & ~(MMP_TUNE_BATCH | MMP_TUNE_FORCE)) return fail(MMP_E_INVAL, "unknown flags 0x%x", flags);
  if (!has(ctx, MMP_T_DEMAG)) return fail(MMP_E_INVAL, "autotune needs the demag term (it tunes the FFT passes)");
  TRY(prepare(ctx));
  const bool batch = (flags & MMP_TUNE_BATCH) != 0;
  const auto key = std::make_tuple(ctx->g.nx, ctx->g.ny, ctx->g.nz, ctx->nsub, batch ? 1 : 0);
  const int reps = 4;
  double ta = 0, tb = 0, tc = 0;
  if (!(flags & MMP_TUNE_FORCE)) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      TRY(apply_shape(ctx, it->second));
      if (chosen) *chosen = it->second;
      if (eval_ms) {
        TRY(time_passes(ctx, reps, &ta, &tb, &tc));
        *eval_ms = ta + tb + tc;
      }
      return MMP_OK;
    }
  }
  const char* why = "";
  mmp_shape start = current_shape(ctx);
  if (batch) {
    start.R = 1;
    start.stage_kernel = 0;
    start.engine = 0;   // batch members run the block engine
    start.ty = 8;   // the largest tiles that fit
    while (start.ty > 2 && !shape_ok(ctx, start, &why)) start.ty >>= 1;
    if (!shape_ok(ctx, start, &why)) return fail(MMP_E_INVAL, "no batch shape fits this grid: %s", why);
  }
  TRY(apply_shape(ctx, start));
  // warm-up: at least ~100 ms of evaluations, so that every candidate is
  // timed at the clocks of a loaded GPU
  for (int w = 0; w < 200; ++w) {
    TRY(time_passes(ctx, 4, &ta, &tb, &tc));
    if ((w + 1) * 4 * (ta + tb + tc) > 100.0) break;
  }
  // candidates: passes A and C (tile rows, x plan) with pass B as started;
  // pass B (residues, kernel staging, y plan) with A and C as started
  std::vector<mmp_shape> cand_ac, cand_b;
  for (int ty : {2, 4, 8})
    for (int tyc : {2, 4, 8})
      for (int rx = 0; rx < 2; ++rx) {
        if (batch && ty != start.ty) continue;   // a batch gets its parallelism from its members
        mmp_shape s = start;
        s.ty = ty;
        s.tyc = tyc;
        s.radix_x = rx;
        s.engine &= ~MMP_ENGINE_WARP_X;
        if (shape_ok(ctx, s, &why)) cand_ac.push_back(s);
      }
  if (!batch) {
    mmp_shape s = start;
    s.engine |= MMP_ENGINE_WARP_X;
    if (shape_ok(ctx, s, &why)) cand_ac.push_back(s);
  }
  for (int R : {1, 2, 4, 8})
    for (int st = 0; st < 2; ++st)
      for (int ry = 0; ry < 2; ++ry) {
        if (batch && (R != 1 || st != 0)) continue;
        mmp_shape s = start;
        s.R = R;
        s.stage_kernel = st;
        s.radix_y = ry;
        s.engine &= ~(MMP_ENGINE_WARP_B | MMP_ENGINE_TC_Y);
        if (shape_ok(ctx, s, &why)) cand_b.push_back(s);
      }
  for (int R : {1, 2})
    for (int tc = 0; tc < 2; ++tc) {
      if (batch) break;
      mmp_shape s = start;
      s.R = R;
      s.stage_kernel = 0;
      s.radix_y = 0;
      s.engine = (s.engine & ~MMP_ENGINE_TC_Y) | MMP_ENGINE_WARP_B | (tc ? MMP_ENGINE_TC_Y : 0);
      if (shape_ok(ctx, s, &why)) cand_b.push_back(s);
    }
  // two interleaved rounds; a candidate's time is its better round
  std::vector<double> t_ac(cand_ac.size(), 1e300), t_b(cand_b.size(), 1e300);
  for (int round = 0; round < 2; ++round) {
    for (size_t i = 0; i < cand_ac.size(); ++i) {
      TRY(apply_shape(ctx, cand_ac[i]));
      TRY(time_passes(ctx, reps, &ta, &tb, &tc));
      t_ac[i] = std::min(t_ac[i], ta + tc);
    }
    for (size_t i = 0; i < cand_b.size(); ++i) {
      TRY(apply_shape(ctx, cand_b[i]));
      TRY(time_passes(ctx, reps, &ta, &tb, &tc));
      t_b[i] = std::min(t_b[i], tb);
    }
  }
  mmp_shape best = start;
  double best_ac = 1e300, best_b = 1e300;
  for (size_t i = 0; i < cand_ac.size(); ++i)
    if (t_ac[i] < best_ac) {
      best_ac = t_ac[i];
      best.ty = cand_ac[i].ty;
      best.tyc = cand_ac[i].tyc;
      best.radix_x = cand_ac[i].radix_x;
      best.engine = (best.engine & ~MMP_ENGINE_WARP_X) | (cand_ac[i].engine & MMP_ENGINE_WARP_X);
    }
  for (size_t i = 0; i < cand_b.size(); ++i)
    if (t_b[i] < best_b) {
      best_b = t_b[i];
      best.R = cand_b[i].R;
      best.stage_kernel = cand_b[i].stage_kernel;
      best.radix_y = cand_b[i].radix_y;
      best.engine = (best.engine & ~(MMP_ENGINE_WARP_B | MMP_ENGINE_TC_Y)) |
                    (cand_b[i].engine & (MMP_ENGINE_WARP_B | MMP_ENGINE_TC_Y));
    }
  // keep the starting shape unless the combination measures faster by > 2 %
  // (longer, interleaved measurement of both)
  double t_start = 1e300, t_best = 1e300;
  for (int round = 0; round < 2; ++round) {
    TRY(apply_shape(ctx, start));
    TRY(time_passes(ctx, 2 * reps, &ta, &tb, &tc));
    t_start = std::min(t_start, ta + tb + tc);
    TRY(apply_shape(ctx, best));
    TRY(time_passes(ctx, 2 * reps, &ta, &tb, &tc));
    t_best = std::min(t_best, ta + tb + tc);
  }
  if (!(t_best < 0.98 * t_start)) {
    best = start;
    t_best = t_start;
  }
  best_ac = t_best;
  best_b = 0.0;
  TRY(apply_shape(ctx, best));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best;
  }
  if (chosen) *chosen = best;
  if (eval_ms) *eval_ms = best_ac + best_b;
  return MMP_OK;
}

int mmp_sync(mmp_ctx* ctx) {
  TRY(check_ctx(ctx));
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  return check_flag(ctx);
}

}  // extern "C"

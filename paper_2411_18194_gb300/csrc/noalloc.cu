// noalloc.cu -- the demagnetising field of a caller-given magnetisation
// without any device allocation.
//
// Some callers cannot call cudaMalloc: code running where the device memory
// is owned and budgeted by someone else (a host framework whose allocator
// must not be bypassed, a real-time loop that must not allocate after start,
// a sandbox that forbids allocation calls).  For them this entry point keeps
// all its working memory -- the x-transformed spectrum, the demag kernel
// octant, the FP64 buffers that build it, twiddle tables, a coefficient
// table and a torque buffer the field pass writes -- in one file-scope
// static device array of MMP_NOALLOC_SCRATCH_BYTES.  Every GPU that loads
// the library holds that array until the process exits.  The caller passes
// the input M and the output B.
//
// In host code the array's name is only a stand-in, not a device address:
// its address is looked up with cudaGetSymbolAddress once per device, with
// that device current, and cached.
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "kernels.h"
#include "mmp.h"
#include "plan.h"

namespace mmp {
int report_error(int code, const char* msg);
}  // namespace mmp

using namespace mmp;

namespace {

static __device__ __align__(256) unsigned char g_scratch[MMP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;

struct Setup {
  bool have_base = false;
  unsigned char* base = nullptr;   // device address of g_scratch on this device
  bool ready = false;              // tables built for the geometry below
  int n[3] = {0, 0, 0};
  double cell[3] = {0, 0, 0};
  Grid g;
  DemagArgs d;
  Coefs co;
  float* tau = nullptr;
  int thrA = 0, thrB = 0, thrC = 0;
};

Setup g_setup[kMaxDevices];
std::mutex g_mu;

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Layout {
  size_t T, khat, buf0, buf1, trig[3], tw_x, tw_y, tw_ly, tw_z, coef, tau, total;
};

Layout plan_layout(const Grid& g, int R) {
  Layout L;
  size_t at = 0;
  auto take = [&](size_t bytes) { size_t o = at; at = up256(at + bytes); return o; };
  const long long nk = (long long)g.kxn * g.kyn * g.kzn;
  const long long ext = std::max<long long>({(long long)g.nx * g.ny * g.nz, (long long)g.kxn * g.ny * g.nz,
                                             (long long)g.kxn * g.kyn * g.nz, nk});
  L.T = take((size_t)g.kxn * 3 * g.nz * g.ny * sizeof(float2));
  L.khat = take((size_t)g.kxn * g.kyn * g.krow * sizeof(float));
  L.buf0 = take((size_t)ext * 6 * sizeof(double));
  L.buf1 = take((size_t)ext * 6 * sizeof(double));
  const int P[3] = {g.Px, g.Py, g.Pz};
  for (int a = 0; a < 3; ++a) L.trig[a] = take((size_t)P[a] * sizeof(double2));
  L.tw_x = take((size_t)g.Px * sizeof(float2));
  L.tw_y = take((size_t)g.Py * sizeof(float2));
  L.tw_ly = take((size_t)(g.Py / R) * sizeof(float2));
  L.tw_z = take((size_t)g.Pz * sizeof(float2));
  L.coef = take((size_t)2 * MMP_MAX_REGIONS * sizeof(RegionCoef));
  L.tau = take((size_t)3 * g.n * sizeof(float));
  L.total = at;
  return L;
}

int err(int code, const char* msg) { return report_error(code, msg); }

int cuda_err(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  return err(MMP_E_CUDA, buf);
}

// Build the tables of one geometry into the scratch of the current device
// (host-to-device copies, the FP64 kernel build, one synchronisation).
int set_up(Setup& S, int nx, int ny, int nz, const double* cell, cudaStream_t s) {
  Grid g;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.n = (long long)nx * ny * nz;
  g.Px = nice_length(nx); g.Py = nice_length(ny); g.Pz = nice_length(nz);
  g.kxn = g.Px / 2 + 1; g.kyn = g.Py / 2 + 1; g.kzn = g.Pz / 2 + 1;
  g.krow = (6 * g.kzn + 3) & ~3;
  g.ty = pick_tile_rows(g.ny, g.nz, g.Px);
  g.xb = 1;
  g.tyc = pick_tile_rows_c(g.ty, g.Px);
  g.xbc = 1;
  for (int a = 0; a < 3; ++a) {
    g.h[a] = (float)cell[a];
    g.ih[a] = (float)(1.0 / cell[a]);
  }
  if (g.Px > 4096 || g.Py > 4096 || g.Pz > 32)
    return err(MMP_E_INVAL, "demag: padded lengths must be <= 4096 (x, y) and nz <= 16");
  const int R = pick_residues(g);
  if (R == 0) return err(MMP_E_INVAL, "y-z plane too large for pass B");
  DemagArgs d;
  memset(&d, 0, sizeof d);
  if (!make_plan(g.Px, d.plan_x) || !make_plan(g.Py / R, d.plan_ly)) return err(MMP_E_INVAL, "unsupported FFT length");
  const Layout L = plan_layout(g, R);
  if (L.total > (size_t)MMP_NOALLOC_SCRATCH_BYTES) {
    char buf[200];
    snprintf(buf, sizeof buf, "grid needs %zu bytes of scratch, more than the %d bytes of mmp_demag_noalloc",
             L.total, MMP_NOALLOC_SCRATCH_BYTES);
    return err(MMP_E_INVAL, buf);
  }
  unsigned char* b = S.base;
  auto put = [&](size_t off, const void* src, size_t bytes) {
    return cudaMemcpyAsync(b + off, src, bytes, cudaMemcpyHostToDevice, s);
  };
  cudaError_t e = cudaSuccess;
  std::vector<float2> wx = pass_twiddles(d.plan_x), wy = roots(g.Py), wly = pass_twiddles(d.plan_ly),
                     wz = roots(g.Pz);
  if (e == cudaSuccess) e = put(L.tw_x, wx.data(), wx.size() * sizeof(float2));
  if (e == cudaSuccess) e = put(L.tw_y, wy.data(), wy.size() * sizeof(float2));
  if (e == cudaSuccess) e = put(L.tw_ly, wly.data(), wly.size() * sizeof(float2));
  if (e == cudaSuccess) e = put(L.tw_z, wz.data(), wz.size() * sizeof(float2));
  const int P[3] = {g.Px, g.Py, g.Pz};
  std::vector<double2> trig[3];
  for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
    trig[a].resize(P[a]);
    for (int t = 0; t < P[a]; ++t) {
      double ang = 2.0 * 3.14159265358979323846 * (double)t / (double)P[a];
      trig[a][t] = make_double2(cos(ang), sin(ang));
    }
    e = put(L.trig[a], trig[a].data(), trig[a].size() * sizeof(double2));
  }
  // one region, Ms = 1: the stage fed to the passes is M itself
  std::vector<RegionCoef> rc(2 * MMP_MAX_REGIONS);
  memset(rc.data(), 0, rc.size() * sizeof(RegionCoef));
  rc[0].ms = 1.0f;
  rc[0].inv_ms = 1.0f;
  if (e == cudaSuccess) e = put(L.coef, rc.data(), rc.size() * sizeof(RegionCoef));
  if (e != cudaSuccess) return cuda_err(e, "mmp_demag_noalloc set-up copies");
  KernelBuild kb;
  kb.n[0] = nx; kb.n[1] = ny; kb.n[2] = nz;
  kb.P[0] = g.Px; kb.P[1] = g.Py; kb.P[2] = g.Pz;
  for (int a = 0; a < 3; ++a) {
    kb.cell[a] = cell[a];
    kb.trig[a] = reinterpret_cast<const double2*>(b + L.trig[a]);
  }
  kb.rc = 10.0;
  kb.buf0 = reinterpret_cast<double*>(b + L.buf0);
  kb.buf1 = reinterpret_cast<double*>(b + L.buf1);
  kb.out = reinterpret_cast<float*>(b + L.khat);
  kb.krow = g.krow;
  e = build_kernel_spectrum(kb, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(e, "mmp_demag_noalloc kernel build");
  d.T = reinterpret_cast<float2*>(b + L.T);
  d.khat = reinterpret_cast<const float*>(b + L.khat);
  d.tw_x = reinterpret_cast<const float2*>(b + L.tw_x);
  d.tw_y = reinterpret_cast<const float2*>(b + L.tw_y);
  d.tw_ly = reinterpret_cast<const float2*>(b + L.tw_ly);
  d.tw_z = reinterpret_cast<const float2*>(b + L.tw_z);
  d.R = R;
  S.g = g;
  S.d = d;
  S.co.reg = reinterpret_cast<const RegionCoef*>(b + L.coef);
  S.co.regions = nullptr;
  S.co.hA = nullptr;
  S.co.uniform = 1;
  S.tau = reinterpret_cast<float*>(b + L.tau);
  launch_threads(g, R, &S.thrA, &S.thrB, &S.thrC);
  S.n[0] = nx; S.n[1] = ny; S.n[2] = nz;
  for (int a = 0; a < 3; ++a) S.cell[a] = cell[a];
  S.ready = true;
  return MMP_OK;
}

}  // namespace

extern "C" int mmp_demag_noalloc(int nx, int ny, int nz, double cx, double cy, double cz, const float* M, float* B,
                                 void* stream) {
  if (nx < 1 || ny < 1 || nz < 1) return err(MMP_E_INVAL, "grid extents must be >= 1");
  if (!(cx > 0) || !(cy > 0) || !(cz > 0)) return err(MMP_E_INVAL, "cell sizes must be > 0");
  if (!M || !B) return err(MMP_E_INVAL, "M and B must be device pointers");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_err(e, "no CUDA device");
  }
  if (dev < 0 || dev >= kMaxDevices) return err(MMP_E_INVAL, "device index out of range");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mu);
  Setup& S = g_setup[dev];
  if (!S.have_base) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress of the scratch array");
    S.base = static_cast<unsigned char*>(p);
    S.have_base = true;
  }
  const double cell[3] = {cx, cy, cz};
  if (!S.ready || S.n[0] != nx || S.n[1] != ny || S.n[2] != nz || S.cell[0] != cx || S.cell[1] != cy ||
      S.cell[2] != cz) {
    S.ready = false;
    int rc = set_up(S, nx, ny, nz, cell, s);
    if (rc != MMP_OK) return rc;
  }
  StageArgs sa;
  memset(&sa, 0, sizeof sa);
  sa.stage = const_cast<float*>(M);
  sa.nparts = 1;
  sa.nsub = 1;
  FieldArgs f;
  memset(&f, 0, sizeof f);
  f.stage = M;
  f.kout = S.tau;
  f.Bout = B;
  f.terms = MMP_T_DEMAG;
  e = launch_passA(S.g, sa, S.d, S.co, S.thrA, s);
  if (e == cudaSuccess) e = launch_passB(S.g, S.d, S.thrB, s);
  if (e == cudaSuccess) e = launch_field(S.g, S.d, S.co, f, 1, true, S.thrC, s);
  if (e != cudaSuccess) return cuda_err(e, "mmp_demag_noalloc launch");
  return MMP_OK;
}

// ctx.h -- the context object behind the opaque mmp_ctx handle, shared by
// the per-context driver (mmp.cu) and the batched driver (batch.cu).
#pragma once
#include <cuda_runtime.h>

#include <tuple>
#include <utility>
#include <vector>

#include "kernels.h"
#include "mmp.h"

struct mmp_ctx {
  using Grid = mmp::Grid;
  using RegionCoef = mmp::RegionCoef;
  using FftPlan = mmp::FftPlan;
  Grid g;
  int nsub = 1;
  double cell[3];
  cudaStream_t stream = nullptr;
  mmp_alloc_fn ualloc = nullptr;
  mmp_free_fn ufree = nullptr;
  void* uuser = nullptr;
  bool poisoned = false;
  unsigned terms = 0;
  int bc = MMP_BC_NEUMANN;        // boundary condition of the exchange and DMI stencils
  // parameter tables (FP64)
  double scal[MMP_NPARAM][2][MMP_MAX_REGIONS];
  double vec[MMP_NPARAM3][2][MMP_MAX_REGIONS][3];
  double glob[MMP_NGLOBAL];
  bool uniform = true;
  bool used[MMP_MAX_REGIONS] = {true};   // regions present in the map
  bool coef_dirty = true, khat_dirty = true;
  // device buffers
  uint8_t* d_regions = nullptr;
  RegionCoef* d_coef = nullptr;
  float2* d_hA = nullptr;
  float* d_y = nullptr;
  float* d_stage = nullptr;
  float* d_k[7] = {};
  float* d_B = nullptr;
  float* d_eps = nullptr;
  float* d_sig = nullptr;
  float2* d_T = nullptr;
  float* d_khat = nullptr;     // shared spectrum (build_khat), not owned
  std::tuple<int, int, int, int, double, double, double> khat_key;
  float2 *d_tw_x = nullptr, *d_tw_y = nullptr, *d_tw_ly = nullptr, *d_tw_z = nullptr;
  float2* d_tw_wy = nullptr;   // warp pass B twiddles (engine & MMP_ENGINE_WARP_B)
  float2 *d_tw_wx = nullptr, *d_tw_wx2 = nullptr;   // warp passes A and C (MMP_ENGINE_WARP_X)
  float* d_tw_tc = nullptr;    // tensor-core DFT32 matrices (MMP_ENGINE_TC_Y)
  unsigned* d_flag = nullptr;  // set by a device wait that ran past its limit
  unsigned* d_red = nullptr;   // [0] error bits, [1] torque bits
  double* d_energy = nullptr;  // [MMP_NTERMS] (mmp_energy)
  unsigned* h_red = nullptr;   // pinned
  int nparts = 0;              // 3-vectors in the state
  long long nstate = 0;        // floats in the state
  FftPlan plan_x{}, plan_ly{};
  int R = 1, thrA = 256, thrB = 256, thrC = 256;
  int ks = 1;                  // pass B stages the kernel slice in shared memory
  int radix_x = 0, radix_y = 0;   // FFT plan variants (make_plan)
  int engine = 0;              // mmp_shape.engine
  // solver
  int method = 0;              // MMP_DP45, ... (dp45.h tableau)
  int adaptive = 0;
  double dt = 1e-13, tol = 1e-5, dt_min = 1e-18, dt_max = 1e-11;
  double t = 0.0;
  long long steps = 0, rejected = 0, evals = 0;
  bool k1_valid = false;
  int k1_relax = 0;
  // fixed-step graph (replay_pairs): two captured steps and what they assumed
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
  cudaGraphExec_t gexec = nullptr;
  float* g_y = nullptr;
  float* g_k0 = nullptr;
  double g_dt = 0.0;
  int g_method = -1, g_ks = 0;
  long long config_gen = 0, g_config_gen = -1;   // bumped by changes a graph would have baked in
  // tracing
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events[MMP_NKERNEL];
  size_t prof_used[MMP_NKERNEL] = {};
};

// Term word of the field kernels: the enabled terms plus the boundary bit.
inline unsigned kernel_terms(const mmp_ctx* c) {
  return c->terms | (c->bc == MMP_BC_OPEN ? mmp::kTermOpenBC : 0u);
}

namespace mmp {
// Allocate the state, upload coefficients, build the demag kernel spectrum
// (first use) -- everything an evaluation needs (mmp.cu).
int ctx_prepare(mmp_ctx* ctx);
// Record an error message for mmp_last_error() and return `code`.
int report_error(int code, const char* msg);
}  // namespace mmp

// kernels.h -- launch interface between the C-ABI layer (mmp.cu) and the
// device passes (passes.cu, tensor.cu).
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"
#include "fft.cuh"

namespace mmp {

// ---------------------------------------------------------------- tensor --
struct KernelBuild {
  int n[3];            // grid extents
  int P[3];            // padded lengths
  double cell[3];      // cell size (m)
  double rc;           // Newell/asymptotic cutoff in units of max(cell)
  double* buf0;        // FP64 scratch, 6 * max(extent products) doubles
  double* buf1;
  const double2* trig[3];   // (cos, sin)(2 pi t / P_a), device
  float* out;          // [Px/2+1][Py/2+1][krow], row = (kz, 6 components) + padding
  int krow;
};
cudaError_t build_kernel_spectrum(const KernelBuild& kb, cudaStream_t s);

// ------------------------------------------------------------ geometry ---
struct Grid {
  int nx, ny, nz;
  long long n;          // nx*ny*nz
  int Px, Py, Pz;       // padded lengths (1 on axes with n = 1)
  int kxn;              // Px/2 + 1
  int kyn, kzn;         // Py/2 + 1, Pz/2 + 1
  int krow;             // floats per (kx, ky) row of the kernel octant: 6 kzn rounded up to 4
  int ty;               // rows (y) per tile of passes A and C: 2, 4 or 8 (row pairs = ty / 2)
  int xb;               // components per x-FFT call of pass A: 3 (all at once) or 1
  int tyc;              // rows (y) per tile of pass C: 2, 4 or 8 (independent of pass A's)
  int xbc;              // components per x-FFT call of pass C: 3 or 1
  float h[3];           // cell size (m)
  float ih[3];          // 1 / h
  // bounds-checked build (MMP_CHECK_BOUNDS): the word the index checks set
  // (null: not checked) and the element counts they check against
  unsigned* chk;
  long long lim_state;  // floats of a state-shaped vector (y, k_j, stage, derivative): 3 parts n
  long long lim_B;      // floats of B_eff: 3 nsub n
  long long lim_T;      // complex elements of the spectrum T: kxn 3 nz ny
  long long lim_khat;   // floats of the kernel octant: kxn kyn krow
};

// Index checks of the bounds-checked build (compiled with -DMMP_CHECK_BOUNDS):
// an access whose element index falls outside its buffer is skipped and
// bit 1 of the context's flag word set, which the host reports as
// MMP_E_BOUNDS after the call.  In the normal build MMP_IN is `true` and
// the checks vanish.
#ifdef MMP_CHECK_BOUNDS
__device__ __forceinline__ bool in_bounds(const Grid& g, long long i, long long lim) {
  if (!g.chk || (i >= 0 && i < lim)) return true;
  atomicOr(g.chk, 2u);
  return false;
}
#define MMP_IN(g, i, lim) (::mmp::in_bounds((g), (long long)(i), (long long)(lim)))
#else
#define MMP_IN(g, i, lim) true
#endif

// State layout: one float vector per RK quantity,
//   [sub 0: m (3n)] [sub 1: m (3n)] [u (3n)] [v (3n)]   (u, v with elastic)
struct StageArgs {
  const float* y;            // state at the start of the step
  const float* k[7];         // previous stages (nk used)
  float coef[7];             // dt * a_ij (rounded from FP64)
  int nk;
  int normalize;             // renormalise m (the 5th-order stage)
  float* stage;              // output stage state
  int nparts;                // 3-vectors in the state (nsub, + 2 with elastic)
  int nsub;
};

struct DemagArgs {
  float2* T;                 // spectrum [kxn][3][nz][ny] complex
  const float* khat;         // kernel octant [kxn][kyn][krow] (krow >= 6 kzn, 16-byte rows)
  const float2* tw_x;        // pass-ordered twiddles of plan_x (Px entries)
  const float2* tw_y;        // Py roots
  const float2* tw_ly;       // pass-ordered twiddles of plan_ly (Ly = Py / R entries)
  const float2* tw_z;        // Pz roots
  FftPlan plan_x, plan_ly;
  int R;                     // residue classes of ky per cluster
  int ks;                    // pass B stages the kernel slice in shared memory
  // warp engine (wfft.cuh): twiddle tables w_N^(l k1) at [k1 * 32 + l]
  const float2* tw_wy;       // N = Ly (pass B)
  const float2* tw_wx;       // N = Px / 2 (passes A and C)
  const float2* tw_wx2;      // w_Px^x, x < Px / 2 (natural order; passes A and C)
  const float* tw_tc;        // tensor-core DFT32 matrices, split TF32 (tcdft.cuh layout)
  unsigned* err;             // set to 1 by a device wait that ran past its limit
  int engine;                // pass B: 0 block Stockham passes, 1 warp passes, 2 warp passes with
                             // the final DFT32 of each y transform on the tensor cores
};

struct Coefs {
  const RegionCoef* reg;     // [nsub][256]
  const uint8_t* regions;    // [n] or null when uniform
  const float2* hA;          // harmonic-mean A pair table [nsub][256][256] (multi-region)
  int uniform;
};

// Bit of the kernels' term word (above the public mmp_term bits): open
// boundary, a missing neighbour drops out of the exchange and DMI sums.
constexpr unsigned kTermOpenBC = 1u << 16;

struct FieldArgs {
  const float* stage;        // stage state
  float* kout;               // output derivative (same layout as the state)
  float* Bout;               // optional B_eff [nsub][3][n]
  const float* eps;          // strain [6][n] (magnetoelastic)
  unsigned terms;            // mmp_term bits | kTermOpenBC
  // error estimate of the 5th-order stage: err = max |sum_j e_j k_j|
  const float* ek[6];
  float ecoef[7];            // dt * (b_j - b*_j)
  unsigned* err;             // atomicMax target (float bits)
  int relax;                 // damping-only torque (relax mode)
  unsigned* torque_max;      // max |m x B| (float bits) in relax mode
};

struct ElasticArgs {
  const float* stage;        // stage state (u, v at parts nsub, nsub+1)
  float* kout;
  float* eps;                // [6][n] strain out
  float* sig;                // [6][n] stress out
  float c11, c12, c44, eta, inv_rho;
  unsigned terms;
};

// Energy of every field term (energy.cu): accumulators out[i] for the term
// with bit (1 << i), in J.
struct EnergyArgs {
  const float* m;          // state: sublattice parts first
  const float* Bd;         // demag field [nsub][3][n] (DEMAG) or null
  const float* eps;        // strain [6][n] (MEL, ELASTIC) or null
  const float* sig;        // stress [6][n] (ELASTIC) or null
  const float* vel;        // elastic velocity [3][n] (ELASTIC) or null
  double* out;             // [MMP_NTERMS] accumulators (J)
  unsigned terms;
  int nsub;
  double dV;
  double a12;              // A12 (J/m)
  double a0c;              // 4 A0 / a^2 (J/m^3)
  double rho;
};

// launchers (return cudaGetLastError())
cudaError_t launch_assemble(const Grid& g, const StageArgs& a, cudaStream_t s);
cudaError_t launch_passA(const Grid& g, const StageArgs& a, const DemagArgs& d, const Coefs& c,
                         int threads, cudaStream_t s);
cudaError_t launch_passB(const Grid& g, const DemagArgs& d, int threads, cudaStream_t s);
// warp pass B (passb_w.cuh) for Ly = Py / R = 32 M, M in {8, 16, 32}
template <int M>
cudaError_t launch_passB_w_len(const Grid& g, const DemagArgs& d, cudaStream_t s);
template <> cudaError_t launch_passB_w_len<8>(const Grid& g, const DemagArgs& d, cudaStream_t s);
template <> cudaError_t launch_passB_w_len<16>(const Grid& g, const DemagArgs& d, cudaStream_t s);
template <> cudaError_t launch_passB_w_len<32>(const Grid& g, const DemagArgs& d, cudaStream_t s);
// warp passes A and C (xfft_w.cuh): tiles of one row pair, Px = 2048
cudaError_t launch_passA_w(const Grid& g, const StageArgs& a, const DemagArgs& d, const Coefs& c, cudaStream_t s);
cudaError_t launch_field_w(const Grid& g, const DemagArgs& d, const Coefs& c, const FieldArgs& f, int nsub,
                           cudaStream_t s);
inline bool xw_supported(const Grid& g) { return g.Px == 2048; }
// whether the warp pass B handles this grid at residue count R
inline bool passb_w_supported(const Grid& g, int R) {
  if (R != 1 && R != 2) return false;
  if (g.Py % R != 0) return false;
  const int Ly = g.Py / R;
  if (Ly != 256 && Ly != 512 && Ly != 1024) return false;
  if (g.ny > Ly) return false;
  return g.nz == 1 || g.nz == 2 || g.nz == 4 || g.nz == 8;
}
// whether the tensor-core DFT32 stage applies on top of the warp pass B
inline bool passb_tc_supported(const Grid& g, int R) { return passb_w_supported(g, R); }
cudaError_t launch_field(const Grid& g, const DemagArgs& d, const Coefs& c, const FieldArgs& f,
                         int nsub, bool demag, int threads, cudaStream_t s);
cudaError_t launch_strain(const Grid& g, const ElasticArgs& e, int nsub, cudaStream_t s);
cudaError_t launch_elastic_rhs(const Grid& g, const ElasticArgs& e, const Coefs& c, int nsub,
                               cudaStream_t s);
cudaError_t launch_normalize(float* m, long long n, cudaStream_t s);
cudaError_t launch_energy(const Grid& g, const Coefs& co, const EnergyArgs& a, cudaStream_t s);

// Shared-memory carve-up of one pass-B CTA (bytes from the start).
struct PassBSmem {
  size_t twl, twf, twc, ks, total;
};

// The fold and recombination twiddles exist only for R > 1; the kernel
// slice only when it is staged (ks).
__host__ __device__ __forceinline__ PassBSmem passb_smem(int ny, int nz, int Py, int kzn, int R, bool ks) {
  const int Ly = Py / R;
  const int cnt = (ny + R - 1) / R;
  PassBSmem s;
  size_t at = (size_t)3 * nz * fft_pitch(Ly) * sizeof(float2);
  s.twl = at; at += (size_t)Ly * sizeof(float2);
  s.twf = at; if (R > 1) at += (size_t)Ly * sizeof(float2);
  s.twc = at; if (R > 1) at += (size_t)cnt * sizeof(float2);
  at = (at + 15) & ~(size_t)15;   // 16-byte rows for cp.async
  s.ks = at; if (ks) at += (size_t)Ly * ((6 * kzn + 3) & ~3) * sizeof(float);
  s.total = at;
  return s;
}

// shared memory bytes of each pass (host side planning)
size_t smem_passA(const Grid& g);
size_t smem_passB(const Grid& g, int R, bool ks);
size_t smem_field(const Grid& g, bool demag);

}  // namespace mmp

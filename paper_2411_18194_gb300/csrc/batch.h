// batch.h -- device side of the batched driver (batch.cu): the per-member
// descriptor, work items, and the pass kernels over a work list, one block
// per (member, tile) item, launched once per pass, z group and block-size
// class (batch_a.cu, batch_b.cu, batch_c.cu).
#pragma once
#include "kernels.h"

namespace mmp {

// Per-member descriptor (device copy read by the batched kernels).
struct BatchInst {
  Grid g;
  DemagArgs d;
  Coefs co;
  float* ybuf[2];      // state / stage ping-pong: y = ybuf[par], stage = ybuf[par ^ 1]
  float* kbuf[2];      // FSAL ping-pong: k1 = kbuf[par], k7 = kbuf[par ^ 1]
  float* kmid[5];      // k2 .. k6
  unsigned* red;       // [2]: error bits, torque bits of the attempt
  unsigned terms;
  int relax;           // damping-only torque
  int par;             // flipped on every accepted step
  int pad;
  float coef[7][7];    // coef[i][j] = dt a_ij, stage i = 1..6
  float ecoef[7];      // dt (b_j - b*_j)
};

struct BatchItem {
  int inst;            // member (index into the descriptor array)
  int a, b;            // passes A, C: (y tile, z); pass B: (kx, 0)
};

constexpr int kBatchThreads = 512;

// One launch of a pass over items[0, nitems), one block per item in list
// order (the list is sorted longest first, and the block scheduler hands
// blocks out in index order).  A persistent loop over an atomic counter was
// the first design; around these bodies it made the compiler cut the
// kernel to 64 registers and spill the FFT registers (kilobytes of stack).
// `stage`: 0 evaluates k1 at y (no assembly); 1..6 assemble stage i and
// evaluate k_{i+1}; stage 6 also forms the error estimate and torque
// maximum.
// `threads` <= kBatchThreads: the block size of the launch (items are
// grouped by the block size their member needs).
cudaError_t launch_batch_passA(const BatchInst* insts, const BatchItem* items, int nitems, int stage, int threads,
                               size_t smem, cudaStream_t s);
cudaError_t launch_batch_passB(int nz_group, const BatchInst* insts, const BatchItem* items, int nitems,
                               int threads, size_t smem, cudaStream_t s);
cudaError_t launch_batch_field(const BatchInst* insts, const BatchItem* items, int nitems, int stage, int threads,
                               size_t smem, cudaStream_t s);
cudaError_t launch_batch_accept(BatchInst* insts, int n, cudaStream_t s);
// Warp-engine members (batch_w.cu): passes A and C on row-pair tiles
// (Px = 2048), pass B on warp transforms of folded y length Py / R = 1024;
// one launch per pass (`kind` 0 = A, 1 = B, 2 = C) and member `inst`.
bool batch_warp_supported(const Grid& g, int R);
cudaError_t batch_warp_prepare();   // shared-memory attributes (outside graph capture)
cudaError_t launch_batch_warp(int kind, const BatchInst* insts, int inst, const Grid& g, int R, int stage,
                              cudaStream_t s);

// Stage and field arguments of item descriptor `I` at stage `stage`
// (built by one thread into shared memory).
__device__ __forceinline__ void batch_args(const BatchInst& I, int stage, StageArgs& sa, FieldArgs& fa) {
  const int p = I.par;
  float* kk[7] = {I.kbuf[p], I.kmid[0], I.kmid[1], I.kmid[2], I.kmid[3], I.kmid[4], I.kbuf[p ^ 1]};
  memset(&sa, 0, sizeof sa);
  memset(&fa, 0, sizeof fa);
  sa.nparts = 1;
  sa.nsub = 1;
  if (stage == 0) {
    sa.stage = I.ybuf[p];
  } else {
    sa.y = I.ybuf[p];
    sa.nk = stage;
    for (int j = 0; j < stage; ++j) {
      sa.k[j] = kk[j];
      sa.coef[j] = I.coef[stage][j];
    }
    sa.normalize = stage == 6;
    sa.stage = I.ybuf[p ^ 1];
  }
  fa.stage = sa.stage;
  fa.kout = kk[stage];
  fa.terms = I.terms;
  fa.relax = I.relax;
  if (stage == 6) {
    fa.err = I.red;
    fa.torque_max = I.red + 1;
    for (int j = 0; j < 7; ++j) fa.ecoef[j] = I.ecoef[j];
    for (int j = 0; j < 6; ++j) fa.ek[j] = kk[j];
  }
}

// This block's item and a shared-memory copy of its member descriptor.
// Ends with a barrier.
__device__ __forceinline__ BatchItem batch_item(const BatchInst* insts, const BatchItem* items, BatchInst& si) {
  const BatchItem w = items[blockIdx.x];
  const int* src = reinterpret_cast<const int*>(insts + w.inst);
  int* dst = reinterpret_cast<int*>(&si);
  for (int i = threadIdx.x; i < (int)(sizeof(BatchInst) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  return w;
}

}  // namespace mmp

// tcdft.cuh -- a length-32 DFT stage as a dense split-TF32 GEMM on the
// tensor cores (tcgen05.mma kind::tf32), for the warp y transforms of pass B.
//
// The final stage of a warp transform (wfft.cuh) is a DFT32 across each
// lane's 32 registers: with X[l][m] the m-th value of lane l, Y[l][k] =
// sum_m X[l][m] F[m][k], F[m][k] = w32^(m k).  A warpgroup (four warps, one
// column group each) stacks its four 32 x 32 X into a 128 x 32 complex A
// operand in tensor memory (thread = row = TMEM lane), F sits in shared
// memory as the B operand, and the real and imaginary parts of Y accumulate
// in tensor memory:
//   Yr = Xr Fr + Xi (-Fi),   Yi = Xr Fi + Xi Fr,
// each real product as three TF32 products (hi hi + hi lo + lo hi; x = hi +
// lo with hi the TF32 rounding of x), FP32 accumulation.  F is symmetric,
// so the K-major and N-major readings of its layout are the same matrix.
//
// Shared-memory layout of a 32 x 32 fp32 B matrix (no swizzle): core matrix
// (i, j) = rows (N) 8 i .. 8 i + 7, K elements 4 j .. 4 j + 3, at byte
// (8 i + j) * 128, row r of it at 16 r.  A K-step of 8 covers core matrices
// j = 2 kk, 2 kk + 1: leading-dimension offset 128 B (along K), stride
// offset 1024 B (along N).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "tmem.cuh"

namespace mmp {

constexpr int kTcB = 32 * 32;   // floats of one B matrix (4 KB)
// Order of the four B matrices in shared memory / in the host table.
enum { kTcFrH = 0, kTcFrL = 1, kTcFiH = 2, kTcFiL = 3 };
// Tensor-memory columns of one warpgroup: A = Xr_hi, Xi_hi, Xr_lo, Xi_lo
// (32 each), then D (32): Yr and Yi are formed one after the other.
constexpr int kTcCols = 160;

// TF32 rounding (round to nearest, ties away) of an FP32 value, in a 32-bit container.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading- and
// stride-dimension byte offsets (>> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_smem_desc(const void* smem, uint32_t lbo, uint32_t sbo) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  uint64_t d = 0;
  d |= (uint64_t)((a >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // version
  return d;                 // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::tf32: D f32, A and B tf32, both K-major,
// N = 32, M = 128; negB negates B.
__host__ __device__ constexpr uint32_t tc_idesc(bool negB) {
  return (1u << 4)             // D format: f32
       | (2u << 7)             // A format: tf32
       | (2u << 10)            // B format: tf32
       | ((negB ? 1u : 0u) << 14)
       | ((32u >> 3) << 17)    // N >> 3
       | ((128u >> 4) << 24);  // M >> 4
}

// D (+)= A[tmem] x B[smem desc], issued by one thread.
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc, bool acc) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(acc ? 1u : 0u)
      : "memory");
}

// Arrive on the mbarrier once every MMA issued so far by this thread completes.
__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(mbar));
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(a) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(mbar));
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}

// Wait for the completion of phase `parity` of the mbarrier, giving up after
// `limit` polls (each poll may suspend the thread for a short time).
// Returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t limit) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(mbar));
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Named barrier of the four warps of warpgroup g (ids 1..4; 0 is __syncthreads).
__device__ __forceinline__ void wg_sync(int g) {
  asm volatile("bar.sync %0, 128;\n" ::"r"(g + 1) : "memory");
}

// 32 consecutive columns of the thread's lane from / into v (32x32b.x32).
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]),
      "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]),
      "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]),
        "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15]), "=f"(v[16]),
        "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]), "=f"(v[22]), "=f"(v[23]), "=f"(v[24]),
        "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31])
      : "r"(taddr)
      : "memory");
}

// A DFT32 across each lane's registers on the tensor cores, for the four
// warps of warpgroup g (lane l holds the 32 inputs v[m] of its row).  On
// return lane l holds v[k] = sum_m v[m] w32^(m k).
//   tbase: the CTA's tensor memory; cols: this warpgroup's first column
//   Bs: the four B matrices in shared memory; mbar: this warpgroup's
//   mbarrier, phase: its next phase parity (flipped twice here)
//   err: set to 1 if a wait runs past its limit (the values are then not valid)
__device__ __forceinline__ void tc_stage32(float2 (&v)[32], uint32_t tbase, int cols, const float* Bs, uint64_t* mbar,
                                           uint32_t& phase, unsigned* err) {
  const int warp = threadIdx.x >> 5, g = warp >> 2;
  const bool leader = (warp & 3) == 0 && (threadIdx.x & 31) == 0;
  const uint32_t tA = tmem_addr(tbase, cols), tD = tmem_addr(tbase, cols + 128);
  const uint32_t a0 = tbase + (uint32_t)cols;   // lane 0 of the warpgroup's columns (MMA operands)
  // A: this thread's row, split into TF32 hi and lo parts
  {
    float xr[32], xi[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) {
      xr[m] = tf32_rna(v[m].x);
      xi[m] = tf32_rna(v[m].y);
    }
    tmem_st32(tA, xr);
    tmem_st32(tA + 32, xi);
#pragma unroll
    for (int m = 0; m < 32; ++m) {
      xr[m] = v[m].x - xr[m];
      xi[m] = v[m].y - xi[m];
    }
    tmem_st32(tA + 64, xr);
    tmem_st32(tA + 96, xi);
  }
  tmem_wait_st();
  tmem_fence_before_sync();
  wg_sync(g);
  tmem_fence_after_sync();
  const uint32_t XrH = a0, XiH = a0 + 32, XrL = a0 + 64, XiL = a0 + 96, D = a0 + 128;
  float out[2][32];
#pragma unroll
  for (int part = 0; part < 2; ++part) {   // 0: Yr, 1: Yi
    if (leader) {
      // (A, B, negate B) triples: Yr = Xr Fr + Xi (-Fi), Yi = Xr Fi + Xi Fr
      const uint32_t Aop[6] = {XrH, XrH, XrL, XiH, XiH, XiL};
      const int Bre[6] = {kTcFrH, kTcFrL, kTcFrH, kTcFiH, kTcFiL, kTcFiH};
      const int Bim[6] = {kTcFiH, kTcFiL, kTcFiH, kTcFrH, kTcFrL, kTcFrH};
#pragma unroll
      for (int t = 0; t < 6; ++t) {
        const int bsel = part == 0 ? Bre[t] : Bim[t];
        const bool neg = part == 0 && t >= 3;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t bd = tc_smem_desc(Bs + bsel * kTcB + kk * 64, 128, 1024);
          tc_mma(D, Aop[t] + 8 * kk, bd, tc_idesc(neg), t > 0 || kk > 0);
        }
      }
      tc_commit(mbar);
    }
    const bool ok = mbar_wait(mbar, phase, 1u << 20);
    phase ^= 1u;
    if (!ok && err) atomicExch(err, 1u);
    tmem_fence_after_sync();
    tmem_ld32(tD, out[part]);
    // every warp has read D before the next products overwrite it
    tmem_fence_before_sync();
    wg_sync(g);
    tmem_fence_after_sync();
  }
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = make_float2(out[0][k], out[1][k]);
}

}  // namespace mmp

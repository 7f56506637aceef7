// tmem.cuh -- tensor memory (TMEM): allocation, fences and addressing.
//
// sm_103a has 256 KB of tensor memory per SM (128 lanes x 512 columns of
// 32 bits) next to the tensor cores.  A warp accesses the lane quarter
// 32 (w mod 4) .. 32 (w mod 4) + 31 of its warp index w; data moves between
// a thread's registers and its own lane (tcgen05.st / tcgen05.ld, 32x32b
// shape), and the MMAs read and write it directly (tcdft.cuh).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mmp {

// Allocate `ncols` columns (a power of two, 32..512) for the CTA; executed
// by every thread of one warp.  The base address is written to *slot
// (shared memory).  Blocks while another CTA on the SM holds the columns
// (it frees them when it finishes).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(slot));
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(s), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
// Free them again (the allocating warp, after every access has completed).
__device__ __forceinline__ void tmem_free(uint32_t base, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(base), "r"(ncols) : "memory");
}
// Ordering of tensor-memory accesses around thread barriers.
__device__ __forceinline__ void tmem_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// Address of column `col` of this warp's lane quarter.
__device__ __forceinline__ uint32_t tmem_addr(uint32_t base, int col) {
  const uint32_t lane0 = 32u * ((threadIdx.x >> 5) & 3u);
  return base + (lane0 << 16) + (uint32_t)col;
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

}  // namespace mmp

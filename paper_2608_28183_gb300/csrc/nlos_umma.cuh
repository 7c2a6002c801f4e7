// 5th-generation tensor-core (tcgen05) building blocks for sm_103a, written
// as inline PTX: tensor-memory allocation, shared-memory matrix descriptors,
// the instruction descriptor of kind::f16 MMAs, MMA issue/commit and
// accumulator reads.
//
// Operand layout used throughout: K-major, no swizzle. A matrix of R rows and
// K columns (16-bit elements) is stored as 8 x 8 "core matrices" (8 rows of
// 16 bytes, 128 contiguous bytes each); core matrix (row group g, column
// group k) sits at byte offset g * SBO + k * LBO from the operand's start.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nlos_tma.cuh"

namespace nlos {

// ---- tensor memory ----------------------------------------------------------
// One warp allocates ncols columns (a power of two >= 32) of the CTA's TMEM and
// writes the base address to shared memory; the same warp frees them.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ordering of tcgen05 operations around thread synchronisation
__device__ __forceinline__ void tc_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---- descriptors --------------------------------------------------------------
// Shared-memory matrix descriptor: start address, leading-dimension (K
// direction) byte offset and stride-dimension (row-group) byte offset, all in
// 16-byte units; descriptor version 1; base offset 0; no swizzle.
__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of a kind::f16 MMA: fp32 accumulator, f16 A and B
// (bf16 when kBf16), both K-major, no negation, shape M x N (x 16).
template <bool kBf16>
__host__ __device__ constexpr uint32_t umma_idesc_f16(int M, int N) {
  return (1u << 4)                                   // D: f32
         | ((kBf16 ? 1u : 0u) << 7)                  // A format
         | ((kBf16 ? 1u : 0u) << 10)                 // B format
         | ((uint32_t)(N >> 3) << 17)                // N / 8
         | ((uint32_t)(M >> 4) << 24);               // M / 16
}

// ---- MMA ------------------------------------------------------------------------
// D[tmem] (+)= A[smem] * B[smem]^T for one K = 16 slab; issued by one thread.
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// arrive on an mbarrier once every MMA this thread issued before has completed
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// ---- accumulator reads ----------------------------------------------------------
// Warp w of the CTA reads TMEM lanes 32 (w % 4) .. + 31 (thread t: lane
// 32 (w % 4) + t), 16 consecutive 32-bit columns starting at taddr's column.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 1D bulk copy global -> shared completing `bytes` of transaction count on
// bar (addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// asynchronous copy of `bytes` (4, 8 or 16) global -> shared by this thread;
// src_bytes = 0 writes zeros instead of reading src (src must still be a
// valid address). Completion: cp_async_commit / cp_async_wait<n>.
__device__ __forceinline__ void cp_async(void* dst, const void* src, uint32_t src_bytes, int bytes) {
  if (bytes == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most n of this thread's committed groups are still pending
template <int n>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(n) : "memory");
}

// hint: bring `bytes` of global memory at src into L2 (src 16-byte aligned,
// bytes a multiple of 16)
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<uint64_t>(src)), "r"(bytes)
               : "memory");
}

// byte offset of element (r, k) of a K-major no-swizzle operand whose rows
// hold kcols elements (16-bit): core matrix (r / 8, k / 8), LBO = 128 bytes,
// SBO = kcols / 8 * 128 bytes
__host__ __device__ constexpr uint32_t umma_kmajor_offset(int r, int k, int kcols) {
  return (uint32_t)(((r >> 3) * (kcols >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

}  // namespace nlos

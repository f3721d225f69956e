// tc.cuh -- 5th-generation tensor-core (tcgen05) building blocks for the
// split-precision DFT: tensor-memory allocation, shared-memory matrix and
// instruction descriptors, the MMA issue, its completion on an mbarrier, and
// the read-back of the accumulator.
//
// Conventions (one CTA, cta_group::1):
//   * D[M x N] (FP32, tensor memory) = sum over K of A[M x K] B[N x K]^T:
//     A and B are both stored K-major in shared memory -- row m of A holds
//     its K values contiguously -- in the 128-byte swizzled layout: rows of
//     128 bytes (32 TF32 values), groups of 8 rows (1024 bytes, 1024-byte
//     aligned) in which 16-byte chunk c of row r sits at chunk c ^ (r mod 8).
//   * M = 128: accumulator row m is tensor-memory lane m, column n is
//     tensor-memory column base + n; warp w of the warpgroup reads lanes
//     32 (w mod 4) .. + 31.
//   * K advances 8 TF32 values (32 bytes) per MMA by moving the descriptor's
//     start address inside the swizzle atom.
#pragma once

#include <cstdint>

#include "fft_tile.cuh"

namespace tfft {
namespace tc {

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);          // start address
  d |= (uint64_t)(16u >> 4) << 16;                  // leading byte offset (unused for this layout)
  d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;    // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                           // version
  d |= (uint64_t)2 << 61;                           // layout: 128-byte swizzle
  return d;
}

// The same for a 64-byte swizzle (rows of 64 bytes, 8-row groups 512 bytes
// apart, layout code 4): 16-byte chunk c of row r at chunk c ^ ((r / 2) mod 4).
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);          // start address
  d |= (uint64_t)(16u >> 4) << 16;                  // leading byte offset (unused for this layout)
  d |= (uint64_t)((512u >> 4) & 0x3FFFu) << 32;     // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                           // version
  d |= (uint64_t)4 << 61;                           // layout: 64-byte swizzle
  return d;
}

// Instruction descriptor: FP32 accumulator, A and B of format `fmt`
// (TF32 = 2 for kind::tf32, BF16 = 1 for kind::f16), both K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D (+)= A B^T, kind::tf32.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// D (+)= A B^T, kind::f16 (BF16 operands here).
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
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

// The mbarrier completes once every MMA issued before by this thread has.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// Round to TF32 (nearest, ties away from zero): the high part of a split.
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// BF16 split: the high part rounded to nearest, and the rounded remainder;
// packed two values (x0 low half, x1 high half) per 32-bit word.
__device__ __forceinline__ void split_bf16x2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x1), "f"(x0));
  const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xFFFF0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(x1 - h1), "f"(x0 - h0));
}

// Byte offset of 16-byte chunk c (0..7) of row m in a 128-byte-swizzled,
// K-major operand.
__device__ __forceinline__ uint32_t sw128_off(int m, int c) {
  return (uint32_t)((m >> 3) * 1024 + (m & 7) * 128 + ((c ^ (m & 7)) << 4));
}
// ... and of chunk c (0..3) of row m in a 64-byte-swizzled one.
__device__ __forceinline__ uint32_t sw64_off(int m, int c) {
  return (uint32_t)(m * 64 + ((c ^ ((m >> 1) & 3)) << 4));
}

}  // namespace tc
}  // namespace tfft

// Fifth-generation tensor-core (tcgen05) helpers: shared-memory matrix
// descriptors in the 128-byte swizzled layout, the BF16 instruction
// descriptor, MMA issue and completion, TMEM loads, and exact splitting of
// floating-point values into BF16 digits for error-free products.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hs_common.cuh"

namespace hs {
namespace tc {

// Shared-memory descriptor: start address >> 4 in bits 0-13, leading byte
// offset >> 4 in 16-29, stride byte offset >> 4 in 32-45, version 1 in 46-47,
// layout in 61-63 (2 = 128-byte swizzle).  MN-major operand: 64-element atoms
// (128-byte rows) LBO apart along M/N, 8-row K groups SBO apart.  K-major
// operand: 8-row groups of 128-byte rows SBO apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46) | (2ull << 61);
}
// Instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A and B bf16
// (bits 7-9, 10-12 = 1), A/B major (bits 15, 16; 1 = MN-major), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// D (TMEM) = A B^T (+ D when accumulate != 0), one CTA.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on an mbarrier once every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Generic-proxy shared-memory writes become visible to the tensor cores.
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// TMEM allocation by one whole warp (columns: a power of two >= 32).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)), "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols));
}
// 32 lanes x 16 consecutive columns of TMEM into 16 registers per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// 32 lanes x 8 consecutive columns of TMEM into 8 registers per thread.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Byte offset of element (K row r, M/N index k < 64) in a 128-byte-swizzled
// MN-major atom (or of element (row r, column k) of a K-major block) whose
// 8-row groups are 1024 bytes apart.  Offsets of 8 consecutive k starting at
// a multiple of 8 are one contiguous, 16-byte-aligned run.
__host__ __device__ __forceinline__ uint32_t sw128_off(int r, int k) {
  const uint32_t byte = (uint32_t)k * 2;
  return (uint32_t)(r >> 3) * 1024u + (uint32_t)(r & 7) * 128u + ((((byte >> 4) ^ (uint32_t)(r & 7)) & 7u) << 4) +
         (byte & 15u);
}

// ---- exact BF16 digits ------------------------------------------------------
// A value v with |v| < 1 is written as v = sum_{t=1..S} d_t 2^{-8t} + rest,
// d_t = rint(256 r_{t-1}), r_t = 256 r_{t-1} - d_t (r_0 = v), so |d_1| <= 256
// and |d_t| <= 128 for t >= 2, |rest| <= 2^{-8S-1}.  Every digit is an integer
// with at most 8 significant bits, exact in BF16, and every step is exact in
// binary floating point (scaling by 256, rounding to an integer, and the
// difference of two numbers within 1/2 of each other).  The product of two
// digits is exact in FP32 and a sum of products of digits of equal weight is
// exact in an FP32 accumulator while it stays below 2^24.
__host__ __device__ __forceinline__ float digit_step(float& r) {
  const float s = r * 256.0f;
  const float d = rintf(s);
  r = s - d;
  return d;
}
__host__ __device__ __forceinline__ double digit_step(double& r) {
  const double s = r * 256.0;
  const double d = rint(s);
  r = s - d;
  return d;
}
// Eight digits (one per value, the same digit position) packed as BF16 into 16 bytes.
__device__ __forceinline__ uint4 pack8_bf16(const float (&d)[8]) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(d[2 * i], d[2 * i + 1]);
    w[i] = *reinterpret_cast<const uint32_t*>(&h);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

}  // namespace tc
}  // namespace hs

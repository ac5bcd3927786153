// Device helpers shared by the kernels of the Horseshoe-probit sweep:
// Philox4x32-10, the exact uniform map, the truncated-normal inverse CDF,
// mbarrier / bulk-copy wrappers and the device error word.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hs_internal.h"

namespace hs {

// Counter purposes (Philox counter word 2, low byte).
enum : uint32_t { kPurZ = 1, kPurLambda = 2, kPurTau = 3, kPurBeta = 4, kPurNu = 5, kPurXi = 6 };

__device__ __forceinline__ void set_error(int* err, int bits) {
  if (err) atomicOr(err, bits);
}
// a bounded wait at `site` ran out
__device__ __forceinline__ void set_timeout(int* err, int site) {
  set_error(err, kErrTimeout | (1 << (kErrSiteShift + site)));
}

// ---- Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) --------------------
// Ten rounds of (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1,
// lo(M0 c0)) with the key bumped by the Weyl constants after each round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

struct Rng {
  uint32_t k0, k1;       // key = seed
  uint32_t chain, problem;
  __device__ __forceinline__ uint4 words(uint32_t index, uint32_t sweep, uint32_t purpose) const {
    return philox4x32_10(make_uint4(index, sweep, purpose | (chain << 8), problem), k0, k1);
  }
};

// u = (2m + 1) 2^-53 with m = (hi << 20) | (lo >> 12); uc = 1 - u, both exact.
__device__ __forceinline__ void unit_pair(uint32_t hi, uint32_t lo, double& u, double& uc) {
  const uint64_t m = ((uint64_t)hi << 20) | (uint64_t)(lo >> 12);
  const uint64_t mc = ((1ull << 52) - 1ull) - m;
  u = (double)(2ull * m + 1ull) * 0x1p-53;
  uc = (double)(2ull * mc + 1ull) * 0x1p-53;
}

// Standard normal quantile of u on the accurate side: Phi^{-1}(u) for u <= 1/2,
// -Phi^{-1}(1-u) otherwise.
__device__ __forceinline__ double std_normal_from_unit(double u, double uc) {
  return (u <= uc) ? normcdfinv(u) : -normcdfinv(uc);
}

// ---- truncated normal by inverse CDF (Eq. 12, first line) -----------------
// z+ ~ N(ms, 1) truncated to (0, inf) is the solution of
//   Phi(ms - z+) = u Phi(ms),  i.e.  z+ = ms - Phi^{-1}(u Phi(ms)).
// Phi^{-1} is applied to the smaller of q = u Phi(ms) and
// 1 - q = (1 - u) + u Phi(-ms).  For ms below a threshold the same equation is
// solved for z directly: with a = -ms and the Mills ratio R(x) = Phi(-x)/phi(x)
// = sqrt(pi/2) erfcx(x / sqrt 2),
//   h(z) = a z + z^2/2 - ln(R(a+z)/R(a)) + ln u = 0,   h'(z) = 1 / R(a+z),
// h is increasing and convex and h(-ln(u)/a) >= 0, so Newton from z0 = -ln(u)/a
// decreases monotonically to the root without cancellation.
template <typename T> struct TnMath;
template <> struct TnMath<double> {
  static constexpr double kTail = -30.0;
  static constexpr int kNewton = 7;
  static __device__ __forceinline__ double ncdf(double x) { return normcdf(x); }
  static __device__ __forceinline__ double ncdfinv(double x) { return normcdfinv(x); }
  static __device__ __forceinline__ double erfcx_(double x) { return erfcx(x); }
  static __device__ __forceinline__ double log_(double x) { return log(x); }
  static __device__ __forceinline__ double log1p_(double x) { return log1p(x); }
  static __device__ __forceinline__ double tiny() { return 2.2250738585072014e-308; }
};
template <> struct TnMath<float> {
  static constexpr float kTail = -9.0f;
  static constexpr int kNewton = 5;
  static __device__ __forceinline__ float ncdf(float x) { return normcdff(x); }
  static __device__ __forceinline__ float ncdfinv(float x) { return normcdfinvf(x); }
  static __device__ __forceinline__ float erfcx_(float x) { return erfcxf(x); }
  static __device__ __forceinline__ float log_(float x) { return logf(x); }
  static __device__ __forceinline__ float log1p_(float x) { return log1pf(x); }
  static __device__ __forceinline__ float tiny() { return 1.17549435e-38f; }
};

// Main arm (valid for ms >= kTail).
template <typename T>
__device__ __forceinline__ T tn_main(T ms, T u, T uc) {
  using M = TnMath<T>;
  const T pm = M::ncdf(ms);
  const T pc = M::ncdf(-ms);
  const T q = u * pm;
  const T qc = fma(u, pc, uc);
  const bool lower = q <= qc;
  const T w0 = M::ncdfinv(lower ? q : qc);
  return ms - (lower ? w0 : -w0);
}

// Tail arm (intended for ms < kTail; any a > 0 works).
template <typename T>
__device__ __forceinline__ T tn_tail(T ms, T u, T uc) {
  using M = TnMath<T>;
  const T kInvSqrt2 = (T)0.70710678118654752440;
  const T kSqrtHalfPi = (T)1.25331413731550025121;
  const T a = -ms;
  const T lnu = (u > (T)0.5) ? M::log1p_(-uc) : M::log_(u);
  const T ra = M::erfcx_(a * kInvSqrt2);
  T z = -lnu / a;
#pragma unroll
  for (int it = 0; it < M::kNewton; ++it) {
    const T rz = M::erfcx_((a + z) * kInvSqrt2);
    const T h = fma(a, z, (T)0.5 * z * z) - M::log_(rz / ra) + lnu;
    z = fma(-h, kSqrtHalfPi * rz, z);
  }
  return z;
}

// ---- shared-memory barriers and bulk copies (sm_90+ PTX) -------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase with the given parity; false once limit_ns nanoseconds
// have passed without it (the caller records kErrTimeout and winds down).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          uint64_t limit_ns = 2000000000ull) {
  if (mbar_test(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_test(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
// One contiguous global -> shared copy completing on an mbarrier
// (addresses and size multiples of 16 bytes).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// The same with an L2 eviction-priority policy (createpolicy).
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
// Data read once: evicted from L2 first, so it does not push out the working
// sets of kernels running beside it.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ---- warp reductions --------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

}  // namespace hs

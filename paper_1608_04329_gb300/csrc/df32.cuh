// FP32-pair ("double-float") arithmetic for the p x p factorization.
//
// GB300 runs FP64 at about 1/64 of the FP32 rate, and FP64 latency-bound code
// (a 32 x 32 Cholesky, divisions, square roots) is slower still, so the
// Cholesky factor and the inverse factor of the precision matrix are held and
// computed as unevaluated sums x = hi + lo of two FP32 numbers (about 48
// significant bits).  The building blocks are the published error-free
// transformations: Knuth's TwoSum, Dekker's Fast2Sum (here after a sum whose
// larger term is known) and the FMA-based TwoProduct (Ogita, Rump & Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005); division
// and square root take one Newton correction of the FP32 quotient or root.
// Relative error of each operation is a small multiple of 2^-48.  The exact
// operations are host-callable too, so the CPU tests check these bounds.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace hs {

struct __align__(8) df2 {
  float hi, lo;
};

__host__ __device__ __forceinline__ df2 df_split(double x) {
  const float hi = (float)x;
  const float lo = (float)(x - (double)hi);
  return {hi, lo};
}
__host__ __device__ __forceinline__ double df_value(df2 a) { return (double)a.hi + (double)a.lo; }
__host__ __device__ __forceinline__ double df_value(float hi, float lo) { return (double)hi + (double)lo; }

// Fast2Sum: |a| >= |b| or a == 0.
__host__ __device__ __forceinline__ df2 df_renorm(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__host__ __device__ __forceinline__ df2 df_add(df2 a, df2 b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  return df_renorm(s, e);
}
__host__ __device__ __forceinline__ df2 df_neg(df2 a) { return {-a.hi, -a.lo}; }
__host__ __device__ __forceinline__ df2 df_sub(df2 a, df2 b) { return df_add(a, df_neg(b)); }
__host__ __device__ __forceinline__ df2 df_mul(df2 a, df2 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_renorm(p, e);
}
// 1 / b: FP32 reciprocal q, residual 1 - b q in pair arithmetic, one correction.
__host__ __device__ __forceinline__ df2 df_recip(df2 b) {
  const float q = 1.0f / b.hi;
  const df2 r = df_sub(df2{1.0f, 0.0f}, df_mul(b, df2{q, 0.0f}));
  return df_renorm(q, r.hi * q);
}
// sqrt(a), a > 0: FP32 root s, exact s^2 = p + e, one correction.
__host__ __device__ __forceinline__ df2 df_sqrt(df2 a) {
  const float s = sqrtf(a.hi);
  const float p = s * s;
  const float e = fmaf(s, s, -p);
  const float r = ((a.hi - p) - e) + a.lo;
  return df_renorm(s, r / (2.0f * s));
}

// Same from a hardware-approximate seed q (about 2^-22): the residual
// 1 - b q is formed by FMAs and applied once, about 2^-44 relative, without
// the slow path of a correctly rounded FP32 division.  Used on the pivots.
__device__ __forceinline__ df2 df_recip_fast(df2 b) {
  const float q = __fdividef(1.0f, b.hi);
  float e = fmaf(-b.hi, q, 1.0f);
  e = fmaf(-b.lo, q, e);
  return df_renorm(q, q * e);
}
// sqrt(a) and 1/sqrt(a), a > 0, from the approximate reciprocal square root.
__device__ __forceinline__ void df_sqrt_rsqrt_fast(df2 a, df2& sq, df2& rs) {
  const float y = rsqrtf(a.hi);
  const float s = a.hi * y;
  const float p = s * s;
  const float e = fmaf(s, s, -p);
  const float r = ((a.hi - p) - e) + a.lo;
  sq = df_renorm(s, 0.5f * r * y);
  rs = df_recip_fast(sq);
}

// (sh, sl) += a * b with a lazily accumulated low word; df_renorm(sh, sl)
// gives the pair at the end.
__host__ __device__ __forceinline__ void df_fma(float& sh, float& sl, df2 a, df2 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s = sh + p;
  const float bb = s - sh;
  const float t = (sh - (s - bb)) + (p - bb);
  sh = s;
  sl += t + e;
}

// The six BF16 digits of a pair x with |x| <= 1 on the fixed grid 2^0:
// x = sum_{t=1..6} d_t 2^{-8t} + rest, |rest| <= 2^{-49}, d_t = rint(256 r_{t-1})
// with the remainder r kept as an exact pair (TwoSum after each step), so
// |d_1| <= 256 and |d_t| <= 128 for t >= 2; each digit is an integer of at
// most 8 significant bits, returned as its BF16 bit pattern (the low half of
// its FP32 bits is zero).
__host__ __device__ __forceinline__ void df_digits6(df2 x, uint16_t (&d)[6]) {
  float rh = x.hi, rl = x.lo;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const float sh = rh * 256.0f, sl = rl * 256.0f;
    const float dd = rintf(sh);
    const float a = sh - dd;
    const float s = a + sl, bb = s - a;
    rl = (a - (s - bb)) + (sl - bb);
    rh = s;
    uint32_t bits;
    memcpy(&bits, &dd, 4);
    d[t] = (uint16_t)(bits >> 16);
  }
}

__device__ __forceinline__ df2 df_shfl_xor(df2 v, int mask) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, mask), __shfl_xor_sync(0xffffffffu, v.lo, mask)};
}

}  // namespace hs

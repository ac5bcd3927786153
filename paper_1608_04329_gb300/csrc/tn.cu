// Truncated-normal samplers of the latent draw, standalone (Eq. 12, first
// line: z+ ~ N(mu*, 1) restricted to (0, inf)), for comparing the two ways of
// drawing it on the GPU:
//
//  inverse CDF   z+ = mu* - Phi^{-1}(u Phi(mu*)) with Phi^{-1} on the accurate
//                side and the log-space Newton tail arm for mu* < -9; one
//                uniform pair per draw, no data-dependent loop.  The same
//                arithmetic (tn_main / tn_tail, FP32) as the X-stream's
//                sampler, on the same counters (index i, sweep, purpose z).
//  rejection     the paper's two-arm sampler (Sect. 5, z steps b and c): for
//                mu* > 0.47 propose N(mu*, 1) until positive; otherwise
//                Robert's (1995) exponential proposal z ~ Exp(theta),
//                theta = (-mu* + sqrt(mu*^2 + 4)) / 2, accepted with
//                probability exp(-(z - mu* - theta)^2 / 2).  Attempt t of
//                draw i uses the counter (i, sweep, 8 + t): words (0, 1) give
//                the proposal's uniform, words (2, 3) the acceptance uniform.
//                A warp runs until its last lane accepts, which is the
//                divergence the inverse CDF avoids.  After 64 rejections
//                (probability below 1e-30 for either arm) the draw falls back
//                to the inverse CDF and reports 65 attempts.
//
// One thread per draw; FP32 arithmetic as in the X-stream's FP32 path.
#include <cuda_runtime.h>

#include <cstdint>

#include "hs_common.cuh"
#include "hs_internal.h"
#include "hs_probit.h"
#include "hs_tn.h"

namespace hs {
namespace {

constexpr uint32_t kPurZRej = 8;  // attempts use purposes 8 .. 8 + kMaxTries - 1
constexpr int kMaxTries = 64;

__device__ __forceinline__ float invcdf_draw(float ms, const Rng& rng, uint32_t i, uint32_t sweep) {
  const uint4 w = rng.words(i, sweep, kPurZ);
  double u, uc;
  unit_pair(w.x, w.y, u, uc);
  float zp = tn_main<float>(ms, (float)u, (float)uc);
  if (ms < TnMath<float>::kTail) zp = tn_tail<float>(ms, (float)u, (float)uc);
  return zp > TnMath<float>::tiny() ? zp : TnMath<float>::tiny();
}

__global__ void __launch_bounds__(256) tn_invcdf_kernel(const float* __restrict__ mu, int64_t n, Rng rng,
                                                        uint32_t sweep, float* __restrict__ z,
                                                        int32_t* __restrict__ tries) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  z[i] = invcdf_draw(mu[i], rng, (uint32_t)i, sweep);
  if (tries) tries[i] = 1;
}

__global__ void __launch_bounds__(256) tn_rejection_kernel(const float* __restrict__ mu, int64_t n, Rng rng,
                                                           uint32_t sweep, float* __restrict__ z,
                                                           int32_t* __restrict__ tries) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float m = mu[i];
  float x = 0.0f;
  int t = 0;
  bool done = false;
  if (m > 0.47f) {
    // Gaussian arm: mu* + N(0, 1) until positive
    while (!done && t < kMaxTries) {
      const uint4 w = rng.words((uint32_t)i, sweep, kPurZRej + (uint32_t)t);
      ++t;
      double u, uc;
      unit_pair(w.x, w.y, u, uc);
      const float g = u <= uc ? normcdfinvf((float)u) : -normcdfinvf((float)uc);
      x = m + g;
      done = x > 0.0f;
    }
  } else {
    // Robert's arm: exponential proposal on (0, inf) with rate theta
    const float theta = 0.5f * (-m + sqrtf(fmaf(m, m, 4.0f)));
    while (!done && t < kMaxTries) {
      const uint4 w = rng.words((uint32_t)i, sweep, kPurZRej + (uint32_t)t);
      ++t;
      double u1, uc1, u2, uc2;
      unit_pair(w.x, w.y, u1, uc1);
      unit_pair(w.z, w.w, u2, uc2);
      x = -logf((float)u1) / theta;
      const float d = x - m - theta;
      done = (float)u2 < expf(-0.5f * d * d);
    }
  }
  if (!done) {
    x = invcdf_draw(m, rng, (uint32_t)i, sweep);
    t = kMaxTries + 1;
  }
  z[i] = x;
  if (tries) tries[i] = t;
}

}  // namespace
}  // namespace hs

extern "C" int hs_tn_sample(const float* mu, int64_t n, uint64_t seed, uint32_t chain, uint32_t sweep, int32_t method,
                            float* z, int32_t* tries, void* stream) {
  if (n < 0 || (n > 0 && (!mu || !z)) || n > (int64_t)0xFFFFFFFF || chain >= (1u << 24) ||
      (method != HS_TN_INVCDF && method != HS_TN_REJECTION))
    return HS_EINVAL;
  if (n == 0) return HS_OK;
  const hs::Rng rng{(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32), chain, 0u};
  const unsigned blocks = (unsigned)((n + 255) / 256);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (method == HS_TN_INVCDF)
    hs::tn_invcdf_kernel<<<blocks, 256, 0, s>>>(mu, n, rng, sweep, z, tries);
  else
    hs::tn_rejection_kernel<<<blocks, 256, 0, s>>>(mu, n, rng, sweep, z, tries);
  return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ECUDA;
}

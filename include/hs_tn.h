/* Truncated-normal samplers of the latent draw, standalone.
 *
 * The latent step of the sweep (Eq. 12, first line; Sect. 5, z steps) draws
 * z+ ~ N(mu*, 1) restricted to (0, inf), mu* = y*_i x_i beta.  The library's
 * sweep uses the branch-free inverse CDF; the paper draws it with a two-arm
 * rejection sampler (a Gaussian proposal for mu* > 0.47, Robert's 1995
 * exponential proposal otherwise; Sect. 5, z steps b and c).  This entry point
 * runs either one over an array of mu* so the two can be compared on the GPU
 * (time, attempts per draw, and how long a warp waits for its slowest lane).
 */
#ifndef HS_TN_H
#define HS_TN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HS_TN_INVCDF     0 /* z+ = mu* - Phi^{-1}(u Phi(mu*)), the sweep's FP32 arithmetic and counters */
#define HS_TN_REJECTION  1 /* the paper's two-arm rejection sampler, FP32 */

/* Draw z[i] ~ N(mu[i], 1) restricted to (0, inf) for i < n, FP32, one thread
 * per draw, enqueued on `stream` (a cudaStream_t; NULL: the legacy default
 * stream); returns without synchronizing.
 *   mu, z    device arrays of n floats (caller-owned; z is written)
 *   tries    device array of n int32 receiving the proposals each draw used
 *            (1 for HS_TN_INVCDF; 65 marks a rejection draw that gave up
 *            after 64 proposals and used the inverse CDF), or NULL
 *   seed, chain, sweep   Philox key and counter fields: draw i of the inverse
 *            CDF uses the counter (i, sweep, 1 | chain << 8, 0), exactly the
 *            latent draw of that sweep and chain; attempt t of the rejection
 *            sampler uses (i, sweep, (8 + t) | chain << 8, 0)
 * Returns HS_OK, HS_EINVAL (n < 0 or n >= 2^32, a NULL mu or z with n > 0,
 * chain >= 2^24, an unknown method; nothing is launched) or HS_ECUDA (the
 * launch failed). */
int hs_tn_sample(const float* mu, int64_t n, uint64_t seed, uint32_t chain, uint32_t sweep, int32_t method,
                 float* z, int32_t* tries, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HS_TN_H */

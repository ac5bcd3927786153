/*
 * hs_probit.h -- C ABI of the GB300 (sm_103a) Gibbs sweep for Horseshoe
 * probit regression.
 *
 * Model and sampler: Terenin, Dong & Draper, "GPU-accelerated Gibbs sampling:
 * a case study of the Horseshoe Probit model", Sect. 5.
 *   likelihood  y_i = round[Phi(z_i)], z_i | x_i, beta ~ N(x_i beta, 1)   (Eq. 9)
 *   prior       beta_j ~ N(0, lambda_j^2 tau^2), lambda_j, tau ~ C+(0, 1)  (Eq. 10)
 *   conditionals of z, lambda^{-2}, nu^{-1}, beta, tau^{-2}, xi^{-1}       (Eq. 12)
 *   schedule    (i) z and lambda^{-2} in parallel, then tau^{-2};
 *               (ii) beta, nu^{-1} and xi^{-1} in parallel.
 * One call of hs_probit_sweep(h, n) runs n such sweeps on the GPU.
 *
 * Conventions for every entry point:
 *   - Pointers marked "host" are ordinary host memory owned by the caller;
 *     pointers marked "device" are CUDA device memory on the handle's device,
 *     also owned by the caller.  The library never frees caller memory.
 *   - The handle owns all device memory it allocates; hs_probit_free
 *     releases it.
 *   - Matrices are row-major.  X is N x p with rows contiguous (row stride p).
 *   - Status codes are the HS_* values below: 0 on success, < 0 on error.
 *   - A handle may be used from one host thread at a time.
 *
 * Random numbers: every uniform is Philox4x32-10 (Salmon et al., SC'11, the
 * generator the paper recommends in Sect. 5) of the counter
 *     (index, k, purpose | chain << 8, problem)  with key (seed lo, seed hi),
 * where k is the 1-based sweep number; purposes are z = 1, lambda = 2,
 * tau = 3, beta noise = 4, nu = 5, xi = 6.  Two 32-bit words (hi, lo) give
 * u = (2m + 1) 2^-53 with m = (hi << 20) | (lo >> 12).  Runs are therefore
 * bit-reproducible and resumable from a saved state.
 */
#ifndef HS_PROBIT_H
#define HS_PROBIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define HS_OK            0
#define HS_EINVAL       -1  /* bad argument (sizes, y not in {0,1}, NULL) */
#define HS_ENOMEM       -2  /* device or pinned host allocation failed */
#define HS_ECUDA        -3  /* a CUDA runtime call failed */
#define HS_ENOTPD       -4  /* X^T X + tau^{-2} Lambda^{-2} not positive definite */
#define HS_ENONFINITE   -5  /* a non-finite value appeared in X beta, z or beta */
#define HS_ETIMEOUT     -6  /* a bounded device wait ran out */
#define HS_ESTATE       -7  /* handle is in an error state; call set_state */
#define HS_EUNSUPPORTED -8  /* option not supported on this device or with these settings */

/* ---- storage type of X -------------------------------------------------- */
#define HS_X_F64      0  /* double; the sweep computes X beta and X^T z in FP64 */
#define HS_X_F32      1  /* float; FP32 arithmetic and accumulation */
#define HS_X_BF16     2  /* bfloat16 bit patterns (uint16); FP32 arithmetic */
#define HS_X_FP8E4M3  3  /* e4m3 codes (uint8) times a per-column FP32 scale */

/* ---- arithmetic of the p x p Cholesky and inverse factor ----------------- */
#define HS_CHOL_F64   0  /* native FP64 (GB300 runs FP64 at ~1/64 of the FP32 rate) */
#define HS_CHOL_DF32  1  /* FP32 pairs (~48-bit significand) on the FP32 pipe; default */

/* ---- launch schedule of the HS_CHOL_DF32 factorization -------------------
 * COLUMNS and SINGLE compute the same tiles with the same operations in the
 * same order, so their results are bit-identical. */
#define HS_SCHED_AUTO     0  /* TENSOR for several chains or p > 2016, else the single launch
                                where the device has cooperative launch, else columns */
#define HS_SCHED_COLUMNS  1  /* one launch per 32-wide block column (P / 32 launches) */
#define HS_SCHED_SINGLE   2  /* one cooperative launch, tiles scheduled by data readiness;
                                init fails with HS_EUNSUPPORTED where the device lacks it */
#define HS_SCHED_TENSOR   3  /* block columns of 128: each block column factored by the
                                readiness-scheduled FP32-pair tile tasks (one launch), the
                                rank-128 updates of the matrix to its right as exact
                                products of BF16 digits on the tensor cores (one launch);
                                factor only, so beta comes by substitution (HS_BETA_SUBST
                                or AUTO); not bit-identical to the other two schedules */

/* ---- how beta is drawn from the factor -----------------------------------
 * beta = S L~^{-T} (L~^{-1} S X^T z + s) either way (Sect. 5, beta update);
 * the two forms round differently (agreement to about 1e-12 relative). */
#define HS_BETA_AUTO     0  /* HS_BETA_SUBST on the single-launch schedule for several
                                chains or p > 2016, else HS_BETA_INVERSE */
#define HS_BETA_INVERSE  1  /* the factorization also forms L~^{-1}; beta by two
                                parallel matrix-vector products */
#define HS_BETA_SUBST    2  /* factor only (half the tile products); beta by block
                                forward and back substitution, one block per chain;
                                needs HS_CHOL_DF32 on the single-launch schedule,
                                else init fails with HS_EUNSUPPORTED */

typedef struct hs_probit hs_probit;  /* opaque handle */

typedef struct hs_probit_config {
  int32_t x_dtype;     /* HS_X_*; hs_probit_init uses HS_X_F32 */
  int32_t x_is_device; /* 1: X, y and x_scales are device pointers (copied);
                          HS_X_ADOPT: as 1, but X is used in place (see hs_probit_init_ex) */
  int32_t thin;        /* keep every thin-th sweep in the draw ring (>= 1) */
  int32_t ring_size;   /* number of draws the device ring holds (>= 1) */
  int32_t debug;       /* 1: keep z and X^T z of the last sweep for debug_* */
  int32_t use_graph;   /* 1: replay each sweep as a captured CUDA graph */
  int32_t chol_arith;  /* HS_CHOL_* */
  int32_t device;      /* CUDA device ordinal */
  uint32_t chain;      /* chain id in the counter (0..2^24-1) */
  uint32_t problem;    /* problem id in the counter */
  void* stream;        /* cudaStream_t for the sweep; NULL: library-owned stream */
  const float* x_scales; /* HS_X_FP8E4M3 only: p column scales (host or device) */
  int32_t chol_sched;  /* HS_SCHED_*; ignored for HS_CHOL_F64 */
  int32_t num_chains;  /* K independent chains sharing X (1..32) */
  int32_t beta_solve;  /* HS_BETA_* */
  int32_t update_mask; /* test hook: 0 = every variable is drawn (the sampler); otherwise
                          only the HS_UPD_* variables set here are drawn each sweep, the
                          others keep their values (z and beta are always drawn) */
  int32_t reserved[4];
} hs_probit_config;

/* cfg.x_is_device value: adopt the caller's device X without a copy. */
#define HS_X_ADOPT 2

/* Bits of cfg.update_mask (Eq. 12: the shrinkage variables). */
#define HS_UPD_LAMBDA 1  /* lambda_j^{-2} */
#define HS_UPD_TAU    2  /* tau^{-2} */
#define HS_UPD_NU     4  /* nu_j^{-1} */
#define HS_UPD_XI     8  /* xi^{-1} */

/* Values of one sampler state (Eq. 12 variables).  Arrays are host memory of
 * length p owned by the caller. */
typedef struct hs_probit_state_view {
  double* beta;        /* beta_j */
  double* lambda_inv2; /* lambda_j^{-2} */
  double* nu_inv;      /* nu_j^{-1} */
  double tau_inv2;     /* tau^{-2} */
  double xi_inv;       /* xi^{-1} */
  int64_t k;           /* sweeps done; the next sweep uses counter k + 1 */
} hs_probit_state_view;

/* Fill *cfg with defaults: F32 host X, thin 1, ring 1024, no debug, no graph,
 * HS_CHOL_DF32 with HS_SCHED_AUTO, device 0, chain 0, problem 0, library stream,
 * one chain. */
void hs_probit_config_default(hs_probit_config* cfg);

/* Create a sampler for host X (float32, N x p row-major) and host y (N bytes in
 * {0,1}) with the cold start of Sect. 6.1 (beta = 0; lambda = nu = tau = xi = 1).
 * N >= 2 (Sect. 4, Eq. 1) and 1 <= p <= 8192 (4096 for FP64 X).  X and y are copied; the
 * one-time Gram matrix X^T X (Sect. 5, beta update, step i) is formed in FP64
 * on the GPU.  Returns NULL on error; hs_probit_last_error() gives the status. */
hs_probit* hs_probit_init(const float* X, const uint8_t* y, int64_t N, int64_t p,
                          uint64_t seed);

/* As hs_probit_init with a configuration.  X is of type cfg->x_dtype (double,
 * float, uint16 bf16 bits or uint8 e4m3 codes), host or device per
 * cfg->x_is_device, and copied; with cfg->x_is_device = HS_X_ADOPT the
 * device X is used in place instead (zero copy, e.g. a torch CUDA tensor):
 * its rows must be 16-byte multiples (p * element size) and X 16-byte
 * aligned, else HS_EINVAL; the caller keeps X alive and unchanged until
 * hs_probit_free.  For HS_X_FP8E4M3 the value of X[i][j] is
 * x_scales[j] * e4m3(X[i][j]).  cfg may be NULL (defaults). */
hs_probit* hs_probit_init_ex(const hs_probit_config* cfg, const void* X, const uint8_t* y,
                             int64_t N, int64_t p, uint64_t seed);

/* Status of the last failed hs_probit_init / hs_probit_init_ex in this thread. */
int hs_probit_last_error(void);

/* Static text for a status code. */
const char* hs_probit_status_string(int status);

/* Run n_iter >= 0 Gibbs sweeps (Sect. 5, schedule (i)-(ii)) on the handle's
 * stream and wait for them.  Returns HS_OK, or the first device error seen
 * (HS_ENOTPD, HS_ENONFINITE, HS_ETIMEOUT).  After an error the state stays at
 * the last good sweep and further sweeps return HS_ESTATE until
 * hs_probit_set_state. */
int hs_probit_sweep(hs_probit* h, int64_t n_iter);

/* Copy the oldest undrained recorded draws into caller host arrays:
 * beta[d * p + j], lambda_inv2[d * p + j], tau_inv2[d] for d < returned count.
 * Any of the three pointers may be NULL.  At most max_draws are copied; draws
 * older than the last ring_size recorded ones are lost.  Returns the count
 * (>= 0) or a status < 0. */
int64_t hs_probit_draws(hs_probit* h, double* beta, double* lambda_inv2, double* tau_inv2,
                        int64_t max_draws);

/* Number of recorded, undrained draws (capped at the ring size), or < 0. */
int64_t hs_probit_draws_available(const hs_probit* h);

/* Copy the current state into caller host arrays (out->beta, out->lambda_inv2,
 * out->nu_inv must each hold p doubles; NULL arrays are skipped). */
int hs_probit_get_state(const hs_probit* h, hs_probit_state_view* out);

/* Replace the state (all three arrays required) and clear a sticky error.
 * The next sweep is number in->k + 1.  Values are not validated beyond
 * finiteness of the scalars; a state that makes the precision matrix
 * indefinite is reported by the next sweep as HS_ENOTPD. */
int hs_probit_set_state(hs_probit* h, const hs_probit_state_view* in);

/* z of the last sweep (N doubles, host), if the handle was made with debug = 1. */
int hs_probit_debug_z(hs_probit* h, double* z_out);

/* X^T z of the last sweep (p doubles, host), if made with debug = 1. */
int hs_probit_debug_xtz(hs_probit* h, double* xtz_out);

/* The Gram matrix X^T X in FP64 (p x p row-major, host). */
int hs_probit_gram(hs_probit* h, double* G_out);

/* Sizes of the handle: N, p and the CUDA stream the sweep runs on
 * (cudaStream_t as void*).  Any out pointer may be NULL. */
int hs_probit_info(const hs_probit* h, int64_t* N, int64_t* p, void** stream);

/* Profiling.  While on, CUDA events on the launching stream bracket each
 * kernel group (in a captured graph, as event-record nodes re-pointed at fresh
 * events before each launch); hs_probit_kernel_time
 * returns the summed milliseconds and the number of launches timed since
 * profiling was switched on.  which: 0 X-stream kernel, 1 X^T z reduce,
 * 2 lambda/tau kernel, 3 Cholesky+inverse branch (all its launches),
 * 4 beta/nu/xi tail, 5 Gram (setup). */
int hs_probit_set_profiling(hs_probit* h, int on);
int hs_probit_kernel_time(hs_probit* h, int which, double* total_ms, int64_t* launches);

/* Number of kernel launches one sweep makes (for launch accounting). */
int64_t hs_probit_launches_per_sweep(const hs_probit* h);

/* Failure-path test hook: run a kernel that waits, at most max_spins polls,
 * on a device flag that nothing sets.  Returns HS_ETIMEOUT (the wait ran out
 * and the kernel returned normally) or HS_ECUDA.  Does not touch the state. */
int hs_probit_debug_wait_timeout(hs_probit* h, int64_t max_spins);

/* The factorization's work matrix of one chain after the last sweep (FP32
 * pairs as doubles, P x P row-major with P = 32 ceil(p / 32), host): the
 * tiles on and below the diagonal hold the factor L~ of the equilibrated
 * precision matrix (strictly lower tiles; a diagonal tile holds the updated
 * block it was factored from).  HS_EUNSUPPORTED for HS_CHOL_F64.  For
 * diagnosis. */
int hs_probit_debug_factor(hs_probit* h, int chain, double* L_out);

/* The device error word the last hs_probit_sweep (or init) read back: the
 * status bits behind HS_ENOTPD, HS_ENONFINITE, HS_ETIMEOUT, and, for a bounded
 * wait that ran out, one bit per place that gave up (bit 8 + site: 0 and 1
 * the factorization's diagonal chain, 2 its tile tasks, 3 to 5 the loads, MMA
 * issue and epilogue of the tensor-core trailing updates, 6 the chain's SM
 * election).  For diagnosis; *word receives it. */
int hs_probit_debug_error_word(const hs_probit* h, int* word);

/* The X-stream of one sweep on caller-owned buffers, allocating nothing.
 * (The paper has no counterpart; this is a deployment entry point.)
 *
 * For callers that must not call cudaMalloc while they run: cudaMalloc can
 * synchronize the whole device and takes memory outside the caller's own
 * pool, so a runtime that plans all device memory up front, or a
 * latency-critical loop that treats a device-wide synchronization as a fault,
 * cannot create a handle (which allocates work buffers) mid-run.  This entry
 * point runs the same kernels as the X-stream part of hs_probit_sweep:
 *   z_i = y*_i TN+(y*_i x_i beta) with the counters of sweep number `sweep`
 *   (purpose z, `chain`, `problem`, key `seed`), and X^T z.
 * All arguments are device pointers on the current device:
 *   X       N rows of type x_dtype with row stride ld elements, starting on a
 *           16-byte boundary; ld * element size must be a multiple of 16
 *           bytes; columns p..ld-1 must be zero.
 *   y       N bytes in {0, 1} (not checked here).
 *   beta_c  ld values, double for HS_X_F64 and float otherwise (naturally
 *           aligned), equal to beta_j * x_scales[j] (FP8) or beta_j, zero
 *           for j >= p.
 *   x_scales p floats for HS_X_FP8E4M3 (multiplied into X^T z); must be NULL
 *           for every other x_dtype.
 *   xtz     output, p doubles.   z  output, N doubles, or NULL.
 *   stream  cudaStream_t or NULL.
 * The call is synchronous: it waits for its own work on `stream` and reads
 * the device error word back, so it cannot be called while `stream` (or the
 * legacy default stream) is being captured into a CUDA graph.
 * The per-block partial sums live in one fixed device array of 4 MiB
 * (plus a 256-byte header) that every GPU loading the library holds until
 * the process exits: sizes whose partials (one row of ld values per SM)
 * exceed it are rejected with HS_EINVAL, as are p > 8192 and ld > 16384.
 * Every argument check is made on the host before any CUDA call.  The first
 * call on a device looks up that array's device address (no allocation) and
 * keeps it for the life of the process, so the entry point must not be used
 * on a device after cudaDeviceReset.  Every call shares the array: calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialized by the caller.  The error word in the array is cleared by each
 * call.  Returns HS_OK, HS_EINVAL, HS_ENONFINITE, HS_ETIMEOUT or HS_ECUDA. */
int hs_probit_xstream_noalloc(int x_dtype, const void* X, int64_t ld, const uint8_t* y, int64_t N,
                              int64_t p, const void* beta_c, const float* x_scales, uint64_t seed,
                              uint32_t chain, uint32_t problem, int64_t sweep, double* xtz, double* z,
                              void* stream);

/* The worker task list of the single-launch factorization for T tiles of 32
 * (host only; no CUDA call): the order the kernel hands out its tile tasks,
 * one code per task, kind | k << 2 | i << 10 | j << 18 with kind 0 = C(i,k)
 * (L_ik = A_ik L_kk^{-T}), 1 = X(k,j) (X_kj = L_kk^{-1} B_kj), 2 = UA(i,j,k)
 * (A_ij -= L_ik L_jk^T), 3 = UB(i,j,k) (B_ij -= L_ik X_kj); inverse = 0 lists
 * the factor-only form (kinds 0 and 2).  A C entry carries j = k + 1: that
 * task also applies UA(i,k+1,k) from the L_ik it holds, and the list leaves
 * UA(i,k+1,k) out.  The list is a topological order of the task graph (with
 * those updates merged), found by a list schedule for `workers` concurrent tasks.
 * Writes min(count, max_codes) codes to the caller's array and returns the
 * count, or HS_EINVAL (T outside 1..256, workers < 1, inverse not 0 or 1,
 * max_codes < 0, codes NULL with max_codes > 0). */
int64_t hs_chol_task_list(int32_t T, int32_t workers, int32_t inverse, int32_t* codes, int64_t max_codes);

/* The worker task list of one block-column launch of the HS_SCHED_TENSOR
 * factorization (host only; no CUDA call): tile columns [k0, k1) of T tiles,
 * the tasks C(i, k) and UA(i, j, k) with j < k1 in the order the kernel hands
 * them out (a list schedule for `workers` concurrent tasks, like
 * hs_chol_task_list), as codes of hs_chol_task_list (C entries with j = k:
 * nothing merged).  Writes
 * min(count, max_codes) codes and returns the count, or HS_EINVAL (T outside
 * 1..256, not 0 <= k0 < k1 <= T, workers < 1, max_codes < 0, codes NULL with
 * max_codes > 0). */
int64_t hs_chol_block_task_list(int32_t T, int32_t k0, int32_t k1, int32_t workers, int32_t* codes,
                                int64_t max_codes);

/* ---- K chains on one X (Sect. 5 sweep for each chain; batched form) --------
 * A handle made with cfg.num_chains = K > 1 runs K independent chains on the
 * same X.  Chain m uses chain id cfg.chain + m in its Philox counters, so
 * it is the same transition as a one-chain handle with that chain id.  For
 * BF16 and FP8 X the X-stream of all K chains runs on the tensor cores
 * (eta = X B and X^T Z as BF16 products, beta and z each split into two BF16
 * parts, FP8 codes converted to BF16 exactly, FP32 accumulation): one pass
 * over X for BF16 X with p <= 1536 (K > 16) or p <= 3584 (K <= 16), else
 * two passes (eta and the z draws, then X^T Z) for p <= 2048 (K > 16) or
 * p <= 4096 (K <= 16); other cases take one pass of the one-chain X-stream
 * per chain.  The
 * factorizations of all chains are one launch (on the single-launch
 * schedule, by default without the inverse factor, beta then coming from
 * block substitution: see beta_solve), and the other steps run per chain.
 * The sweep count k is shared: hs_probit_sweep advances every chain, and the
 * last set_state call sets k for all of them.  The functions without a chain
 * argument act on chain 0. */

/* Asynchronous form of hs_probit_draws_chain: starts copying up to
 * max_draws of the chain's unread draws into the caller's host buffers on a
 * side stream and returns the count at once, so the copy runs while later
 * sweeps compute (Sect. 5: Monte Carlo output downloaded through CUDA
 * streams while the sampler runs).  Page-locked buffers make the copy truly
 * asynchronous; the buffers must stay valid, and are not to be read, until
 * hs_probit_draws_wait returns.  A later sweep that would overwrite a ring
 * slot still being copied waits for the copy first. */
int64_t hs_probit_draws_async(hs_probit* h, int chain, double* beta, double* lambda_inv2, double* tau_inv2,
                              int64_t max_draws);
/* Wait for every copy started by hs_probit_draws_async on the handle. */
int hs_probit_draws_wait(hs_probit* h);

/* Number of chains of the handle (>= 1), or HS_EINVAL. */
int hs_probit_num_chains(const hs_probit* h);

/* hs_probit_get_state / set_state for chain 0 <= chain < K.  HS_EINVAL for a
 * chain out of range. */
int hs_probit_get_state_chain(const hs_probit* h, int chain, hs_probit_state_view* out);
int hs_probit_set_state_chain(hs_probit* h, int chain, const hs_probit_state_view* in);

/* hs_probit_draws_available / hs_probit_draws for one chain (each chain keeps
 * its own read position). */
int64_t hs_probit_draws_available_chain(const hs_probit* h, int chain);
int64_t hs_probit_draws_chain(hs_probit* h, int chain, double* beta, double* lambda_inv2, double* tau_inv2,
                              int64_t max_draws);

/* Debug copies (cfg.debug) of the last sweep's z (N values) and X^T z (p
 * values) of one chain; host buffers owned by the caller. */
int hs_probit_debug_z_chain(hs_probit* h, int chain, double* z_out);
int hs_probit_debug_xtz_chain(hs_probit* h, int chain, double* xtz_out);

/* ---- launch shapes ---------------------------------------------------------
 * Grid and tile sizes of a handle's kernels.  They change how the work of a
 * sweep is spread over the GPU, never what a sweep computes: every shape
 * gives the same transition (bit for bit for everything but the order of
 * the X^T z partial sums, which depends on the X-stream's CTA count).  The
 * batch tuner (below) sets them; hs_probit_set_launch_shape lets a caller do
 * the same.  A field of 0 leaves that size as it is. */
typedef struct hs_launch_shape {
  int32_t xk_chains;    /* chain columns of a tensor-core X-stream tile: 16 (K <= 16) or 32 */
  int32_t xk_stages;    /* shared-memory ring stages of that X-stream: 4, 6 or 8 (the two-pass form
                           has one fixed value per width) */
  int32_t xstream_ctas; /* CTAs of the X-stream: 1 .. the value the handle started with (for the
                           tensor-core X-stream, x 32 / xk_chains, at most one per 128 rows) */
  int32_t chol_ctas;    /* blocks of each factorization launch: K + 1 .. the starting value */
  int32_t trail_ctas;   /* CTAs of the tensor-core trailing updates: 1 .. the starting value */
  int32_t xk_ctas_per_sm; /* CTAs per SM the tensor-core X-stream is built for: 1, or 2 with 16
                             chain columns, 4 stages and p <= 1536 (half the TMEM each) */
  int32_t overlap;      /* K chains: 1 = the factorization runs beside the X-stream, 2 = after it
                           (the starting value); one chain always overlaps */
  int32_t reserved[1];  /* must be 0 */
} hs_launch_shape;

/* Current shapes (fields that do not apply to the handle read 0). */
int hs_probit_get_launch_shape(const hs_probit* h, hs_launch_shape* out);
/* Set shapes; waits for the handle's work in flight and drops its captured
 * graph.  HS_EINVAL for a size out of range (nothing is changed),
 * HS_EUNSUPPORTED for X-stream tile fields on a handle without the
 * tensor-core X-stream. */
int hs_probit_set_launch_shape(hs_probit* h, const hs_launch_shape* in);

/* ---- many problems in one launch (Sect. 4: exchangeable models) ------------
 * The sweep applies to any data-augmented model with an exchangeable
 * likelihood (Sect. 4, Eqs. 1-3); a batch runs n independent Horseshoe probit
 * problems of uneven N and p side by side, each with K = cfg->num_chains
 * chains.  Problem m is an ordinary handle made by hs_probit_init_ex(cfg', X_m,
 * y_m, N_m, p_m, seed) with cfg'.problem = cfg->problem + m (its own Philox
 * counter field, so its transition is exactly that handle's) and
 * cfg'.x_scales = problems[m].x_scales.  One call of hs_probit_batch_sweep
 * replays, per sweep, a single CUDA graph holding every problem's sweep on
 * branches of its own, so the problems' kernels share the GPU. */
typedef struct hs_problem {
  const void* X;          /* N x p of cfg->x_dtype; host, or device if cfg->x_is_device (copied) */
  const uint8_t* y;       /* N values in {0, 1}; same memory kind as X (copied) */
  int64_t N;              /* >= 2 */
  int64_t p;              /* >= 1 */
  const float* x_scales;  /* p column scales for HS_X_FP8E4M3, else NULL */
} hs_problem;

typedef struct hs_probit_batch hs_probit_batch;  /* opaque */

/* Make n >= 1 problems (problems: host array of n).  cfg->stream, if set, is
 * the stream the batch's graph is launched on; cfg->use_graph is ignored.
 * NULL on error; hs_probit_last_error() gives the status. */
hs_probit_batch* hs_probit_batch_init(const hs_probit_config* cfg, int32_t n, const hs_problem* problems,
                                      uint64_t seed);
/* Number of problems, or HS_EINVAL. */
int32_t hs_probit_batch_size(const hs_probit_batch* b);
/* Problem m's handle (owned by the batch): draws, get/set_state, launch
 * shapes (the batch recaptures its graph after a change) and the debug copies
 * work on it as on any handle; hs_probit_free ignores it (the batch releases
 * it).  NULL if m is out of range. */
hs_probit* hs_probit_batch_problem(hs_probit_batch* b, int32_t m);
/* n_iter sweeps of every problem.  HS_ESTATE if a problem is in an error
 * state; otherwise the first failing problem's status (the others' states
 * are valid). */
int hs_probit_batch_sweep(hs_probit_batch* b, int64_t n_iter);
/* The autotuner: times trial launch shapes over `sweeps` sweeps each and
 * keeps the fastest.  Candidates: for each problem, X-stream CTAs, trailing-
 * update CTAs and factorization blocks in proportion to its share of the
 * batch's X bytes and factorization work, at four oversubscription factors;
 * then the factorization blocks' factor alone (1/8 .. 2 of that); then the
 * tensor-core X-stream's tile (chain columns, ring stages, CTAs per SM); then
 * the K chains' factorization beside the X-stream instead of after it.  Every problem's
 * state is saved first and restored after, so tuning leaves the chains where
 * they were.  *best_ms receives the best time per sweep (may be NULL). */
int hs_probit_batch_tune(hs_probit_batch* b, int32_t sweeps, double* best_ms);
/* One trial of the last hs_probit_batch_tune call. */
typedef struct hs_tune_trial {
  double ms_per_sweep;  /* measured time per batch sweep */
  double oversub;       /* oversubscription factor of the X-stream and trailing-update shares */
  double chol_oversub;  /* factor of the factorization blocks' shares */
  int32_t xk_chains;    /* tensor-core X-stream chain columns tried (0: unchanged) */
  int32_t xk_stages;    /* its ring stages tried (0: unchanged) */
  int32_t xk_ctas_per_sm; /* its CTAs per SM tried (0: unchanged) */
  int32_t overlap;      /* launch-shape overlap tried (1 beside, 2 after) */
} hs_tune_trial;
/* Copies up to max trials into out (host); returns the number of trials. */
int32_t hs_probit_batch_tune_trials(const hs_probit_batch* b, hs_tune_trial* out, int32_t max);
/* Release the batch and its problems.  NULL is allowed. */
void hs_probit_batch_free(hs_probit_batch* b);

/* Release the handle and everything it owns.  NULL is allowed. */
void hs_probit_free(hs_probit* h);

#ifdef __cplusplus
}
#endif

#endif /* HS_PROBIT_H */

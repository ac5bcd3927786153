// Host-side declarations shared by the translation units of the library
// (kernel launchers and their parameter blocks).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <vector>
#include <stdint.h>

namespace hs {

// ---- device error word bits (atomicOr into one int) -----------------------
enum : int {
  kErrNonFinite = 1,   // non-finite eta, z or beta
  kErrNotPD = 2,       // non-positive pivot in the Cholesky factor
  kErrTimeout = 4,     // a bounded wait ran out
  kErrGamma = 8,       // Cheng's sampler found no acceptance in its round cap
  kErrBadY = 16,       // a y value outside {0, 1}
};
// A bounded wait that runs out also ORs 1 << (kErrSiteShift + site) into the
// word, naming where it gave up (hs_probit_debug_error_word).
constexpr int kErrSiteShift = 8;
enum : int {
  kSiteChainStart = 0,   // factorization: the chain's first diagonal tile of a block column
  kSiteChainStep = 1,    // factorization: the chain's tiles of the next step
  kSiteTask = 2,         // factorization: a worker task's inputs
  kSiteTrailLoad = 3,    // trailing updates: a free stage for the loads
  kSiteTrailMma = 4,     // trailing updates: loaded digits or a free accumulator
  kSiteTrailEpi = 5,     // trailing updates: finished classes
  kSiteStartRole = 6,    // factorization: the chain's SM mark
};

// Philox key and the fixed parts of the counter.
struct RngKey {
  uint32_t k0, k1, chain, problem;
};

// ---- X-stream: eta = X beta, z ~ TN, per-CTA partial sums of X^T z ---------
struct XStreamArgs {
  const void* X;         // N x ld storage type, rows 16-byte aligned, pads zero
  const uint8_t* y;      // N
  int64_t N;
  int ld;                // row stride in elements (multiple of 16 bytes)
  int p;
  const void* beta_c;    // ld values of the compute type (double or float)
  void* partials;        // grid x ld compute-type partial sums (written)
  double* z_out;         // N, or nullptr
  const int64_t* k_dev;  // sweeps done; this sweep is *k_dev + 1
  RngKey rng;
  int* err;
  unsigned int* sm_mark;  // or nullptr: each block writes the sweep number at [its SM id] (< kSmMarks)
};
constexpr int kSmMarks = 1024;

// ---- batched X-stream of K chains on the tensor cores (BF16 X) ---------------
struct XKArgs {
  const uint8_t* y;       // N
  int64_t N;
  int p;
  int nch;                // 64-feature chunks (even)
  int fpad;               // nch * 64
  int K;                  // chains (<= kc)
  int kc;                 // chain columns of the launch shape (16 or 32)
  int stages;             // ring stages of the launch shape (4, 6 or 8)
  int per_sm;             // CTAs per SM of the launch shape (1, or 2 for kc 16 with 4 stages)
  const void* bsw;        // nch x (kc x 256 B): B^T (BF16 high and low parts), swizzled for the MMA
  float* partials;        // grid x fpad x kc FP32 (written)
  double* z_out;          // K x N (chain-major), or nullptr
  const int64_t* k_dev;   // sweeps done; this sweep is *k_dev + 1
  RngKey rng;             // rng.chain is chain 0's id; chain m uses rng.chain + m
  int* err;
  unsigned int* sm_mark;  // or nullptr, as XStreamArgs::sm_mark
  // the split form (xstream_k_split_enqueue): X stored as FP8 codes or BF16,
  // column scales (FP8) folded into B^T and into X^T Z, and the Z^T tiles
  // the first kernel writes for the second
  int fp8;                // 1: X holds e4m3 codes
  const float* colscale;  // p column scales, or nullptr
  void* zt;               // ceil(N / 128) x 4 x kc x 128 B
};
int xstream_k_chunks(int p);
// Launch shapes: kc chain columns (16 or 32), stages ring stages (4, 6 or 8).
// per_sm: CTAs per SM the kernel is compiled for (2 only with kc 16, 4 stages).
bool xstream_k_supported(int p, int kc, int stages, int per_sm);
int xstream_k_default_kc(int K);
constexpr int kXkDefaultStages = 8;
size_t xstream_k_smem_bytes(int kc, int stages);
cudaError_t xstream_k_prepare(int kc, int stages, int per_sm);
int xstream_k_grid(int64_t N, int num_sms);
int64_t xstream_k_tiles(int64_t N);
size_t xstream_k_partial_floats(int p, int grid, int kc);
size_t xstream_k_bsw_bytes(int p, int kc);
// Tensor map of BF16 X (N rows, ld columns) into map_out (128 bytes, 64-byte aligned); 0 on success.
int xstream_k_make_map(const void* X, int64_t N, int ld, void* map_out);
// B^T preparation and the X-stream kernel; then the fixed-order reduce of the partials.
cudaError_t xstream_k_enqueue(const void* map, const XKArgs& a, const double* beta, int64_t beta_stride,
                              unsigned char* bsw, int grid, cudaStream_t s);
cudaError_t xstream_k_reduce(const XKArgs& a, int grid, double* xtz, int64_t xtz_stride, cudaStream_t s);
// The split form: pass 1 (eta = X B, the z draws, Z^T to global memory) and
// pass 2 (X^T Z) as two kernels, so pass 2's TMEM holds every feature group
// (p up to 4096 at 16 chain columns, 2048 at 32) and X may be FP8 (converted
// to BF16 in shared memory, exactly).  X is read twice.
bool xstream_k_split_supported(int p, int kc);
cudaError_t xstream_k_split_prepare(int kc, int fp8);
size_t xstream_k_zt_bytes(int64_t N, int kc);
int xstream_k_split_stages(int kc);  // the split form's fixed ring stages
// Tensor map of FP8 X (N rows, ld columns of one byte): boxes of 64 x 128, no swizzle.
int xstream_k_make_map_fp8(const void* X, int64_t N, int ld, void* map_out);
cudaError_t xstream_k_split_enqueue(const void* map, const XKArgs& a, const double* beta, int64_t beta_stride,
                                    unsigned char* bsw, int grid, cudaStream_t s);

// Per-process kernel attributes (shared-memory carveout); call before launching.
cudaError_t xstream_prepare();
cudaError_t linalg_prepare();

// Persistent grid size (CTAs) the X-stream kernel uses for this shape.
int xstream_grid(int x_dtype, int p, int ld, int64_t N, int num_sms);
// Launch; returns cudaSuccess or the launch error.
cudaError_t xstream_launch(int x_dtype, const XStreamArgs& a, int grid, cudaStream_t s);
// Size in bytes of one partials row element (8 for F64 X, 4 otherwise).
int partial_elem_bytes(int x_dtype);

// X^T z = sum over CTAs of the partials (fixed order, FP64), times the column scale.
cudaError_t reduce_partials_launch(int x_dtype, const void* partials, int grid, int ld, int p,
                                   const float* colscale, double* xtz, cudaStream_t s);

// G = X^T X (p x p, FP64, row-major, full), X as stored (scaled for FP8), on
// the tensor cores with exact digit products (gram_tc.cu).  workspace:
// gram_workspace_bytes(N, p, num_sms) bytes of device memory, free after the
// call's work completes.  A bounded wait that runs out sets kErrTimeout in err.
size_t gram_workspace_bytes(int64_t N, int p, int num_sms);
cudaError_t gram_launch(int x_dtype, const void* X, int64_t N, int ld, int p, const float* colscale, double* G,
                        void* workspace, int num_sms, int* err, cudaStream_t s);

// y must be 0/1: sets kErrBadY in err otherwise.
cudaError_t check_y_launch(const uint8_t* y, int64_t N, int* err, cudaStream_t s);

// ---- shrinkage: lambda^{-2} (Exp), tau^{-2} (Cheng GB) and the scaling -------
struct ShrinkArgs {
  int p, P;
  RngKey rng;
  const int64_t* k_dev;
  const double* beta;     // current beta
  const double* lam;      // current lambda^{-2} (read only)
  const double* nu;       // current nu^{-1}
  const double* scal;     // [0] tau^{-2}, [1] xi^{-1} (current)
  double* lam_new;        // written
  double* tau_new;        // written (one value)
  const double* G;        // p x p (diagonal read)
  double* S;              // P: 1/sqrt(A_jj) rounded to FP32 (1 for padded j)
  double* part;           // ceil(p / 128) block partial sums and the Gamma variate (scratch)
  unsigned int* ticket;   // zero between sweeps (scratch)
  int* err;
  int update_mask;        // HS_UPD_* bits of the variables drawn (the others keep their values)
  int unit_diag;          // 1: S from the new tau^{-2} (unit diagonal, for the digit planes of the
                          // tensor-core trailing updates); 0: from the current tau^{-2}
};
// nchains > 1: chains 0..nchains-1 at fixed strides past a's buffers (blockIdx.y = chain)
cudaError_t shrink_launch(const ShrinkArgs& a, cudaStream_t s, int nchains = 1);

// ---- Cholesky of A = G + tau^{-2} Lambda^{-2} (scaled) and its inverse ------
struct CholArgs {
  int p, P;               // P = number of tiles * tile size
  const double* G;        // p x p
  const double* S;        // P
  const double* lam_new;  // p
  const double* tau_new;  // 1
  void* A;                // P x P workspace (double, or FP32 pairs); lower part becomes L~
  void* Linv;             // P x P; lower part becomes L~^{-1} (diagonal tiles only when !inverse)
  void* LinvT;            // P x P; upper part becomes L~^{-T} (when !inverse: diagonal tiles
                          // L~_kk^{-T}, off-diagonal tiles (k, i) the transposed factor L~_ik^T)
  int* err;
  int arith;              // HS_CHOL_*
  unsigned long long* sync;  // HS_CHOL_DF32 single-launch schedule: readiness words (chol_sync_words)
  int persistent_grid;       // > 0: that schedule with this many blocks; 0: one launch per block column
  const unsigned int* sm_mark;  // SMs the X-stream of this sweep occupies (XStreamArgs::sm_mark), or nullptr
  const int64_t* k_dev;         // sweeps done; this sweep is *k_dev + 1
  // Single-launch schedule for several chains at once: chain m's S, lam_new,
  // tau_new, A, Linv, LinvT and readiness words are at m times P, p, 1, P*P,
  // P*P and sync_words past the pointers above.
  int nchains;                  // 0 or 1: one chain
  size_t sync_words;
  const int* order;             // worker task list (chol_task_codes), or nullptr: canonical order
  int inverse;                  // single-launch schedule: 1 forms all of L~^{-1}; 0 only its diagonal tiles
  // Block-column launches (the trailing updates run on the tensor cores,
  // chol_trail_launch): this launch factors tile columns [k0, k1) only, runs
  // the ntasks entries of order, and writes the six BF16 digit planes of every
  // factor tile it forms below row tile k1 (digits: nchains x 6 planes of P x P).
  int k0, k1;                   // 0, 0: the whole matrix in one launch
  int ntasks;                   // entries of order (when order is given)
  void* digits;                 // or nullptr
  // block-column launches: per-SM claim and role words (2 x kSmMarks, zeroed
  // once) for placing the chains on SMs of their own; or nullptr
  unsigned long long* sm_role;
  int prebuilt;                 // 1: A already holds the equilibrated precision matrix
                                // (lower tiles), so no tile is formed from the Gram matrix
  // 1: the single-launch schedule launches cooperatively (all blocks resident);
  // 0: an ordinary launch, for grids that share the GPU with other work (the
  // tasks are taken in list order and wait only on earlier ones or on the
  // chains, which the first blocks to start walk, so residency is not needed)
  int cooperative;
};
// Enqueues the whole factorization; *launches receives the kernel count.
cudaError_t chol_enqueue(const CholArgs& a, cudaStream_t s, int* launches);
int chol_launch_count(int P, int arith, int persistent_grid);
// Readiness words the single-launch FP32-pair schedule needs (zeroed once).
size_t chol_sync_words(int P);
// Blocks for the single-launch schedule on the current device (all resident
// at once: one per SM for one chain, as many as fit for several), or 0 where
// cooperative launch is unavailable.
int chol_persistent_grid(int device, int nchains = 1);
// Worker task list of the single-launch factorization for T tiles and about
// `workers` concurrent task slots (a topological order; see linalg.cu).
std::vector<int> chol_task_order(int T, int workers, bool inverse);
// The same list with each entry decoded for the kernel: kind (0 C, 1 X, 2 UA,
// 3 UB) | k << 2 | i << 10 | j << 18 (T <= 256); a C(i,k) entry carries
// j = k + 1: the task also applies UA(i,k+1,k), which the list leaves out.
std::vector<int> chol_task_codes(int T, int workers, bool inverse);

// Task list of one block-column launch (tile columns [k0, k1) of T): C(i, k) and
// the updates UA(i, j, k) with j < k1, as codes kind | k << 2 | i << 10 | j << 18,
// in the start order of a list schedule for about `workers` concurrent task slots.
std::vector<int> chol_block_task_codes(int T, int k0, int k1, int workers);

// ---- trailing updates on the tensor cores (chol_trail.cu) -------------------
// Tile columns per block column of the HS_SCHED_TENSOR factorization.
constexpr int kTrailBlockTiles = 4;
struct TrailArgs {
  int p, P, nchains;
  int b;                        // block column (tiles kTrailBlockTiles b ..)
  int col_lo, col_hi;           // output tile columns [col_lo, col_hi) of this launch
  void* A;                      // nchains x P x P FP32 pairs (tiles of A~ and of L~)
  const void* G2;               // P x P FP32 pairs of the Gram matrix (first block column only)
  const double* S;              // nchains x P equilibration
  const double* lam_new;        // nchains x p
  const double* tau_new;        // nchains
  unsigned long long* sync;     // readiness words (chol_sync_words per chain); [0] holds the launch epoch
  size_t sync_words;
  int* err;
};
size_t chol_trail_smem_bytes();
cudaError_t chol_trail_prepare();
int chol_trail_make_maps(const void* digits, int P, int nchains, void* mapA, void* mapB);
int chol_trail_items(int P, int b, int col_lo, int col_hi, int nchains);
cudaError_t chol_trail_launch(const void* mapA, const void* mapB, const TrailArgs& a, int grid, cudaStream_t s);
cudaError_t gram_pairs_launch(const double* G, int p, int P, void* G2, cudaStream_t s);
// A~ = S (G + tau Lambda) S into the work matrix of every chain (lower tiles, FP32 pairs)
cudaError_t precision_pairs_launch(const TrailArgs& a, cudaStream_t s);

// ---- beta tail, nu/xi, commit ----------------------------------------------
struct TailArgs {
  int p, P, ld;
  RngKey rng;
  const int64_t* k_dev;
  const double* xtz;       // p
  const double* S;         // P
  const void* Linv;        // P x P lower (double, or FP32 pairs when df32)
  const void* LinvT;       // P x P upper (same storage)
  int df32;
  // solve != 0 (FP32 pairs, factorization with inverse == 0): beta by block
  // substitution with the factor's tiles, L~_ik in L (tile (i, k), i > k),
  // L~_ik^T in LinvT (tile (k, i)) and L~_kk^{-1} in Linv (tile (k, k))
  int solve;
  const void* L;           // P x P factor tiles (CholArgs::A)
  double* v;               // P scratch: L^{-1} X^T z + s (substitution form: s)
  double* beta_new;        // p
  double* nu_new;          // p
  const double* lam_new;   // p
  const double* tau_new;   // 1
  // state committed when the error word is clear
  double* beta;            // p
  double* lam;             // p
  double* nu;              // p
  double* scal;            // [0] tau^{-2}, [1] xi^{-1}
  int64_t* k_dev_rw;       // incremented on commit
  void* beta_c;            // ld compute-type copy of beta (times column scale)
  int beta_c_is_double;
  const float* colscale;   // p or nullptr
  double* ring_beta;       // ring x p
  double* ring_lam;        // ring x p
  double* ring_tau;        // ring
  int ring_size, thin;
  int* err;
  int update_mask;         // HS_UPD_* bits of the variables drawn (the others keep their values)
};
// The beta tail in two parts: the beta and nu draws, then the commit (every
// chain's commit must follow every chain's draws).
cudaError_t tail_draw_enqueue(const TailArgs& a, cudaStream_t s, int nchains = 1);
cudaError_t commit_enqueue(const TailArgs& a, cudaStream_t s, int nchains = 1);
// Substitution form and FP32-pair factors (TailArgs::solve or df32): the s_j
// and nu_j^{-1} draws, which must precede tail_draw_enqueue and follow the
// shrink kernel; no-op otherwise (the FP64 products draw them themselves).
cudaError_t tail_noise_enqueue(const TailArgs& a, cudaStream_t s, int nchains = 1);

// beta_c = (compute type)(beta * colscale), pads zero.
cudaError_t beta_c_launch(const double* beta, const float* colscale, int p, int ld, void* beta_c,
                          int is_double, cudaStream_t s);

// Test hook: wait on a device flag nothing sets, at most max_spins polls.
cudaError_t wait_timeout_launch(int* flag, int64_t max_spins, int* err, cudaStream_t s);


}  // namespace hs

// The p-dimensional steps of one Gibbs sweep.
//
//  shrink   lambda_j^{-2} ~ Exp(nu_j^{-1} + tau^{-2} beta_j^2 / 2) by inversion
//           (Eq. 12, second line; Sect. 5, lambda/nu/xi update), then
//           tau^{-2} ~ Gamma((p+1)/2, rate xi^{-1} + sum_j lambda_j^{-2} beta_j^2 / 2)
//           (Eq. 12, fifth line) by Cheng's (1977) algorithm GB: one warp makes
//           32 proposals per round and keeps the lowest accepted lane
//           (Sect. 5, tau update, steps a to c; a ballot replaces the scan).
//  chol     A = X^T X + tau^{-2} Lambda^{-2} (Eq. 12 and the definition of Sigma
//           after it; Sect. 5, beta update, steps ii and iii).  The factor is
//           taken of the equilibrated matrix A~ = S A S, S = diag(A)^{-1/2},
//           by a right-looking blocked Cholesky over 32 x 32 tiles, and (one
//           chain, moderate p) the same sweep over the tiles forms L~^{-1} by
//           block forward substitution on the identity.  L = S^{-1} L~, so
//           L^{-1} = L~^{-1} S.
//  tail     w = L^{-1} X^T z, s_j = Phi^{-1}(u_j), beta = L^{-T}(w + s)
//           (Sect. 5, beta update, steps iv to viii, with the transposes read
//           so that Cov(beta) = A^{-1}), as two parallel products with the
//           explicit inverse factor, or (several chains, large p) by block
//           forward and back substitution with the factor itself;
//           nu_j^{-1} ~ Exp(1 + lambda_j^{-2}) and xi^{-1} ~ Exp(1 + tau^{-2})
//           (Eq. 12, third and sixth lines); and the commit of the new state,
//           skipped when the error word is set.
#include <algorithm>
#include <queue>
#include <vector>

#include "df32.cuh"
#include "hs_common.cuh"
#include "hs_internal.h"
#include "hs_probit.h"

namespace hs {
namespace {

constexpr int NB = 32;  // Cholesky tile
// Unused dynamic shared memory requested by each block-step launch: with the
// X-stream's 129 KB resident, it leaves room for one step block per SM, so
// the latency-bound blocks that finish a block column do not share an SM
// with trailing-update blocks (measured: +3-4% sweeps/s).
constexpr int kStepPadBytes = 40 * 1024;

// ---------------------------------------------------------------------------
// shrink: lambda^{-2}, tau^{-2} and the equilibration S
// ---------------------------------------------------------------------------
constexpr int kShrinkThreads = 128;

// S_j = 1/sqrt(d) rounded to FP32 and returned exactly as a double.  Any
// positive diagonal scaling gives the same factorization mathematically
// (L = S^{-1} L~); FP32 keeps this off the FP64 pipe.  d is brought into FP32
// range by an even power of two first.
__device__ __forceinline__ double equil_scale(double d) {
  const int e = ilogb(d) & ~1;
  const float m = (float)scalbn(d, -e);
  return scalbn((double)rsqrtf(m), -e / 2);
}

// Several chains in one launch: blockIdx.y is the chain, whose buffers sit at
// fixed strides past chain 0's (p per vector, P per scaling, 2 scalars, one
// block partial per block of x) and whose counters use chain id + blockIdx.y.
__device__ __forceinline__ ShrinkArgs shrink_chain(ShrinkArgs a, int m) {
  const size_t p = (size_t)a.p;
  a.rng.chain += (uint32_t)m;
  a.beta += m * p;
  a.lam += m * p;
  a.nu += m * p;
  a.scal += 2 * m;
  a.lam_new += m * p;
  a.tau_new += m;
  a.S += (size_t)m * a.P;
  a.part += (size_t)m * (gridDim.x + 1);  // per chain: the block partials, then the Gamma variate
  a.ticket += m;
  return a;
}

// S_j for the diagonal d = G_jj + tau lambda_j^{-2} (1 and an error bit when
// d is not positive and finite).
__device__ __forceinline__ double shrink_scale(double d, int* err) {
  if (!isfinite(d)) {
    set_error(err, kErrNonFinite);
    return 1.0;
  }
  if (!(d > 0.0)) {
    set_error(err, kErrNotPD);
    return 1.0;
  }
  return equil_scale(d);
}

// Cheng (1977) GB for shape a = (p + 1) / 2 >= 1, one proposal per lane and
// round, the first accepted (round, lane) kept.  The accept test does not
// involve the rate, so this runs beside the lambda draws (warp 0 of block 0).
__device__ bool gamma_cheng_warp(const Rng& rng, uint32_t sweep, int p, int lane, double& g) {
  const double sh = 0.5 * (double)(p + 1);
  const double lam = sqrt(2.0 * sh - 1.0);
  const double bconst = sh - 1.3862943611198906;  // a - ln 4
  const double cconst = sh + lam;
  g = sh;
  for (int r = 0; r < 64; ++r) {
    const uint4 w = rng.words((uint32_t)(r * 32 + lane), sweep, kPurTau);
    double u1, uc1, u2, uc2;
    unit_pair(w.x, w.y, u1, uc1);
    unit_pair(w.z, w.w, u2, uc2);
    const double V = (log(u1) - log(uc1)) / lam;
    const double X = sh * exp(V);
    const bool acc = bconst + cconst * V - X >= 2.0 * log(u1) + log(u2);
    const unsigned m = __ballot_sync(0xffffffffu, acc);
    if (m) {
      g = __shfl_sync(0xffffffffu, X, __ffs(m) - 1);
      return true;
    }
  }
  return false;
}

// lambda^{-2} (one thread per j), the equilibration S, and tau^{-2}: block 0
// draws the Gamma variate and stores it past the block partials; the last
// block to finish sums the partials in a fixed order and applies the rate.
// Without the digit planes of the tensor-core trailing updates
// (ShrinkArgs::unit_diag == 0) S_j = 1/sqrt(G_jj + tau lambda_j^{-2}) takes
// the current tau^{-2}, so every block forms its own S without waiting for
// the new one: any positive diagonal scaling gives the same factorization
// (L = S^{-1} L~), and the FP32-pair arithmetic needs only range.  The digit
// planes need a unit diagonal (every factor entry in [-1, 1]), so there the
// last block forms S from the new tau^{-2}.
__global__ void __launch_bounds__(kShrinkThreads) shrink_kernel(ShrinkArgs a0) {
  const ShrinkArgs a = shrink_chain(a0, blockIdx.y);
  __shared__ double s_part[kShrinkThreads / 32];
  __shared__ double s_tau;
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t sweep = (uint32_t)(*a.k_dev + 1);
  const Rng rng{a.rng.k0, a.rng.k1, a.rng.chain, a.rng.problem};
  const double tau = a.scal[0];
  const int j = blockIdx.x * kShrinkThreads + tid;
  double part = 0.0;
  if (j < a.p) {
    const uint4 w = rng.words((uint32_t)j, sweep, kPurLambda);
    double u, uc;
    unit_pair(w.x, w.y, u, uc);
    const double bj = a.beta[j];
    const double l = (a.update_mask & HS_UPD_LAMBDA) ? -log(u) / (a.nu[j] + tau * bj * bj * 0.5) : a.lam[j];
    a.lam_new[j] = l;
    part = l * bj * bj;
    if (!a.unit_diag) a.S[j] = shrink_scale(a.G[(size_t)j * a.p + j] + tau * l, a.err);
  } else if (j < a.P && !a.unit_diag) {
    a.S[j] = 1.0;  // padding past p
  }
  if (blockIdx.x == 0 && warp == 0) {
    double g;
    const bool found = gamma_cheng_warp(rng, sweep, a.p, lane, g);
    if (lane == 0) {
      if (!found) set_error(a.err, kErrGamma);
      a.part[gridDim.x] = g;
    }
  }
  part = warp_sum(part);
  if (lane == 0) s_part[warp] = part;
  __syncthreads();
  if (tid == 0) {
    double bp = 0.0;
    for (int w = 0; w < kShrinkThreads / 32; ++w) bp += s_part[w];
    a.part[blockIdx.x] = bp;
    // release (the block's writes, ordered by the barrier) and acquire (the
    // last block reads every block's partial and block 0's variate) in one atomic
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(a.ticket) : "memory");
    s_last = (old == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  if (warp == 0) {
    double tot = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) tot += __ldcg(a.part + b);
    tot = warp_sum(tot);
    if (lane == 0) {
      const double g = __ldcg(a.part + gridDim.x);
      const double t = (a.update_mask & HS_UPD_TAU) ? g / (a.scal[1] + 0.5 * tot) : a.scal[0];
      *a.tau_new = t;
      s_tau = t;
      *a.ticket = 0u;  // ready for the next sweep
    }
  }
  if (!a.unit_diag) return;
  __syncthreads();
  const double tn = s_tau;
  for (int jj = tid; jj < a.P; jj += kShrinkThreads)
    a.S[jj] = jj < a.p ? shrink_scale(a.G[(size_t)jj * a.p + jj] + tn * __ldcg(a.lam_new + jj), a.err) : 1.0;
}

// ---------------------------------------------------------------------------
// Cholesky of A~ = S (G + tau Lambda) S and its inverse, FP64
// ---------------------------------------------------------------------------
__global__ void build_kernel(CholArgs a) {
  double* Ad = static_cast<double*>(a.A);
  double* Ld = static_cast<double*>(a.Linv);
  const int64_t n = (int64_t)a.P * a.P;
  const double tau = *a.tau_new;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / a.P), j = (int)(e % a.P);
    double v = 0.0;
    if (j <= i) {
      if (i < a.p) {
        double g = a.G[(size_t)i * a.p + j];
        if (i == j) g += tau * a.lam_new[i];
        v = a.S[i] * g * a.S[j];
      } else {
        v = (i == j) ? 1.0 : 0.0;
      }
    }
    Ad[e] = v;
    Ld[e] = (i == j) ? 1.0 : 0.0;  // right-hand side of L~ X = I
  }
}

// In-shared-memory factorization of one 32 x 32 tile (lower) and the inverse
// of its factor.  256 threads.
__device__ void potrf_trtri_tile(double (*L)[NB + 1], double (*Li)[NB + 1], int* err, bool report) {
  const int tid = threadIdx.x;
  for (int c = 0; c < NB; ++c) {
    if (tid == 0) {
      const double d = L[c][c];
      if (!(d > 0.0) || !isfinite(d)) {
        // The first failing pivot is the cause; later ones follow from it.
        if (report && *(volatile int*)err == 0) set_error(err, isfinite(d) ? kErrNotPD : kErrNonFinite);
        L[c][c] = 1.0;
      } else {
        L[c][c] = sqrt(d);
      }
    }
    __syncthreads();
    if (tid > c && tid < NB) L[tid][c] /= L[c][c];
    __syncthreads();
    // trailing update of the lower triangle (c < s <= r < NB)
    const int m = NB - 1 - c;
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int r = c + 1 + e / m, s = c + 1 + e % m;
      if (s <= r) L[r][s] = fma(-L[r][c], L[s][c], L[r][s]);
    }
    __syncthreads();
  }
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, s = e % NB;
    if (s > r) L[r][s] = 0.0;
  }
  __syncthreads();
  // Inverse: column j = tid solves L x = e_j by forward substitution.
  if (tid < NB) {
    const int j = tid;
    for (int r = 0; r < NB; ++r) {
      double x;
      if (r < j) {
        x = 0.0;
      } else {
        double s = (r == j) ? 1.0 : 0.0;
        for (int m2 = j; m2 < r; ++m2) s = fma(-L[r][m2], Li[m2][j], s);
        x = s / L[r][r];
      }
      Li[r][j] = x;
    }
  }
  __syncthreads();
}

// Tile products C = As Bs over one 32 x 32 x 32 block for the native FP64
// factorization; every thread forms rows {ty, ty+16} x cols {tx, tx+16} of C.
template <int ARITH> struct Work;
template <> struct Work<HS_CHOL_F64> {
  using E = double;
  static __device__ __forceinline__ E from(double x) { return x; }
  static __device__ __forceinline__ void mma(const E (*As)[NB + 1], const E (*Bs)[NB + 1], int ty, int tx,
                                             double out[2][2]) {
    double c00 = 0, c01 = 0, c10 = 0, c11 = 0;
#pragma unroll 8
    for (int q = 0; q < NB; ++q) {
      const double a0 = As[ty][q], a1 = As[ty + 16][q];
      const double b0 = Bs[q][tx], b1 = Bs[q][tx + 16];
      c00 = fma(a0, b0, c00);
      c01 = fma(a0, b1, c01);
      c10 = fma(a1, b0, c10);
      c11 = fma(a1, b1, c11);
    }
    out[0][0] = c00;
    out[0][1] = c01;
    out[1][0] = c10;
    out[1][1] = c11;
  }
};

// Step k, panel part.  Block b < T-k: tile row i = k + b of the factor
// (b = 0: the diagonal tile itself).  Block b >= T-k: inverse tile (k, j),
// j = b - (T-k) < k:  X_kj = L_kk^{-1} B_kj.  Every block factors the 32 x 32
// diagonal tile itself (FP64) rather than waiting for another block.
template <int ARITH>
__global__ void __launch_bounds__(256) panel_kernel(CholArgs a, int k) {
  double* Ad = static_cast<double*>(a.A);
  double* Ld = static_cast<double*>(a.Linv);
  double* LTd = static_cast<double*>(a.LinvT);
  (void)Ad; (void)Ld; (void)LTd;
  using W = Work<ARITH>;
  using E = typename W::E;
  __shared__ double L[NB][NB + 1];
  __shared__ double Li[NB][NB + 1];
  __shared__ E As[NB][NB + 1];
  __shared__ E Bs[NB][NB + 1];
  const int T = a.P / NB;
  const int b = blockIdx.x;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const size_t P = (size_t)a.P;
  const size_t kk = (size_t)k * NB;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, s = e % NB;
    L[r][s] = (s <= r) ? Ad[(kk + r) * P + kk + s] : 0.0;
  }
  __syncthreads();
  potrf_trtri_tile(L, Li, a.err, b == 0);
  if (b == 0) {
    // L_kk itself is not needed after this step (the updates use only the
    // off-diagonal panel), and other blocks of this launch are still reading
    // A_kk, so it is not written back.
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      const int r = e / NB, s = e % NB;
      Ld[(kk + r) * P + kk + s] = Li[r][s];
      LTd[(kk + s) * P + kk + r] = Li[r][s];
    }
    return;
  }
  double out[2][2];
  if (b < T - k) {
    // L_ik = A_ik L_kk^{-T}:  As = A_ik, Bs[q][c] = Li[c][q]
    const size_t ii = (size_t)(k + b) * NB;
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      const int r = e / NB, q = e % NB;
      As[r][q] = W::from(Ad[(ii + r) * P + kk + q]);
      Bs[r][q] = W::from(Li[q][r]);
    }
    __syncthreads();
    W::mma(As, Bs, ty, tx, out);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) Ad[(ii + ty + 16 * i) * P + kk + tx + 16 * j] = out[i][j];
    return;
  }
  // Inverse tile (k, j): X_kj = Li B_kj with B_kj held in Linv(k, j)
  const int j = b - (T - k);
  const size_t jj = (size_t)j * NB;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, q = e % NB;
    As[r][q] = W::from(Li[r][q]);
    Bs[r][q] = W::from(Ld[(kk + r) * P + jj + q]);
  }
  __syncthreads();
  W::mma(As, Bs, ty, tx, out);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int jx = 0; jx < 2; ++jx) {
      const int r = ty + 16 * i, c = tx + 16 * jx;
      Ld[(kk + r) * P + jj + c] = out[i][jx];
      LTd[(jj + c) * P + kk + r] = out[i][jx];
    }
}

// Step k, update part.  Blocks [0, nA): A_ij -= L_ik L_jk^T for k < j <= i.
// Blocks [nA, nA + nB): B_ij -= L_ik X_kj for i > k, j <= k.
template <int ARITH>
__global__ void __launch_bounds__(256) update_kernel(CholArgs a, int k) {
  double* Ad = static_cast<double*>(a.A);
  double* Ld = static_cast<double*>(a.Linv);
  double* LTd = static_cast<double*>(a.LinvT);
  (void)Ad; (void)Ld; (void)LTd;
  using W = Work<ARITH>;
  using E = typename W::E;
  __shared__ E As[NB][NB + 1];
  __shared__ E Bs[NB][NB + 1];
  const int T = a.P / NB;
  const int m = T - k - 1;  // trailing tile rows
  const int nA = m * (m + 1) / 2;
  const int b = blockIdx.x;
  const size_t P = (size_t)a.P;
  const size_t kk = (size_t)k * NB;
  int i, j;
  bool isA;
  if (b < nA) {
    int r = (int)((sqrt(8.0 * b + 1.0) - 1.0) / 2.0);
    while ((r + 1) * (r + 2) / 2 <= b) ++r;
    while (r * (r + 1) / 2 > b) --r;
    i = k + 1 + r;
    j = k + 1 + (b - r * (r + 1) / 2);
    isA = true;
  } else {
    const int c = b - nA;
    i = k + 1 + c / (k + 1);
    j = c % (k + 1);
    isA = false;
  }
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const size_t ii = (size_t)i * NB, jj = (size_t)j * NB;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, q = e % NB;
    As[r][q] = W::from(Ad[(ii + r) * P + kk + q]);  // L_ik
    if (isA)
      Bs[q][r] = W::from(Ad[(jj + r) * P + kk + q]);  // Bs[q][c] = L_jk[c][q]
    else
      Bs[r][q] = W::from(Ld[(kk + r) * P + jj + q]);  // X_kj
  }
  __syncthreads();
  double out[2][2];
  W::mma(As, Bs, ty, tx, out);
  double* dst = isA ? Ad : Ld;
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      const int r = ty + 16 * x, c = tx + 16 * y;
      if (isA && i == j && c > r) continue;  // diagonal tile: lower part only
      dst[(ii + r) * P + jj + c] -= out[x][y];
    }
}

// ---------------------------------------------------------------------------
// FP32-pair factorization, one launch per block column
// ---------------------------------------------------------------------------
// Launch k applies the update from block column k-1 to every trailing tile
// and finishes block column k in the same blocks:
//   A_ij -= L_i,k-1 L_j,k-1^T            tiles k <= j <= i  (stored unless j == k)
//   B_ij -= L_i,k-1 X_k-1,j              tiles i >= k, j < k (stored unless i == k)
//   column k:  D = A_kk (updated), D = L_kk L_kk^T, L_kk^{-1};
//              L_ik = A_ik L_kk^{-T} (i > k);  X_kk = L_kk^{-1};  X_kj = L_kk^{-1} B_kj
// where X = L~^{-1} is formed by block forward substitution on the identity
// (B_ij accumulates -sum_m L_im X_mj and starts at zero).  Every block that
// needs L_kk^{-1} factors the (updated) diagonal tile itself, so one launch
// has no inter-block dependency.  Tiles are read from the scaled Gram matrix
// on first touch (launches 0 and 1), so no separate assembly pass is needed.
using DTile = df2[NB][NB + 1];

struct DFCtx {
  int p, P;
  const double* G;
  const double* S;
  const double* lam;
  double tau;
};

__device__ __forceinline__ df2 scaled_gram(const DFCtx& c, int r, int q) {
  if (r < c.p && q < c.p) {
    double g = c.G[(size_t)r * c.p + q];
    if (r == q) g += c.tau * c.lam[r];
    return df_split(c.S[r] * g * c.S[q]);
  }
  return df2{r == q ? 1.0f : 0.0f, 0.0f};
}

// T[r][c] = tile (ti, tj) of M; transposed: T[c][r].
__device__ __forceinline__ void tile_load(df2 (*T)[NB + 1], const df2* M, int P, int ti, int tj, bool transposed) {
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e >> 5, c = e & 31;
    const df2 v = M[(size_t)(ti * NB + r) * P + tj * NB + c];
    if (transposed)
      T[c][r] = v;
    else
      T[r][c] = v;
  }
}
// Three tile loads in one pass, so their global reads are in flight together.
struct TileSrc {
  const df2* M;
  int ti, tj;
  bool transposed;
  df2 (*dst)[NB + 1];
};
__device__ __forceinline__ void tile_load3(const TileSrc& a, const TileSrc& b, const TileSrc& c, int P) {
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e >> 5, q = e & 31;
    const df2 va = a.M[(size_t)(a.ti * NB + r) * P + a.tj * NB + q];
    const df2 vb = b.M[(size_t)(b.ti * NB + r) * P + b.tj * NB + q];
    const df2 vc = c.M[(size_t)(c.ti * NB + r) * P + c.tj * NB + q];
    if (a.transposed) a.dst[q][r] = va; else a.dst[r][q] = va;
    if (b.transposed) b.dst[q][r] = vb; else b.dst[r][q] = vb;
    if (c.transposed) c.dst[q][r] = vc; else c.dst[r][q] = vc;
  }
}
__device__ __forceinline__ void tile_load_gram(df2 (*T)[NB + 1], const DFCtx& cx, int ti, int tj) {
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e >> 5, c = e & 31;
    const int gr = ti * NB + r, gc = tj * NB + c;
    T[r][c] = (gc <= gr) ? scaled_gram(cx, gr, gc) : scaled_gram(cx, gc, gr);
  }
}
__device__ __forceinline__ void tile_zero(df2 (*T)[NB + 1]) {
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) T[e >> 5][e & 31] = df2{0.0f, 0.0f};
}
__device__ __forceinline__ void tile_store(df2* M, int P, int ti, int tj, const df2 (*T)[NB + 1], bool transposed) {
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e >> 5, c = e & 31;
    M[(size_t)(ti * NB + r) * P + tj * NB + c] = transposed ? T[c][r] : T[r][c];
  }
}

// C = As Bt (set) or C -= As Bt (sub); Bt[q][c].  Rows {ty, ty+16}, cols {tx, tx+16}.
// kLower: only the lower triangle of C is wanted (a symmetric update whose
// upper part nobody reads): the block (ty, tx + 16), strictly upper for every
// thread, is skipped and C keeps its old values there.
// kBRows: the second operand is given by rows, Bs[c][q] (C = As Bs^T), which
// spares a transposition pass (rows tx of a half-warp fall on distinct banks).
template <bool kSub, bool kLower = false, bool kBRows = false>
__device__ __forceinline__ void tile_mma(df2 (*C)[NB + 1], const df2 (*As)[NB + 1], const df2 (*Bt)[NB + 1]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float h[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, l[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 4
  for (int q = 0; q < NB; ++q) {
    const df2 a0 = As[ty][q], a1 = As[ty + 16][q];
    const df2 b0 = kBRows ? Bt[tx][q] : Bt[q][tx], b1 = kBRows ? Bt[tx + 16][q] : Bt[q][tx + 16];
    df_fma(h[0][0], l[0][0], a0, b0);
    if (!kLower) df_fma(h[0][1], l[0][1], a0, b1);
    df_fma(h[1][0], l[1][0], a1, b0);
    df_fma(h[1][1], l[1][1], a1, b1);
  }
  __syncthreads();  // all reads of As/Bt/C done before C is written (C may alias)
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (kLower && i == 0 && j == 1) continue;
      const df2 v = df_renorm(h[i][j], l[i][j]);
      df2& dst = C[ty + 16 * i][tx + 16 * j];
      dst = kSub ? df_sub(dst, v) : v;
    }
  __syncthreads();
}

// Inverse Cholesky factor of a 16 x 16 diagonal block of a tile, at rows
// and columns o..o+15.  Elimination in LDL^T form: at column c the
// multipliers m_rc = W_rc / W_cc (r > c) update the trailing lower triangle,
// W_rq -= m_rc W_qc (c < q <= r), and the same row operations act on U (the
// identity at the start), U_rq -= m_rc U_cq (q <= c < r), so that
// U = L_u^{-1} for W = L_u diag(W_cc) L_u^T; then L^{-1} = diag(W_cc)^{-1/2} U.
// Each update is formed as (W_rc y) / W_cc, so the product overlaps the
// reciprocal of the pivot.  No entry read at step c is written at step c
// (column c of W, row c of U), so one barrier per column suffices; thread
// (r, q) = (tid / 16, tid % 16) owns entry (r, q) of W and U.  U is written at
// the same place of Ui; W is destroyed.  A pivot that is not positive and
// finite is replaced by 1 and reported.  blockDim.x must be 256.
__device__ void potri16_df(df2 (*W)[NB + 1], df2 (*Ui)[NB + 1], int o, df2* s_piv, df2* s_rs, int* err,
                           bool report) {
  const int tid = threadIdx.x, r = tid >> 4, q = tid & 15;
  Ui[o + r][o + q] = df2{r == q ? 1.0f : 0.0f, 0.0f};
  __syncthreads();
  for (int c = 0; c < 16; ++c) {
    df2 d = W[o + c][o + c];
    if (!(d.hi > 0.0f) || !isfinite(d.hi)) d = df2{1.0f, 0.0f};
    const bool trailing = q > c;
    const df2 wr = W[o + r][o + c];
    const df2 y = trailing ? W[o + q][o + c] : Ui[o + c][o + q];
    const df2 x = trailing ? W[o + r][o + q] : Ui[o + r][o + q];
    const df2 dinv = df_recip_fast(d);
    const df2 v = df_sub(x, df_mul(df_mul(wr, y), dinv));  // x - (W_rc y) / W_cc
    if (r > c && q <= r) {
      if (trailing)
        W[o + r][o + q] = v;
      else
        Ui[o + r][o + q] = v;
    }
    __syncthreads();
  }
  // W_cc is not written after step c - 1: the pivots are checked here, the
  // first bad one reported, each replaced by 1 as in the loop
  if (tid == 0 && report) {
    for (int c = 0; c < 16; ++c) {
      const float dh = W[o + c][o + c].hi;
      if (!(dh > 0.0f) || !isfinite(dh)) {
        if (*(volatile int*)err == 0) set_error(err, isfinite(dh) ? kErrNotPD : kErrNonFinite);
        break;
      }
    }
  }
  if (tid < 16) {
    df2 d = W[o + tid][o + tid];
    if (!(d.hi > 0.0f) || !isfinite(d.hi)) d = df2{1.0f, 0.0f};
    s_piv[o + tid] = d;
    df2 sq;
    df_sqrt_rsqrt_fast(d, sq, s_rs[o + tid]);
  }
  __syncthreads();
  const df2 u = Ui[o + r][o + q];
  Ui[o + r][o + q] = q < r ? df_mul(u, s_rs[o + r]) : (q == r ? s_rs[o + r] : df2{0.0f, 0.0f});
  __syncthreads();
}

// One entry of a 16 x 16 product of tile blocks, sum_{q in [q0, q1)} a(q) b(q),
// with four accumulators (q mod 4).  The loop is unrolled over all 16 q with
// the terms outside [q0, q1) multiplied as zeros (which leave a pair sum
// unchanged), so the shared-memory loads of several q are in flight at once
// instead of one trip of a data-dependent loop at a time.
template <typename FA, typename FB>
__device__ __forceinline__ df2 dot16(int q0, int q1, FA fa, FB fb) {
  float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const df2 x = fa(q), y = fb(q);
    const bool in = q >= q0 && q < q1;
    df_fma(h[q & 3], l[q & 3], in ? x : df2{0.0f, 0.0f}, y);
  }
  return df_add(df_add(df_renorm(h[0], l[0]), df_renorm(h[1], l[1])),
                df_add(df_renorm(h[2], l[2]), df_renorm(h[3], l[3])));
}

// Inverse Cholesky factor of a 32 x 32 tile, L^{-1} with D = L L^T, by 2 x 2
// blocks of 16: L11^{-1} of D11; L21 = D21 L11^{-T}; S = D22 - L21 L21^T;
// L22^{-1} of S; (L^{-1})21 = -L22^{-1} (L21 L11^{-1}).  Output: Li = L^{-1}
// (lower, zero above) and LiT its transpose; D (W) is destroyed; LiT serves
// as scratch until the end.  s_rs receives the reciprocal square roots of
// the pivots.  blockDim.x must be 256.
__device__ void potri_df(df2 (*W)[NB + 1], df2 (*Li)[NB + 1], df2 (*LiT)[NB + 1], df2* s_piv, df2* s_rs,
                         int* err, bool report) {
  const int tid = threadIdx.x, r = tid >> 4, c = tid & 15;
  potri16_df(W, Li, 0, s_piv, s_rs, err, report);  // Li11
  // L21[r][c] = sum_{q <= c} D21[r][q] Li11[c][q]       -> LiT[r][c]
  LiT[r][c] = dot16(0, c + 1, [&](int q) { return W[16 + r][q]; }, [&](int q) { return Li[c][q]; });
  __syncthreads();
  // S = D22 - L21 L21^T (lower part), in place in W
  if (c <= r) {
    const df2 t = dot16(0, 16, [&](int q) { return LiT[r][q]; }, [&](int q) { return LiT[c][q]; });
    W[16 + r][16 + c] = df_sub(W[16 + r][16 + c], t);
  }
  // T2 = L21 Li11: T2[r][c] = sum_{q >= c} L21[r][q] Li11[q][c]   -> LiT[16 + r][16 + c]
  LiT[16 + r][16 + c] = dot16(c, 16, [&](int q) { return LiT[r][q]; }, [&](int q) { return Li[q][c]; });
  __syncthreads();
  potri16_df(W, Li, 16, s_piv, s_rs, err, report);  // Li22
  // Li21[r][c] = -sum_{q <= r} Li22[r][q] T2[q][c]; upper block zero
  Li[16 + r][c] = df_neg(dot16(0, r + 1, [&](int q) { return Li[16 + r][16 + q]; },
                               [&](int q) { return LiT[16 + q][16 + c]; }));
  Li[r][16 + c] = df2{0.0f, 0.0f};
  __syncthreads();
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int rr = e >> 5, cc = e & 31;
    LiT[cc][rr] = Li[rr][cc];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) step_df_kernel(CholArgs a, int k) {
  __shared__ DTile sD, sW, sX1, sX2, sLi;
  __shared__ df2 s_piv[NB], s_rs[NB];
  const int T = a.P / NB;
  // Block order: the blocks that finish block column k (they carry the
  // critical path) come first so they are dispatched in the first wave:
  //   [0, T-k)          column tiles (k + b, k)
  //   [T-k, T)          inverse row tiles (k, b - (T-k))
  //   then trailing A tiles (i, j), k < j <= i, and trailing B tiles (i, j), i > k, j < k.
  const int b = blockIdx.x;
  const int m = T - k;
  int i, j;
  bool isA;
  if (b < m) {
    i = k + b;
    j = k;
    isA = true;
  } else if (b < T) {
    i = k;
    j = b - m;
    isA = false;
  } else {
    const int bt = b - T;
    const int mt = m - 1;  // trailing tile rows below the column
    const int nA = mt * (mt + 1) / 2;
    if (bt < nA) {
      int r = (int)((sqrtf(8.0f * bt + 1.0f) - 1.0f) * 0.5f);
      while ((r + 1) * (r + 2) / 2 <= bt) ++r;
      while (r * (r + 1) / 2 > bt) --r;
      i = k + 1 + r;
      j = k + 1 + (bt - r * (r + 1) / 2);
      isA = true;
    } else {
      const int c = bt - nA;
      i = k + 1 + c / k;
      j = c % k;
      isA = false;
    }
  }
  df2* A = reinterpret_cast<df2*>(a.A);
  df2* Linv = reinterpret_cast<df2*>(a.Linv);
  df2* LinvT = reinterpret_cast<df2*>(a.LinvT);
  const DFCtx cx{a.p, a.P, a.G, a.S, a.lam_new, *a.tau_new};
  const bool from_gram = (k <= 1);

  // ---- own tile and its pending update from block column k-1 ----
  if (isA) {
    if (from_gram) {
      tile_load_gram(sW, cx, i, j);
      if (k >= 1) {
        tile_load(sX1, A, a.P, i, k - 1, false);
        tile_load(sX2, A, a.P, j, k - 1, true);
      }
    } else {
      tile_load3(TileSrc{A, i, j, false, sW}, TileSrc{A, i, k - 1, false, sX1}, TileSrc{A, j, k - 1, true, sX2},
                 a.P);
    }
    if (k >= 1) {
      __syncthreads();
      tile_mma<true>(sW, sX1, sX2);
    }
    if (j > k) {
      __syncthreads();
      tile_store(A, a.P, i, j, sW, false);
      return;
    }
  } else {
    if (j == k - 1) {
      tile_zero(sW);
      tile_load(sX1, A, a.P, i, k - 1, false);
      tile_load(sX2, Linv, a.P, k - 1, j, false);
    } else {
      tile_load3(TileSrc{Linv, i, j, false, sW}, TileSrc{A, i, k - 1, false, sX1},
                 TileSrc{Linv, k - 1, j, false, sX2}, a.P);
    }
    __syncthreads();
    tile_mma<true>(sW, sX1, sX2);
    if (i > k) {
      tile_store(Linv, a.P, i, j, sW, false);
      return;
    }
  }
  // ---- the updated diagonal tile, its factor and inverse ----
  if (isA && i == k) {
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) sD[e >> 5][e & 31] = sW[e >> 5][e & 31];
    __syncthreads();
  } else {
    if (from_gram) {
      tile_load_gram(sD, cx, k, k);
      if (k >= 1) {
        tile_load(sX1, A, a.P, k, k - 1, false);
        tile_load(sX2, A, a.P, k, k - 1, true);
      }
    } else {
      tile_load3(TileSrc{A, k, k, false, sD}, TileSrc{A, k, k - 1, false, sX1}, TileSrc{A, k, k - 1, true, sX2},
                 a.P);
    }
    __syncthreads();
    if (k >= 1) tile_mma<true>(sD, sX1, sX2);
  }
  potri_df(sD, sLi, sX1, s_piv, s_rs, a.err, isA && i == k);  // sX1 <- (L_kk^{-1})^T
  if (isA && i == k) {
    tile_store(Linv, a.P, k, k, sLi, false);
    tile_store(LinvT, a.P, k, k, sLi, true);
  } else if (isA) {
    tile_mma<false>(sX2, sW, sX1);  // L_ik = A_ik L_kk^{-T}
    tile_store(A, a.P, i, k, sX2, false);
  } else {
    tile_mma<false>(sX2, sLi, sW);  // X_kj = L_kk^{-1} B_kj
    tile_store(Linv, a.P, k, j, sX2, false);
    tile_store(LinvT, a.P, j, k, sX2, true);
  }
}

// ---------------------------------------------------------------------------
// FP32-pair factorization in ONE persistent launch (tile dataflow)
// ---------------------------------------------------------------------------
// The same tile algebra as step_df_kernel, scheduled by data dependencies
// instead of one launch per block column.  Block 0 runs the diagonal chain:
// for each k it applies the last pending update to A_kk, factors it, forms
// L_kk^{-1}, and computes the next panel tile L_{k+1,k}.  All other blocks
// take the remaining tile tasks in a fixed topological order (round robin):
//   C(i,k)   L_ik = A_ik L_kk^{-T}                  i >= k+2
//   X(k,j)   X_kj = L_kk^{-1} B_kj                   j < k
//   UA(i,j,k) A_ij -= L_ik L_jk^T   k < j <= i, except the diagonal tile's last update
//   UB(i,j,k) B_ij -= L_ik X_kj     i > k, j <= k
// A task list from the host merges each UA(i,k+1,k) into C(i,k) (code j =
// k + 1): the task keeps L_ik in shared memory and applies the next update
// of its own tile row, so every row's path C(i,k) -> UA(i,k+1,k) -> C(i,k+1)
// takes one task per step instead of two.
// Without the inverse factor (CholArgs::inverse == 0) the X and UB tasks are
// left out, so the launch does half the tile products; the chain still forms
// every L_kk^{-1}, and the C tasks and the chain also store L_ik^T at tile
// (k, i) of LinvT, for the block substitutions of the tail.
// Readiness lives in per-tile words tagged with the sweep number e: a flag
// holds e once its tile is published; an update counter holds e*64 + n after
// n updates (values of earlier sweeps are smaller, so nothing is reset).
// Every wait is bounded (2 s) and a global abort word stops all blocks after
// a timeout.  The single-launch schedule is launched cooperatively, and
// one chain's launch then gives the chain to a block on an SM the X-stream
// left free.  An ordinary launch (a grid sharing the GPU with other
// problems' work) needs no residency: the chains go to the first blocks to
// start, and workers take tasks in list order, which respects every
// dependency through the chains, so the earliest unfinished task is always
// held by a running block or not yet taken.
// Word layout of the scheduling buffer (u64, zeroed once when the handle is
// made): header [0] epoch of the last finished launch, [1] exit ticket,
// [2] abort, [3] chain claim (epoch), [4] start ticket, [5] chain SM
// (epoch << 16 | SM id), [6] next worker task, [7] chain ticket of the
// block-column launches; then cntA and cntB (T*T
// each: updates applied to tile (i, j) of A or B, at i*T + j), flagL and
// flagX (T*T: L_ik, X_kj published), flagLi (T: L_kk^{-1} published).
// Flags hold the epoch of the launch that published them; counters hold
// epoch * kEpochStride + updates, so nothing is reset between launches.
constexpr int kSyncHeader = 8;
constexpr unsigned long long kEpochStride = 1024;  // > the largest update count (T <= 256)
constexpr int kMaxTiles = 8192 / NB;

// worker task counts of step k (host and device)
__host__ __device__ __forceinline__ int nC(int T, int k) { return T - k - 2 > 0 ? T - k - 2 : 0; }
__host__ __device__ __forceinline__ int nUA(int T, int k) {
  const int m = T - k - 1;  // tile rows/cols k+1..T-1
  return m > 0 ? m * (m + 1) / 2 - 1 : 0;  // without the diagonal tile (k+1, k+1)
}
__host__ __device__ __forceinline__ int nUB(int T, int k) { return (T - k - 1) * (k + 1); }
// inv: the inverse factor is formed (X and UB tasks); otherwise only C and UA
__host__ __device__ __forceinline__ int nTasks(int T, int k, bool inv) {
  return nC(T, k) + nUA(T, k) + (inv ? k + nUB(T, k) : 0);
}
struct PSync {
  unsigned long long *epoch, *ticket, *abort, *claim, *start, *chain_sm, *next, *chain_ticket;
  unsigned long long *cntA, *cntB, *flagL, *flagX, *flagLi;
  __device__ PSync(unsigned long long* w, int T) {
    epoch = w;
    ticket = w + 1;
    abort = w + 2;
    claim = w + 3;
    start = w + 4;
    chain_sm = w + 5;
    next = w + 6;
    chain_ticket = w + 7;
    cntA = w + kSyncHeader;
    cntB = cntA + T * T;
    flagL = cntB + T * T;
    flagX = flagL + T * T;
    flagLi = flagX + T * T;
  }
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 waits until *p[n] >= target[n] for every n; the block then
// proceeds together.  The words are read together with acquire loads (no
// separate fence: the load that sees the target orders the block's later
// reads, through the barrier; measured: one chain, factorization 0.745 ->
// 0.711 ms against relaxed reads and a trailing fence), so a task whose
// inputs are ready pays one L2 round trip; each poll reads the flag and the
// abort word together.  Returns false (in every thread) if a wait ran out
// (2 s; the timeout bit is set and the abort word raised) or another block
// gave up.
template <int N>
__device__ bool block_wait(const unsigned long long* const (&p)[N], const unsigned long long (&target)[N],
                           const PSync& ps, unsigned long long e, int* err, int site = kSiteChainStep) {
  int ok = 1;
  if (threadIdx.x == 0) {
    unsigned long long v[N];
#pragma unroll
    for (int n = 0; n < N; ++n) v[n] = ld_acquire_u64(p[n]);
#pragma unroll
    for (int n = 0; n < N; ++n) {
      if (ok && v[n] < target[n]) {
        const uint64_t t0 = global_ns();
        for (;;) {
          // the flag and the abort word in one round trip
          const unsigned long long fv = ld_acquire_u64(p[n]);
          const unsigned long long av = ld_relaxed_u64(ps.abort);
          if (fv >= target[n]) break;
          if (av >= e) {
            ok = 0;
            break;
          }
          if (global_ns() - t0 > 2000000000ull) {
            set_timeout(err, site);
            st_release_u64(ps.abort, e);
            ok = 0;
            break;
          }
          __nanosleep(32);
        }
      }
    }
  }
  return __syncthreads_and(ok) != 0;
}
__device__ __forceinline__ bool block_wait(const unsigned long long* p, unsigned long long target, const PSync& ps,
                                           unsigned long long e, int* err, int site = kSiteChainStep) {
  const unsigned long long* const pp[1] = {p};
  const unsigned long long tt[1] = {target};
  return block_wait<1>(pp, tt, ps, e, err, site);
}

// All threads' global writes of the block become visible before *p = v:
// the barrier orders them before thread 0's release store, and a release at
// GPU scope is cumulative over what its thread has synchronized with, so no
// separate (sequentially consistent) fence is needed; readers pair it with
// an acquire (measured: one chain, factorization 0.78 -> 0.75 ms without the
// extra fence on every publish).
__device__ __forceinline__ void block_publish(unsigned long long* p, unsigned long long v) {
  __syncthreads();
  if (threadIdx.x == 0) st_release_u64(p, v);
}

// Tile moves of data other blocks write during this launch go through L2.
// Up to three tiles per call, all global loads issued before the shared
// stores; 16-byte accesses (two FP32 pairs); blockDim.x must be 256.
// Tile traffic of the factorization through L2 with an evict-last policy: the
// working set (a few P x P pair matrices) is small against L2, while the
// X-stream beside it streams X through L2 with an evict-first policy.
__device__ __forceinline__ uint64_t l2_keep_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float4 ld_keep(const float4* a, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.cg.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(a), "l"(pol)
               : "memory");
  return v;
}
__device__ __forceinline__ void st_keep(float4* a, float4 v, uint64_t pol) {
  asm volatile("st.global.cg.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st_keep2(float2* a, float2 v, uint64_t pol) {
  asm volatile("st.global.cg.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(a), "f"(v.x), "f"(v.y), "l"(pol)
               : "memory");
}

struct TileRef {
  const df2* M;
  int ti, tj;
  bool transposed;
  df2 (*dst)[NB + 1];
};
template <int NT>
__device__ __forceinline__ void tiles_load_cg(const TileRef (&t)[NT], int P) {
  const uint64_t pol = l2_keep_policy();
  float4 v[NT][2];
#pragma unroll
  for (int n = 0; n < NT; ++n)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = threadIdx.x + h * 256, r = e >> 4, c = (e & 15) * 2;
      v[n][h] = ld_keep(reinterpret_cast<const float4*>(t[n].M + (size_t)(t[n].ti * NB + r) * P + t[n].tj * NB + c),
                        pol);
    }
#pragma unroll
  for (int n = 0; n < NT; ++n)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = threadIdx.x + h * 256, r = e >> 4, c = (e & 15) * 2;
      const df2 x0{v[n][h].x, v[n][h].y}, x1{v[n][h].z, v[n][h].w};
      if (t[n].transposed) {
        t[n].dst[c][r] = x0;
        t[n].dst[c + 1][r] = x1;
      } else {
        t[n].dst[r][c] = x0;
        t[n].dst[r][c + 1] = x1;
      }
    }
}
__device__ __forceinline__ void tile_store_cg(df2* M, int P, int ti, int tj, const df2 (*T)[NB + 1], bool transposed) {
  const uint64_t pol = l2_keep_policy();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int e = threadIdx.x + h * 256, r = e >> 4, c = (e & 15) * 2;
    const df2 x0 = transposed ? T[c][r] : T[r][c];
    const df2 x1 = transposed ? T[c + 1][r] : T[r][c + 1];
    st_keep(reinterpret_cast<float4*>(M + (size_t)(ti * NB + r) * P + tj * NB + c),
            make_float4(x0.hi, x0.lo, x1.hi, x1.lo), pol);
  }
}

// ---- tile work of a 128-thread group ----------------------------------------
// rows of tile row i inside the p x p matrix (the rest is padding)
__device__ __forceinline__ int tile_rows(int p, int i) {
  const int r = p - i * NB;
  return r < NB ? r : NB;
}
// A worker block runs two independent tile tasks at a time, one per group of
// four warps (warps 0-3 and 4-7), each with its own tiles and named barrier.
struct Grp {
  int t;    // thread index within the group, 0..127
  int bar;  // named barrier of the group (1 or 2)
  __device__ __forceinline__ void sync() const { named_bar_sync(bar, 128); }
  __device__ __forceinline__ bool sync_and(int pred) const {
    int out;
    asm volatile(
        "{\n\t.reg .pred q, r;\n\tsetp.ne.s32 q, %1, 0;\n\tbar.red.and.pred r, %2, 128, q;\n\tselp.s32 %0, 1, 0, r;\n\t}"
        : "=r"(out)
        : "r"(pred), "r"(bar)
        : "memory");
    return out != 0;
  }
};

template <int NT>
__device__ __forceinline__ void gload_cg(const Grp& g, const TileRef (&t)[NT], int P) {
  const uint64_t pol = l2_keep_policy();
  float4 v[NT][4];
#pragma unroll
  for (int n = 0; n < NT; ++n)
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int e = g.t + h * 128, r = e >> 4, c = (e & 15) * 2;
      v[n][h] = ld_keep(reinterpret_cast<const float4*>(t[n].M + (size_t)(t[n].ti * NB + r) * P + t[n].tj * NB + c),
                        pol);
    }
#pragma unroll
  for (int n = 0; n < NT; ++n)
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int e = g.t + h * 128, r = e >> 4, c = (e & 15) * 2;
      const df2 x0{v[n][h].x, v[n][h].y}, x1{v[n][h].z, v[n][h].w};
      if (t[n].transposed) {
        t[n].dst[c][r] = x0;
        t[n].dst[c + 1][r] = x1;
      } else {
        t[n].dst[r][c] = x0;
        t[n].dst[r][c + 1] = x1;
      }
    }
}
__device__ __forceinline__ void gload_gram(const Grp& g, df2 (*T)[NB + 1], const DFCtx& cx, int ti, int tj) {
  for (int e = g.t; e < NB * NB; e += 128) {
    const int r = e >> 5, c = e & 31;
    const int gr = ti * NB + r, gc = tj * NB + c;
    T[r][c] = (gc <= gr) ? scaled_gram(cx, gr, gc) : scaled_gram(cx, gc, gr);
  }
}
__device__ __forceinline__ void gzero(const Grp& g, df2 (*T)[NB + 1]) {
  for (int e = g.t; e < NB * NB; e += 128) T[e >> 5][e & 31] = df2{0.0f, 0.0f};
}
__device__ __forceinline__ void gstore_cg(const Grp& g, df2* M, int P, int ti, int tj, const df2 (*T)[NB + 1],
                                          bool transposed) {
  const uint64_t pol = l2_keep_policy();
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const int e = g.t + h * 128, r = e >> 4, c = (e & 15) * 2;
    const df2 x0 = transposed ? T[c][r] : T[r][c];
    const df2 x1 = transposed ? T[c + 1][r] : T[r][c + 1];
    st_keep(reinterpret_cast<float4*>(M + (size_t)(ti * NB + r) * P + tj * NB + c),
            make_float4(x0.hi, x0.lo, x1.hi, x1.lo), pol);
  }
}
// C = As Bt (set) or C -= As Bt (sub), Bt[q][c]; thread: rows ty + 8i, columns tx, tx + 16.
// Rows r >= rows of As are padding past p, zero in every operand the tasks
// pass here, so their products are zero and are skipped (C keeps those rows,
// or gets zeros when set).
template <bool kSub>
__device__ __forceinline__ void gmma(const Grp& g, df2 (*C)[NB + 1], const df2 (*As)[NB + 1], const df2 (*Bt)[NB + 1],
                                     int rows = NB) {
  const int tx = g.t & 15, ty = g.t >> 4;
  const int ni = rows > ty ? (rows - ty + 7) >> 3 : 0;  // this thread's rows ty + 8i below rows
  float h[4][2], l[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) h[i][j] = l[i][j] = 0.0f;
  if (ni >= 4) {
#pragma unroll 2
    for (int q = 0; q < NB; ++q) {
      df2 av[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[ty + 8 * i][q];
      const df2 b0 = Bt[q][tx], b1 = Bt[q][tx + 16];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        df_fma(h[i][0], l[i][0], av[i], b0);
        df_fma(h[i][1], l[i][1], av[i], b1);
      }
    }
  } else {
    for (int q = 0; q < NB; ++q) {
      const df2 b0 = Bt[q][tx], b1 = Bt[q][tx + 16];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (i < ni) {
          const df2 av = As[ty + 8 * i][q];
          df_fma(h[i][0], l[i][0], av, b0);
          df_fma(h[i][1], l[i][1], av, b1);
        }
    }
  }
  // C is neither As nor Bt, and each thread reads and writes only its own
  // entries of C, so no barrier is needed before the writes
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const df2 v = df_renorm(h[i][j], l[i][j]);
      df2& dst = C[ty + 8 * i][tx + 16 * j];
      dst = kSub ? df_sub(dst, v) : v;
    }
  g.sync();
}
// The trailing update A_ij -= L_ik L_jk^T of a UA task, with both factor
// tiles as loaded (not transposed: Ls[c][q] is read along a row, which with
// the 33-pair row stride touches 16 distinct bank pairs per half-warp) and
// the result stored from registers straight to tile (ti, tj) of M: no
// barrier between the products and the store, and W (the tile's old value,
// read only by its owner thread) is never written in shared memory.
// Thread: rows ty + 8i, columns tx, tx + 16; rows >= rows are padding.
__device__ __forceinline__ void gmma_update_store(const Grp& g, const df2 (*W)[NB + 1], const df2 (*As)[NB + 1],
                                                  const df2 (*Bs)[NB + 1], int rows, df2* M, int P, int ti, int tj) {
  const uint64_t pol = l2_keep_policy();
  const int tx = g.t & 15, ty = g.t >> 4;
  const int ni = rows > ty ? (rows - ty + 7) >> 3 : 0;
  float h[4][2], l[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) h[i][j] = l[i][j] = 0.0f;
  if (ni >= 4) {
#pragma unroll 2
    for (int q = 0; q < NB; ++q) {
      df2 av[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[ty + 8 * i][q];
      const df2 b0 = Bs[tx][q], b1 = Bs[tx + 16][q];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        df_fma(h[i][0], l[i][0], av[i], b0);
        df_fma(h[i][1], l[i][1], av[i], b1);
      }
    }
  } else {
    for (int q = 0; q < NB; ++q) {
      const df2 b0 = Bs[tx][q], b1 = Bs[tx + 16][q];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (i < ni) {
          const df2 av = As[ty + 8 * i][q];
          df_fma(h[i][0], l[i][0], av, b0);
          df_fma(h[i][1], l[i][1], av, b1);
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int r = ty + 8 * i, c = tx + 16 * j;
      const df2 v = df_sub(W[r][c], df_renorm(h[i][j], l[i][j]));
      st_keep2(reinterpret_cast<float2*>(M + (size_t)(ti * NB + r) * P + tj * NB + c), make_float2(v.hi, v.lo),
               pol);
    }
}
// Thread 0 of the group waits for every *p[n] >= target[n] (acquire loads of
// all at once, then polls); bounded as block_wait.
template <int N>
__device__ bool gwait(const Grp& g, const unsigned long long* const (&p)[N], const unsigned long long (&target)[N],
                      const PSync& ps, unsigned long long e, int* err) {
  int ok = 1;
  if (g.t == 0) {
    unsigned long long v[N];
#pragma unroll
    for (int n = 0; n < N; ++n) v[n] = ld_acquire_u64(p[n]);
#pragma unroll
    for (int n = 0; n < N; ++n) {
      if (ok && v[n] < target[n]) {
        const uint64_t t0 = global_ns();
        for (;;) {
          const unsigned long long fv = ld_acquire_u64(p[n]);
          const unsigned long long av = ld_relaxed_u64(ps.abort);
          if (fv >= target[n]) break;
          if (av >= e) {
            ok = 0;
            break;
          }
          if (global_ns() - t0 > 2000000000ull) {
            set_timeout(err, kSiteTask);
            st_release_u64(ps.abort, e);
            ok = 0;
            break;
          }
          __nanosleep(32);
        }
      }
    }
  }
  return g.sync_and(ok);
}
// The group's writes become visible before *p = v (as block_publish).
__device__ __forceinline__ void gpublish(const Grp& g, unsigned long long* p, unsigned long long v) {
  g.sync();
  if (g.t == 0) st_release_u64(p, v);
}

// The buffers of one chain of the launch.
struct ChainView {
  df2 *A, *Linv, *LinvT;
  uint16_t* dig;  // this chain's six digit planes, or nullptr
  DFCtx cx;
  PSync ps;
  __device__ ChainView(const CholArgs& a, int m, int T)
      : A(reinterpret_cast<df2*>(a.A) + (size_t)m * a.P * a.P),
        Linv(reinterpret_cast<df2*>(a.Linv) + (size_t)m * a.P * a.P),
        LinvT(reinterpret_cast<df2*>(a.LinvT) + (size_t)m * a.P * a.P),
        dig(a.digits ? static_cast<uint16_t*>(a.digits) + (size_t)m * 6 * a.P * a.P : nullptr),
        cx{a.p, a.P, a.G, a.S + (size_t)m * a.P, a.lam_new + (size_t)m * a.p, a.tau_new[m]},
        ps(a.sync + (size_t)m * a.sync_words, T) {}
};

// The six BF16 digit planes of factor tile (ti, tk), from a tile in shared
// memory; threads t0, t0 + nthr, ... of the caller (read by chol_trail_kernel).
__device__ __forceinline__ void tile_digits_store(int t0, int nthr, const df2 (*Tl)[NB + 1], uint16_t* dig, int P,
                                                  int ti, int tk) {
  const size_t plane = (size_t)P * P;
  for (int e = t0; e < NB * NB; e += nthr) {
    const int r = e >> 5, c = e & 31;
    uint16_t d[6];
    df_digits6(Tl[r][c], d);
    uint16_t* dst = dig + (size_t)(ti * NB + r) * P + tk * NB + c;
#pragma unroll
    for (int t = 0; t < 6; ++t) dst[t * plane] = d[t];
  }
}

constexpr int kPersistTiles = 6;  // chain: 5 tiles; workers: 3 per group
constexpr size_t kPersistSmem = kPersistTiles * sizeof(DTile);

__global__ void __launch_bounds__(256, 4) chol_persistent_kernel(CholArgs a) {
  extern __shared__ __align__(16) unsigned char dyn_tiles[];
  DTile* const tiles = reinterpret_cast<DTile*>(dyn_tiles);
  DTile& sD = tiles[0];
  DTile& sW = tiles[1];
  DTile& sX1 = tiles[2];
  DTile& sX2 = tiles[3];
  DTile& sLi = tiles[4];
  __shared__ df2 s_piv[NB], s_rs[NB];
  __shared__ int s_step0[kMaxTiles + 1];
  __shared__ unsigned long long s_e;
  __shared__ int s_role;  // 0 worker, 1 chain, 2 idle
  __shared__ int s_chain;
  __shared__ int s_task[2];
  const int T = a.P / NB;
  const int P = a.P;
  const int nch = a.nchains > 1 ? a.nchains : 1;
  const bool inv = a.inverse != 0;
  // tile columns of this launch: all, or one block column whose trailing
  // updates the tensor cores apply between launches
  const int kb = a.k1 > 0 ? a.k0 : 0, ke = a.k1 > 0 ? a.k1 : T;
  const PSync ps0(a.sync, T);  // chain 0's words also hold the launch-wide header
  unsigned int smid;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  if (threadIdx.x == 0) {
    // (kernel-ordered after the previous launch's update); the block-column
    // launches of one factorization share the epoch of its first launch
    const unsigned long long e0 = *ps0.epoch + (kb == 0 ? 1ull : 0ull);
    s_e = e0;
    int role = 0, chain = 0;
    if (nch == 1 && a.k1 == 0 && a.cooperative) {
      // The chain goes to a block on an SM the X-stream left free (no mark
      // of this sweep), else to the last block to start (every block starts:
      // the launch is cooperative).
      const unsigned int stamp = (unsigned int)(*a.k_dev + 1);
      const bool free_sm = a.sm_mark && smid < (unsigned)kSmMarks && __ldcg(a.sm_mark + smid) != stamp;
      if (free_sm && atomicCAS(ps0.claim, e0 - 1, e0) == e0 - 1) role = 1;
      const unsigned long long st = atomicAdd(ps0.start, 1ull);
      if (st == gridDim.x - 1) {
        *ps0.start = 0;  // every block has taken its ticket
        if (role == 0 && atomicCAS(ps0.claim, e0 - 1, e0) == e0 - 1) role = 1;
      }
      if (role == 1) st_release_u64(ps0.chain_sm, (e0 << 16) | smid);
    } else if (a.k1 > 0 && a.sm_role && smid < (unsigned)kSmMarks) {
      // Block-column launches: the first block to start on each SM may walk a
      // chain (the first nch of them do), and the other blocks on a chain's SM
      // stay idle, leaving the latency-bound chain the whole SM.  The tag is
      // unique and increasing per launch, so the per-SM words need no reset.
      const unsigned long long tag = (e0 << 8) | (unsigned long long)(kb + 1);  // kb < 256
      unsigned long long* const claim = a.sm_role + smid;
      unsigned long long* const rword = a.sm_role + kSmMarks + smid;
      if (atomicMax(claim, tag) < tag) {
        const unsigned long long t = atomicAdd(ps0.chain_ticket, 1ull);
        if (t < (unsigned long long)nch) {
          role = 1;
          chain = (int)t;
        }
        st_release_u64(rword, 2 * tag + (role == 1 ? 1ull : 0ull));
      } else {
        unsigned long long v = ld_acquire_u64(rword);
        const uint64_t t0 = global_ns();
        while (v < 2 * tag) {
          if (global_ns() - t0 > 2000000000ull) {
            set_timeout(a.err, kSiteStartRole);
            st_release_u64(ps0.abort, e0);
            break;
          }
          __nanosleep(32);
          v = ld_acquire_u64(rword);
        }
        role = (v < 2 * tag || (v & 1ull)) ? 2 : 0;
      }
    } else {
      // several chains, or an ordinary launch: the first nch blocks to start
      // walk the diagonal chains (a block that has started holds its role, so
      // the chains run whether or not the rest of the grid is resident)
      const unsigned long long st = atomicAdd(ps0.start, 1ull);
      if (st == gridDim.x - 1) *ps0.start = 0;
      if (st < (unsigned long long)nch) {
        role = 1;
        chain = (int)st;
      }
    }
    s_role = role;
    s_chain = chain;
  }
  __syncthreads();
  const unsigned long long e = s_e;
  const unsigned long long base = e * kEpochStride;
  if (nch == 1 && a.k1 == 0 && a.cooperative && s_role == 0 && gridDim.x >= 16) {
    // Blocks that share the chain's SM stay idle, leaving it the whole SM
    // (at most 3 of them: 4 blocks fit on an SM).
    if (block_wait(ps0.chain_sm, e << 16, ps0, e, a.err, kSiteStartRole)) {
      if (threadIdx.x == 0 && (unsigned)(ld_acquire_u64(ps0.chain_sm) & 0xFFFFu) == smid) s_role = 2;
    } else if (threadIdx.x == 0) {
      s_role = 2;
    }
    __syncthreads();
  }

  if (s_role == 1) {
    // ---------------- the diagonal chain ----------------
    const ChainView cv(a, s_chain, T);
    df2* const A = cv.A;
    df2* const Linv = cv.Linv;
    df2* const LinvT = cv.LinvT;
    const DFCtx& cx = cv.cx;
    const PSync& ps = cv.ps;
    // Entering step k, sD holds D_k = A_kk after all k updates.
    bool go = true;
    if (kb == 0 && !a.prebuilt) {
      tile_load_gram(sD, cx, 0, 0);
    } else if (kb == 0) {
      const TileRef t[1] = {{A, 0, 0, false, sD}};
      tiles_load_cg<1>(t, P);
    } else {
      // the first diagonal tile of a later block column, after the tensor-core updates
      go = block_wait(&ps.cntA[kb * T + kb], base + (unsigned long long)kb, ps0, e, a.err, kSiteChainStart);
      if (go) {
        const TileRef t[1] = {{A, kb, kb, false, sD}};
        tiles_load_cg<1>(t, P);
      }
    }
    __syncthreads();
    for (int k = kb; k < ke && go; ++k) {
      potri_df(sD, sLi, sX1, s_piv, s_rs, a.err, true);  // sLi <- L_kk^{-1}, sX1 <- its transpose
      tile_store_cg(Linv, P, k, k, sLi, false);
      tile_store_cg(LinvT, P, k, k, sLi, true);
      block_publish(&ps.flagLi[k], e);
      if (k + 1 == T) break;
      // the next tile row starts the next block column: its diagonal tile
      // takes this block column's updates on the tensor cores
      const bool last = (k + 1 == ke);
      // A_{k+1,k} and A_{k+1,k+1} after updates 0..k-1 (workers)
      if (k >= 1) {
        const unsigned long long* const wp2[2] = {&ps.cntA[(k + 1) * T + k], &ps.cntA[(k + 1) * T + k + 1]};
        const unsigned long long wt2[2] = {base + (unsigned long long)k, last ? 0ull : base + (unsigned long long)k};
        if (!block_wait<2>(wp2, wt2, ps0, e, a.err)) break;
        if (last) {
          const TileRef t[1] = {{A, k + 1, k, false, sW}};
          tiles_load_cg<1>(t, P);
        } else {
          const TileRef t[2] = {{A, k + 1, k, false, sW}, {A, k + 1, k + 1, false, sD}};
          tiles_load_cg<2>(t, P);
        }
      } else if (!a.prebuilt) {
        tile_load_gram(sW, cx, 1, 0);
        if (!last) tile_load_gram(sD, cx, 1, 1);
      } else if (last) {
        const TileRef t[1] = {{A, 1, 0, false, sW}};
        tiles_load_cg<1>(t, P);
      } else {
        const TileRef t[2] = {{A, 1, 0, false, sW}, {A, 1, 1, false, sD}};
        tiles_load_cg<2>(t, P);
      }
      __syncthreads();
      tile_mma<false>(sLi, sW, sX1);  // L_{k+1,k} = A_{k+1,k} L_kk^{-T}
      tile_store_cg(A, P, k + 1, k, sLi, false);
      if (!inv) tile_store_cg(LinvT, P, k, k + 1, sLi, true);
      if (last && cv.dig) tile_digits_store(threadIdx.x, blockDim.x, sLi, cv.dig, P, k + 1, k);
      block_publish(&ps.flagL[(k + 1) * T + k], e);
      if (last) break;
      tile_mma<true, true, true>(sD, sLi, sLi);  // D_{k+1} = A_{k+1,k+1} - L_{k+1,k} L_{k+1,k}^T (lower part)
    }
  } else if (s_role == 0) {
    // ---------------- workers: tasks in list order from a shared counter ----------------
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int kk = 0; kk <= T; ++kk) {
        s_step0[kk] = acc;
        if (kk < T) acc += nTasks(T, kk, inv);
      }
    }
    __syncthreads();
    // a block-column launch runs exactly its list (which may be empty: a
    // last block column of one tile has no worker task)
    const int total1 = a.order ? a.ntasks : s_step0[T];
    const long long total = (long long)total1 * nch;  // task t: chain t % nch, its list entry t / nch
    const int gi = threadIdx.x >> 7;                  // two groups of four warps, one task each
    const Grp g{(int)(threadIdx.x & 127), 1 + gi};
    DTile& gW = tiles[3 * gi];
    DTile& gX1 = tiles[3 * gi + 1];
    DTile& gX2 = tiles[3 * gi + 2];
    unsigned long long grabbed = 0;
    if (g.t == 0) grabbed = atomicAdd(ps0.next, 1ull);
    for (;;) {
      if (g.t == 0) s_task[gi] = grabbed >= (unsigned long long)total ? -1 : (int)grabbed;
      g.sync();
      const int t = s_task[gi];
      if (t < 0) break;
      if (g.t == 0) grabbed = atomicAdd(ps0.next, 1ull);  // the following task, early
      const ChainView cv(a, t % nch, T);
      df2* const A = cv.A;
      df2* const Linv = cv.Linv;
      df2* const LinvT = cv.LinvT;
      const DFCtx& cx = cv.cx;
      const PSync& ps = cv.ps;
      const int tl = t / nch;
      int kind, i, j, k;
      if (a.order) {
        // list entry, decoded on the host: kind | k << 2 | i << 10 | j << 18
        const int code = __ldg(a.order + tl);
        kind = code & 3;
        k = (code >> 2) & 0xFF;
        i = (code >> 10) & 0xFF;
        j = (code >> 18) & 0xFF;
      } else {
        // canonical order: step k's C, X, UA, UB tasks from s_step0[k]
        int lo = 0, hi = T - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_step0[mid] <= tl) lo = mid; else hi = mid - 1;
        }
        k = lo;
        int u = tl - s_step0[k];
        const int c = nC(T, k), ua = nUA(T, k);
        if (u < c) {
          kind = 0;
          i = k + 2 + u;
          j = k;
        } else if (inv && u - c < k) {
          kind = 1;
          i = k;
          j = u - c;
        } else {
          u -= c + (inv ? k : 0);
          if (u < ua) {
            // the lower triangle of tile rows/cols k+1..T-1, column by column
            // (column k+1, which feeds the diagonal chain, first), without (k+1, k+1)
            const int m = T - k - 1;
            int idx = u + 1, q = 0;
            while (idx >= m - q) {
              idx -= m - q;
              ++q;
            }
            kind = 2;
            j = k + 1 + q;
            i = j + idx;
          } else {
            u -= ua;
            kind = 3;
            i = k + 1 + u / (k + 1);
            j = u % (k + 1);
          }
        }
      }
      const unsigned long long done_k = base + (unsigned long long)k;  // A tile after updates 0..k-1
      if (kind == 0) {
        // C(i,k): L_ik = A_ik L_kk^{-T}
        const unsigned long long* const wp2[2] = {&ps.flagLi[k], &ps.cntA[i * T + k]};
        const unsigned long long wt2[2] = {e, k >= 1 ? done_k : 0ull};
        if (!gwait<2>(g, wp2, wt2, ps0, e, a.err)) break;
        if (k == 0 && !a.prebuilt) {
          gload_gram(g, gW, cx, i, 0);
          const TileRef t1[1] = {{LinvT, k, k, false, gX1}};
          gload_cg<1>(g, t1, P);
        } else {
          const TileRef t2[2] = {{A, i, k, false, gW}, {LinvT, k, k, false, gX1}};  // gX1[q][c] = (L_kk^{-1})[c][q]
          gload_cg<2>(g, t2, P);
        }
        g.sync();
        gmma<false>(g, gX2, gW, gX1, tile_rows(cx.p, i));
        gstore_cg(g, A, P, i, k, gX2, false);
        if (!inv) gstore_cg(g, LinvT, P, k, i, gX2, true);
        if (cv.dig && i >= ke) tile_digits_store(g.t, 128, gX2, cv.dig, P, i, k);
        gpublish(g, &ps.flagL[i * T + k], e);
        if (j != k + 1) continue;
        // the merged UA(i,k+1,k): A_{i,k+1} -= L_ik L_{k+1,k}^T with L_ik still in gX2
        // (the chain publishes L_{k+1,k}; tile (i, k+1) after updates 0..k-1)
        const unsigned long long* const wq2[2] = {&ps.flagL[(k + 1) * T + k], &ps.cntA[i * T + k + 1]};
        const unsigned long long wu2[2] = {e, k >= 1 ? done_k : 0ull};
        if (!gwait<2>(g, wq2, wu2, ps0, e, a.err)) break;
        if (k == 0 && !a.prebuilt) {
          gload_gram(g, gW, cx, i, k + 1);
          const TileRef t1[1] = {{A, k + 1, k, false, gX1}};
          gload_cg<1>(g, t1, P);
        } else {
          const TileRef t2[2] = {{A, i, k + 1, false, gW}, {A, k + 1, k, false, gX1}};
          gload_cg<2>(g, t2, P);
        }
        g.sync();
        gmma_update_store(g, gW, gX2, gX1, tile_rows(cx.p, i), A, P, i, k + 1);
        gpublish(g, &ps.cntA[i * T + k + 1], done_k + 1);
        continue;
      }
      if (kind == 1) {
        // X(k,j): X_kj = L_kk^{-1} B_kj; B_kj after its k - j updates
        const unsigned long long* const wp2[2] = {&ps.flagLi[k], &ps.cntB[k * T + j]};
        const unsigned long long wt2[2] = {e, base + (unsigned long long)(k - j)};
        if (!gwait<2>(g, wp2, wt2, ps0, e, a.err)) break;
        const TileRef t2[2] = {{Linv, k, k, false, gX1}, {Linv, k, j, false, gW}};
        gload_cg<2>(g, t2, P);
        g.sync();
        gmma<false>(g, gX2, gX1, gW, tile_rows(cx.p, k));
        gstore_cg(g, Linv, P, k, j, gX2, false);
        gstore_cg(g, LinvT, P, j, k, gX2, true);
        gpublish(g, &ps.flagX[k * T + j], e);
        continue;
      }
      if (kind == 2) {
        // UA(i,j,k): A_ij -= L_ik L_jk^T
        const unsigned long long* const wp3[3] = {&ps.flagL[i * T + k], &ps.flagL[j * T + k], &ps.cntA[i * T + j]};
        const unsigned long long wt3[3] = {e, e, k >= 1 ? done_k : 0ull};
        if (!gwait<3>(g, wp3, wt3, ps0, e, a.err)) break;
        if (k == 0 && !a.prebuilt) {
          gload_gram(g, gW, cx, i, j);
          const TileRef t2[2] = {{A, i, k, false, gX1}, {A, j, k, false, gX2}};
          gload_cg<2>(g, t2, P);
        } else {
          const TileRef t3[3] = {{A, i, j, false, gW}, {A, i, k, false, gX1}, {A, j, k, false, gX2}};
          gload_cg<3>(g, t3, P);
        }
        g.sync();
        gmma_update_store(g, gW, gX1, gX2, tile_rows(cx.p, i), A, P, i, j);
        gpublish(g, &ps.cntA[i * T + j], done_k + 1);
        continue;
      }
      {
        // UB(i,j,k): B_ij -= L_ik X_kj (X_kk = L_kk^{-1}; B_ik starts at zero)
        const unsigned long long* const wp3[3] = {&ps.flagL[i * T + k], j < k ? &ps.flagX[k * T + j] : &ps.flagLi[k],
                                                   &ps.cntB[i * T + j]};
        const unsigned long long wt3[3] = {e, e, k > j ? base + (unsigned long long)(k - j) : 0ull};
        if (!gwait<3>(g, wp3, wt3, ps0, e, a.err)) break;
        if (k == j) {
          gzero(g, gW);
          const TileRef t2[2] = {{A, i, k, false, gX1}, {Linv, k, j, false, gX2}};
          gload_cg<2>(g, t2, P);
        } else {
          const TileRef t3[3] = {{Linv, i, j, false, gW}, {A, i, k, false, gX1}, {Linv, k, j, false, gX2}};
          gload_cg<3>(g, t3, P);
        }
        g.sync();
        gmma<true>(g, gW, gX1, gX2, tile_rows(cx.p, i));
        gstore_cg(g, Linv, P, i, j, gW, false);
        gpublish(g, &ps.cntB[i * T + j], base + (unsigned long long)(k - j + 1));
      }
    }
  }
  // the last block out records the epoch for the next launch
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ps0.ticket, 1ull) == (unsigned long long)(gridDim.x - 1)) {
      *ps0.ticket = 0;
      *ps0.next = 0;
      *ps0.chain_ticket = 0;
      *ps0.epoch = e;
    }
  }
}

// ---------------------------------------------------------------------------
// tail
// ---------------------------------------------------------------------------
__device__ __forceinline__ double elem(const double* M, size_t idx) { return M[idx]; }

// Several chains in one launch (blockIdx.y = chain), as for the shrink kernel;
// k_dev_rw advances by one slot per chain.
__device__ __forceinline__ TailArgs tail_chain(TailArgs a, int m) {
  const size_t p = (size_t)a.p, P = (size_t)a.P, P2 = P * P;
  const size_t eb = a.df32 ? sizeof(df2) : sizeof(double);
  a.rng.chain += (uint32_t)m;
  a.xtz += m * p;
  a.S += m * P;
  a.Linv = static_cast<const unsigned char*>(a.Linv) + m * P2 * eb;
  a.LinvT = static_cast<const unsigned char*>(a.LinvT) + m * P2 * eb;
  if (a.L) a.L = static_cast<const unsigned char*>(a.L) + m * P2 * eb;
  a.v += m * P;
  a.beta_new += m * p;
  a.nu_new += m * p;
  a.lam_new += m * p;
  a.tau_new += m;
  a.beta += m * p;
  a.lam += m * p;
  a.nu += m * p;
  a.scal += 2 * m;
  a.k_dev_rw += m;
  a.beta_c = static_cast<unsigned char*>(a.beta_c) + (size_t)m * a.ld * (a.beta_c_is_double ? 8 : 4);
  a.ring_beta += m * (size_t)a.ring_size * p;
  a.ring_lam += m * (size_t)a.ring_size * p;
  a.ring_tau += m * (size_t)a.ring_size;
  return a;
}

// v_i = sum_{j <= i} Linv[i][j] S_j xtz_j + s_i   (one warp per row)
template <typename E>
__global__ void __launch_bounds__(256) tail_w_kernel(TailArgs a0) {
  const TailArgs a = tail_chain(a0, blockIdx.y);
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= a.p) return;
  const int i = warp;
  const E* row = reinterpret_cast<const E*>(a.Linv) + (size_t)i * a.P;
  double s = 0.0;
  for (int j = lane; j <= i; j += 32) s = fma(elem(row, j), a.S[j] * a.xtz[j], s);
  s = warp_sum(s);
  if (lane == 0) {
    const uint32_t sweep = (uint32_t)(*a.k_dev + 1);
    const Rng rng{a.rng.k0, a.rng.k1, a.rng.chain, a.rng.problem};
    const uint4 w = rng.words((uint32_t)i, sweep, kPurBeta);
    double u, uc;
    unit_pair(w.x, w.y, u, uc);
    a.v[i] = s + std_normal_from_unit(u, uc);
  }
}

// beta_j = S_j sum_{i >= j} LinvT[j][i] v_i; nu_j^{-1} (one warp per j)
template <typename E>
__global__ void __launch_bounds__(256) tail_beta_kernel(TailArgs a0) {
  const TailArgs a = tail_chain(a0, blockIdx.y);
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= a.p) return;
  const int j = warp;
  const E* row = reinterpret_cast<const E*>(a.LinvT) + (size_t)j * a.P;
  double s = 0.0;
  for (int i = j + lane; i < a.p; i += 32) s = fma(elem(row, i), a.v[i], s);
  s = warp_sum(s);
  if (lane == 0) {
    const double bj = a.S[j] * s;
    a.beta_new[j] = bj;
    // Only a first error is recorded here: after an indefinite or non-finite
    // precision matrix beta is garbage by construction.
    if (!isfinite(bj) && *(volatile int*)a.err == 0) set_error(a.err, kErrNonFinite);
    const uint32_t sweep = (uint32_t)(*a.k_dev + 1);
    const Rng rng{a.rng.k0, a.rng.k1, a.rng.chain, a.rng.problem};
    const uint4 w = rng.words((uint32_t)j, sweep, kPurNu);
    double u, uc;
    unit_pair(w.x, w.y, u, uc);
    a.nu_new[j] = -log(u) / (1.0 + a.lam_new[j]);
  }
}

// The FP32-pair form of the two products (inverse factor in FP32 pairs): the
// dot products run on the FP32 pipe (pair FMAs, two accumulators per lane,
// a pair reduction across the warp), and s_j and nu_j^{-1} come from
// tail_noise_kernel, which draws them beside the factorization.  GB300's FP64
// pipe is 1/64 of its FP32 rate, so the FP64 forms above are bound by the
// FP64 work of their longest rows.  Block: 8 rows, one warp each.
constexpr int kTailChunk = 1024;

__device__ __forceinline__ df2 warp_sum_df(df2 v) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const df2 o{__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off)};
    v = df_add(v, o);
  }
  return v;
}

// v_i = sum_{j <= i} Linv[i][j] (S_j xtz_j) + s_i, with s_i read from v and
// v_i written back in place as an FP32 pair.
__global__ void __launch_bounds__(256) tail_w_df_kernel(TailArgs a0) {
  const TailArgs a = tail_chain(a0, blockIdx.y);
  __shared__ df2 s_u[kTailChunk];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.x * 8, i = i0 + warp;
  const int jend = min(a.p, i0 + 8);  // columns any row of the block reads
  const df2* row = reinterpret_cast<const df2*>(a.Linv) + (size_t)i * a.P;
  float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
  for (int c0 = 0; c0 < jend; c0 += kTailChunk) {
    const int c1 = min(c0 + kTailChunk, jend);
    __syncthreads();
    for (int j = c0 + (int)threadIdx.x; j < c1; j += blockDim.x) s_u[j - c0] = df_split(a.S[j] * a.xtz[j]);
    __syncthreads();
    if (i < a.p) {
      const int e1 = min(c1, i + 1);
      int j = c0 + lane;
      for (; j + 32 < e1; j += 64) {
        df_fma(h0, l0, row[j], s_u[j - c0]);
        df_fma(h1, l1, row[j + 32], s_u[j + 32 - c0]);
      }
      if (j < e1) df_fma(h0, l0, row[j], s_u[j - c0]);
    }
  }
  if (i >= a.p) return;
  const df2 t = warp_sum_df(df_add(df_renorm(h0, l0), df_renorm(h1, l1)));
  if (lane == 0) {
    const double v = df_value(t) + a.v[i];
    reinterpret_cast<df2*>(a.v)[i] = df_split(v);
  }
}

// beta_j = S_j sum_{i >= j} LinvT[j][i] v_i, v as FP32 pairs (tail_w_df_kernel).
__global__ void __launch_bounds__(256) tail_beta_df_kernel(TailArgs a0) {
  const TailArgs a = tail_chain(a0, blockIdx.y);
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= a.p) return;
  const int j = warp;
  const df2* row = reinterpret_cast<const df2*>(a.LinvT) + (size_t)j * a.P;
  const df2* v = reinterpret_cast<const df2*>(a.v);
  float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
  int i = j + lane;
  for (; i + 32 < a.p; i += 64) {
    df_fma(h0, l0, row[i], v[i]);
    df_fma(h1, l1, row[i + 32], v[i + 32]);
  }
  if (i < a.p) df_fma(h0, l0, row[i], v[i]);
  const df2 t = warp_sum_df(df_add(df_renorm(h0, l0), df_renorm(h1, l1)));
  if (lane == 0) {
    const double bj = a.S[j] * df_value(t);
    a.beta_new[j] = bj;
    if (!isfinite(bj) && *(volatile int*)a.err == 0) set_error(a.err, kErrNonFinite);
  }
}

// beta by block substitution, for the factorization without the inverse
// factor (Sect. 5, beta update, steps iv to viii: the same two triangular
// systems the explicit inverse is applied to):
//   b = S X^T z;  L~ y = b:    y_k = L~_kk^{-1} (b_k - sum_{j<k} L~_kj y_j)
//   v = y + s;    L~^T x = v:  x_k = L~_kk^{-T} (v_k - sum_{i>k} L~_ik^T x_i)
//   beta = S x   (s and the nu_j^{-1} draws: tail_noise_kernel, earlier).
// One thread-block cluster of kSolveCTAs blocks per chain, FP32 pairs.  Block
// c of the cluster owns the tile rows t with t % kSolveCTAs == c and keeps
// their part of the right-hand side in its shared memory.  Step k: the owner
// of tile k solves the diagonal tile (y_k or x_k), writes the 32 values into
// every block's shared memory (distributed shared memory) and the cluster
// synchronizes; then every block updates its own rows below (forward,
// reading the transposed factor tiles) or above (backward, the factor's own
// rows) with coalesced reads.  The value buffer alternates between two slots
// by step, so one cluster barrier per step suffices.  Rows past p (padding)
// carry zero.  blockDim.x must be kSolveThreads.
constexpr int kSolveCTAs = 4;
constexpr int kSolveThreads = 256;
constexpr int kSolveMaxRows = (kMaxTiles + kSolveCTAs - 1) / kSolveCTAs * NB;  // rows a block can own

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// *local_ptr in block `cta` of this cluster = v
__device__ __forceinline__ void st_cluster_df2(df2* local_ptr, uint32_t cta, df2 v) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_u32(local_ptr)), "r"(cta));
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(ra), "f"(v.hi), "f"(v.lo) : "memory");
}
// the diagonal tile inverse of tile k: two 16-byte pieces per thread
__device__ __forceinline__ void diag_tile_fetch2(const df2* Li, int P, int k, float4 (&v)[2]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int e = threadIdx.x + h * kSolveThreads, rr = e >> 4, cc = (e & 15) * 2;
    v[h] = __ldg(reinterpret_cast<const float4*>(Li + (size_t)(k * NB + rr) * P + k * NB + cc));
  }
}
__device__ __forceinline__ void diag_tile_put2(df2 (*D)[NB + 1], const float4 (&v)[2]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int e = threadIdx.x + h * kSolveThreads, rr = e >> 4, cc = (e & 15) * 2;
    D[rr][cc] = df2{v[h].x, v[h].y};
    D[rr][cc + 1] = df2{v[h].z, v[h].w};
  }
}

__global__ void __cluster_dims__(kSolveCTAs, 1, 1) __launch_bounds__(kSolveThreads, 1)
    tail_solve_kernel(TailArgs a0) {
  const TailArgs a = tail_chain(a0, blockIdx.x / kSolveCTAs);
  __shared__ df2 r[kSolveMaxRows];       // this block's rows: b, then v, then x
  __shared__ double sv[kSolveMaxRows];   // s (the noise) of this block's rows
  __shared__ DTile sD;                   // diagonal inverse tile of the step this block owns
  __shared__ df2 s_part[4][NB];
  __shared__ df2 s_val[2][NB];           // the solved tile of a step (written by its owner)
  const int P = a.P, p = a.p, T = P / NB, tid = threadIdx.x;
  const int rank = (int)cluster_ctarank();
  const int nt = T > rank ? (T - rank + kSolveCTAs - 1) / kSolveCTAs : 0;  // tiles this block owns
  const df2* const L = static_cast<const df2*>(a.L);
  const df2* const LT = static_cast<const df2*>(a.LinvT);
  const df2* const Li = static_cast<const df2*>(a.Linv);
  // local row lr <-> tile rank + kSolveCTAs (lr / NB), row lr % NB
  auto grow = [&](int lr) { return (rank + kSolveCTAs * (lr / NB)) * NB + (lr % NB); };
  for (int lr = tid; lr < nt * NB; lr += kSolveThreads) {
    const int i = grow(lr);
    r[lr] = i < p ? df_split(a.S[i] * a.xtz[i]) : df2{0.0f, 0.0f};
    sv[lr] = i < p ? a.v[i] : 0.0;
  }
  // step st = 0 .. 2T-1: forward tile k = st, then backward tile k = 2T-1-st
  auto tile_of = [&](int st) { return st < T ? st : 2 * T - 1 - st; };
  auto next_owned = [&](int st) {
    for (int s2 = st; s2 < 2 * T; ++s2)
      if (tile_of(s2) % kSolveCTAs == rank) return s2;
    return 2 * T;
  };
  float4 nxt[2];
  int nst = next_owned(0);
  if (nst < 2 * T) diag_tile_fetch2(Li, P, tile_of(nst), nxt);
  cluster_sync_all();  // every block of the cluster runs before any remote write
  for (int st = 0; st < 2 * T; ++st) {
    const bool fwd = st < T;
    const int k = tile_of(st), buf = st & 1;
    if (k % kSolveCTAs == rank) {
      // the owner solves the diagonal tile from its rows of tile k
      diag_tile_put2(sD, nxt);
      nst = next_owned(st + 1);
      if (nst < 2 * T) diag_tile_fetch2(Li, P, tile_of(nst), nxt);
      __syncthreads();
      const int lt = k / kSolveCTAs;
      if (tid < 4 * NB) {
        const int c = tid & 31, q0 = (tid >> 5) * 8;
        float h = 0.0f, l = 0.0f;
#pragma unroll
        for (int q = q0; q < q0 + 8; ++q)
          df_fma(h, l, fwd ? sD[c][q] : sD[q][c], r[lt * NB + q]);  // L~_kk^{-1} or its transpose
        s_part[tid >> 5][c] = df_renorm(h, l);
      }
      __syncthreads();
      if (tid < NB) {
        const int i = k * NB + tid;
        df2 y = df_add(df_add(s_part[0][tid], s_part[1][tid]), df_add(s_part[2][tid], s_part[3][tid]));
        if (i >= p) y = df2{0.0f, 0.0f};
        // forward: the rows of tile k become v = y + s; backward: x
        r[lt * NB + tid] = fwd ? (i < p ? df_split(df_value(y) + sv[lt * NB + tid]) : df2{0.0f, 0.0f}) : y;
#pragma unroll
        for (int c = 0; c < kSolveCTAs; ++c) st_cluster_df2(&s_val[buf][tid], (uint32_t)c, y);
      }
    }
    cluster_sync_all();
    // this block's rows below tile k (forward) or above it (backward)
    const df2* const M = (fwd ? LT : L) + (size_t)k * NB * P;
    for (int lr = tid; lr < nt * NB; lr += kSolveThreads) {
      const int t = rank + kSolveCTAs * (lr / NB);
      if (fwd ? t <= k : t >= k) continue;
      const int i = t * NB + (lr % NB);
      float hh = 0.0f, ll = 0.0f;
      float2 m[NB];
#pragma unroll
      for (int c = 0; c < NB; ++c) m[c] = __ldg(reinterpret_cast<const float2*>(M + (size_t)c * P + i));
#pragma unroll
      for (int c = 0; c < NB; ++c) df_fma(hh, ll, df2{m[c].x, m[c].y}, s_val[buf][c]);
      r[lr] = df_sub(r[lr], df_renorm(hh, ll));
    }
    __syncthreads();
  }
  for (int lr = tid; lr < nt * NB; lr += kSolveThreads) {
    const int i = grow(lr);
    if (i < p) {
      const double bj = a.S[i] * df_value(r[lr]);
      a.beta_new[i] = bj;
      if (!isfinite(bj) && *(volatile int*)a.err == 0) set_error(a.err, kErrNonFinite);
    }
  }
  cluster_sync_all();  // no block leaves while another may still write into it
}

// The draws the FP32-pair tails need, apart from the factor: s_j (into v)
// and nu_j^{-1}.  They depend only on the counters and lambda^{-2}, so they
// run beside the factorization.  One thread per j, chains on blockIdx.y.
__global__ void __launch_bounds__(256) tail_noise_kernel(TailArgs a0) {
  const TailArgs a = tail_chain(a0, blockIdx.y);
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.p) return;
  const uint32_t sweep = (uint32_t)(*a.k_dev + 1);
  const Rng rng{a.rng.k0, a.rng.k1, a.rng.chain, a.rng.problem};
  const uint4 w = rng.words((uint32_t)j, sweep, kPurBeta);
  double u, uc;
  unit_pair(w.x, w.y, u, uc);
  a.v[j] = std_normal_from_unit(u, uc);
  const uint4 wn = rng.words((uint32_t)j, sweep, kPurNu);
  unit_pair(wn.x, wn.y, u, uc);
  a.nu_new[j] = -log(u) / (1.0 + a.lam_new[j]);
}

// Commit (single CTA): xi^{-1}, state, compute-type beta, ring, k.
__global__ void __launch_bounds__(1024) commit_kernel(TailArgs a0) {
  const TailArgs a = tail_chain(a0, blockIdx.y);
  __shared__ int s_ok;
  __shared__ int64_t s_sweep;
  if (threadIdx.x == 0) {
    s_ok = (*(volatile int*)a.err == 0);
    s_sweep = *a.k_dev + 1;
  }
  __syncthreads();
  if (!s_ok) return;
  const int64_t sweep = s_sweep;
  const bool rec = (sweep % a.thin) == 0;
  const int64_t slot = rec ? ((sweep / a.thin) - 1) % a.ring_size : 0;
  for (int j = threadIdx.x; j < a.ld; j += blockDim.x) {
    double bj = 0.0;
    if (j < a.p) {
      bj = a.beta_new[j];
      a.beta[j] = bj;
      a.lam[j] = a.lam_new[j];
      if (a.update_mask & HS_UPD_NU) a.nu[j] = a.nu_new[j];
      if (rec) {
        a.ring_beta[slot * a.p + j] = bj;
        a.ring_lam[slot * a.p + j] = a.lam_new[j];
      }
      if (a.colscale) bj *= (double)a.colscale[j];
    }
    if (a.beta_c_is_double)
      static_cast<double*>(a.beta_c)[j] = bj;
    else
      static_cast<float*>(a.beta_c)[j] = (float)bj;
  }
  if (threadIdx.x == 0) {
    const double tn = *a.tau_new;
    const Rng rng{a.rng.k0, a.rng.k1, a.rng.chain, a.rng.problem};
    const uint4 w = rng.words(0u, (uint32_t)sweep, kPurXi);
    double u, uc;
    unit_pair(w.x, w.y, u, uc);
    a.scal[0] = tn;
    if (a.update_mask & HS_UPD_XI) a.scal[1] = -log(u) / (1.0 + tn);
    if (rec) a.ring_tau[slot] = tn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    *a.k_dev_rw = sweep;
  }
}

__global__ void beta_c_kernel(const double* beta, const float* colscale, int p, int ld, void* beta_c, int is_double) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ld; j += gridDim.x * blockDim.x) {
    double b = 0.0;
    if (j < p) b = beta[j] * (colscale ? (double)colscale[j] : 1.0);
    if (is_double)
      static_cast<double*>(beta_c)[j] = b;
    else
      static_cast<float*>(beta_c)[j] = (float)b;
  }
}

__global__ void wait_timeout_kernel(int* flag, int64_t max_spins, int* err) {
  const uint64_t t0 = global_ns();
  bool seen = false;
  for (int64_t i = 0; i < max_spins; ++i) {
    if (*(volatile int*)flag != 0) {
      seen = true;
      break;
    }
    if (global_ns() - t0 > 2000000000ull) break;
  }
  if (!seen) set_error(err, kErrTimeout);
}

}  // namespace

// Every kernel that may run beside the X-stream asks for the maximum shared
// memory carveout: an SM whose resident blocks use one L1/shared split cannot
// take a block that wants another, so a kernel left at the default split
// would wait for the X-stream's blocks to drain.
cudaError_t linalg_prepare() {
  const void* fns[] = {(const void*)shrink_kernel,
                       (const void*)build_kernel,
                       (const void*)panel_kernel<HS_CHOL_F64>,

                       (const void*)update_kernel<HS_CHOL_F64>,

                       (const void*)step_df_kernel,
                       (const void*)chol_persistent_kernel,
                       (const void*)tail_w_kernel<double>,
                       (const void*)tail_beta_kernel<double>,
                       (const void*)tail_w_df_kernel,
                       (const void*)tail_beta_df_kernel,
                       (const void*)tail_solve_kernel,
                       (const void*)tail_noise_kernel,
                       (const void*)commit_kernel,
                       (const void*)beta_c_kernel,
                       (const void*)wait_timeout_kernel};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaFuncSetAttribute((const void*)step_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kStepPadBytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute((const void*)chol_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kPersistSmem);
}

int chol_persistent_grid(int device, int nchains) {
  int coop = 0, sms = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chol_persistent_kernel, 256, kPersistSmem) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  if (!coop || sms < 2 || per_sm < 1) return 0;
  // one chain: one block per SM (the X-stream shares the SMs); several: every
  // block that fits, and at least one worker besides the chain blocks
  if (nchains <= 1) return sms;
  const int g = sms * per_sm;
  return g > nchains ? g : 0;
}

cudaError_t shrink_launch(const ShrinkArgs& a, cudaStream_t s, int nchains) {
  shrink_kernel<<<dim3((a.p + kShrinkThreads - 1) / kShrinkThreads, nchains), kShrinkThreads, 0, s>>>(a);
  return cudaGetLastError();
}

size_t chol_sync_words(int P) {
  const size_t T = (size_t)(P / NB);
  return kSyncHeader + 4 * T * T + T;
}

// ---- the worker task list of the single-launch factorization -------------
// Canonical task ids: step k's tasks are numbered from s0[k] in the order
// C(i,k) (i = k+2..T-1), X(k,j) (j < k), UA(i,j,k) (lower triangle of tile
// rows/cols k+1..T-1 column by column without (k+1,k+1)), UB(i,j,k) (row by
// row).  The list is the start order of a simulated schedule (list
// scheduling): W workers take the ready task with the longest remaining path
// (bottom level) whenever they are free, beside one processor that runs the
// diagonal chain's two nodes per step (L_kk^{-1}; then L_{k+1,k} and the next
// diagonal update).  The start order is a topological order of the whole graph
// including the chain, which is what the kernel's wait-free progress argument
// needs; it is checked here and replaced by the canonical order if the check
// fails.
namespace {
struct HostIds {
  int T;
  bool inv;
  std::vector<int> s0;
  HostIds(int T_, bool inv_) : T(T_), inv(inv_), s0(T_ + 1, 0) {
    for (int k = 0; k < T; ++k) s0[k + 1] = s0[k] + nTasks(T, k, inv);
  }
  int C(int i, int k) const { return s0[k] + (i - k - 2); }
  int X(int k, int j) const { return s0[k] + nC(T, k) + j; }
  int UA(int i, int j, int k) const {
    const int m = T - k - 1, q = j - k - 1;
    return s0[k] + nC(T, k) + (inv ? k : 0) + q * m - q * (q - 1) / 2 + (i - j) - 1;
  }
  int UB(int i, int j, int k) const { return s0[k] + nC(T, k) + k + nUA(T, k) + (i - k - 1) * (k + 1) + j; }
  // kind 0 C, 1 X, 2 UA, 3 UB
  void decode(int t, int& kind, int& i, int& j, int& k) const {
    int lo = 0, hi = T - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s0[mid] <= t) lo = mid; else hi = mid - 1;
    }
    k = lo;
    int u = t - s0[k];
    const int c = nC(T, k), ua = nUA(T, k);
    if (u < c) { kind = 0; i = k + 2 + u; j = k; return; }
    u -= c;
    if (inv) {
      if (u < k) { kind = 1; i = k; j = u; return; }
      u -= k;
    }
    if (u < ua) {
      const int m = T - k - 1;
      int idx = u + 1, q = 0;
      while (idx >= m - q) { idx -= m - q; ++q; }
      kind = 2; j = k + 1 + q; i = j + idx; return;
    }
    u -= ua;
    kind = 3; i = k + 1 + u / (k + 1); j = u % (k + 1);
  }
};
}  // namespace

std::vector<int> chol_task_order(int T, int workers, bool inverse) {
  const HostIds id(T, inverse);
  const int n = id.s0[T];
  const int N = n + 2 * T;  // chain nodes: n + 2k (L_kk^{-1}), n + 2k + 1 (L_{k+1,k}, next diagonal)
  // Each panel task C(i,k) also applies UA(i,k+1,k), the next update of its
  // own tile row, from the L_ik it still holds (one task instead of two on
  // every row's path C(i,k) -> UA(i,k+1,k) -> C(i,k+1)); rep maps a merged
  // update to its C task.  The canonical order without the merged updates
  // is still topological (a C task is listed at the start of its step).
  std::vector<int> rep(N);
  for (int v = 0; v < N; ++v) rep[v] = v;
  for (int k = 0; k + 2 < T; ++k)
    for (int i = k + 2; i < T; ++i) rep[id.UA(i, k + 1, k)] = id.C(i, k);
  std::vector<int> canonical;
  for (int t = 0; t < n; ++t)
    if (rep[t] == t) canonical.push_back(t);
  const int nlive = (int)canonical.size();
  if (nlive == 0 || workers < 1) return canonical;
  auto Li = [&](int k) { return n + 2 * k; };
  auto Ln = [&](int k) { return n + 2 * k + 1; };
  std::vector<std::vector<int>> deps(N);
  for (int t = 0; t < n; ++t) {
    int kind, i, j, k;
    id.decode(t, kind, i, j, k);
    auto& d = deps[t];
    if (kind == 0) {
      d.push_back(Li(k));
      if (k >= 1) d.push_back(id.UA(i, k, k - 1));
    } else if (kind == 1) {
      d.push_back(Li(k));
      d.push_back(id.UB(k, j, k - 1));
    } else if (kind == 2) {
      d.push_back(i == k + 1 ? Ln(k) : id.C(i, k));
      if (j != i) d.push_back(j == k + 1 ? Ln(k) : id.C(j, k));
      if (k >= 1) d.push_back(id.UA(i, j, k - 1));
    } else {
      d.push_back(i == k + 1 ? Ln(k) : id.C(i, k));
      d.push_back(j < k ? id.X(k, j) : Li(k));
      if (k > j) d.push_back(id.UB(i, j, k - 1));
    }
  }
  for (int k = 0; k < T; ++k) {
    if (k >= 1) deps[Li(k)].push_back(Ln(k - 1));
    if (k >= 2) deps[Li(k)].push_back(id.UA(k, k, k - 2));
    if (k + 1 < T) {
      deps[Ln(k)].push_back(Li(k));
      if (k >= 1) {
        deps[Ln(k)].push_back(id.UA(k + 1, k, k - 1));
        deps[Ln(k)].push_back(id.UA(k + 1, k + 1, k - 1));
      }
    }
  }
  // the merged updates' inputs join their C tasks; readers of either read the C task
  for (int v = 0; v < N; ++v) {
    if (rep[v] == v) continue;
    for (int d : deps[v]) deps[rep[v]].push_back(d);
    deps[v].clear();
  }
  for (int v = 0; v < N; ++v) {
    std::vector<int> dd;
    for (int d : deps[v]) {
      if (d < 0 || d >= N) return canonical;
      const int r = rep[d];
      if (r != v && std::find(dd.begin(), dd.end(), r) == dd.end()) dd.push_back(r);
    }
    deps[v].swap(dd);
  }
  // durations (us, measured on GB300): diagonal tile 10, panel tile and next
  // diagonal 6, tile task 6, a C task with its merged update 12
  std::vector<double> dur(N, 6.0);
  for (int k = 0; k + 2 < T; ++k)
    for (int i = k + 2; i < T; ++i) dur[id.C(i, k)] = 12.0;
  for (int k = 0; k < T; ++k) {
    dur[Li(k)] = 10.0;
    dur[Ln(k)] = 6.0;
  }
  std::vector<std::vector<int>> succ(N);
  for (int v = 0; v < N; ++v)
    for (int d : deps[v]) succ[d].push_back(v);
  // bottom levels in reverse topological order
  std::vector<int> cnt(N), topo;
  topo.reserve(N);
  std::vector<int> stack;
  for (int v = 0; v < N; ++v) {
    cnt[v] = (int)deps[v].size();
    if (cnt[v] == 0) stack.push_back(v);
  }
  while (!stack.empty()) {
    const int v = stack.back();
    stack.pop_back();
    topo.push_back(v);
    for (int w : succ[v])
      if (--cnt[w] == 0) stack.push_back(w);
  }
  if ((int)topo.size() != N) return canonical;
  std::vector<double> bl(N, 0.0);
  for (int x = N - 1; x >= 0; --x) {
    const int v = topo[x];
    double m = 0.0;
    for (int w : succ[v]) m = std::max(m, bl[w]);
    bl[v] = dur[v] + m;
  }
  // event simulation
  std::vector<int> rem(N);
  for (int v = 0; v < N; ++v) rem[v] = (int)deps[v].size();
  using RQ = std::pair<double, int>;  // (-bottom level, id): largest bottom level first, then smallest id
  std::priority_queue<RQ, std::vector<RQ>, std::greater<RQ>> ready;
  std::priority_queue<int, std::vector<int>, std::greater<int>> chain_ready;
  using EV = std::pair<double, int>;
  std::priority_queue<EV, std::vector<EV>, std::greater<EV>> ev;
  for (int v = 0; v < N; ++v)
    if (rem[v] == 0 && rep[v] == v) {
      if (v >= n) chain_ready.push(v); else ready.push({-bl[v], v});
    }
  std::vector<int> out;
  out.reserve(nlive);
  std::vector<double> start(N, -1.0);
  double now = 0.0;
  int free_w = workers;
  bool chain_busy = false;
  for (;;) {
    while (free_w > 0 && !ready.empty()) {
      const int v = ready.top().second;
      ready.pop();
      start[v] = now;
      out.push_back(v);
      --free_w;
      ev.push({now + dur[v], v});
    }
    if (!chain_busy && !chain_ready.empty()) {
      const int v = chain_ready.top();
      chain_ready.pop();
      start[v] = now;
      chain_busy = true;
      ev.push({now + dur[v], v});
    }
    if (ev.empty()) break;
    now = ev.top().first;
    const int v = ev.top().second;
    ev.pop();
    if (v >= n) chain_busy = false; else ++free_w;
    for (int w : succ[v])
      if (--rem[w] == 0) {
        if (w >= n) chain_ready.push(w); else ready.push({-bl[w], w});
      }
  }
  if ((int)out.size() != nlive) return canonical;
  // check: a permutation of the live tasks, and every node starts no earlier than its inputs
  std::vector<char> seen(n, 0);
  for (int v : out) {
    if (v < 0 || v >= n || rep[v] != v || seen[v]) return canonical;
    seen[v] = 1;
  }
  for (int v = 0; v < N; ++v)
    for (int d : deps[v])
      if (!(start[d] >= 0.0 && start[v] >= start[d] + dur[d] - 1e-9)) return canonical;
  return out;
}

std::vector<int> chol_task_codes(int T, int workers, bool inverse) {
  const HostIds id(T, inverse);
  std::vector<int> order = chol_task_order(T, workers, inverse);
  for (int& t : order) {
    int kind, i, j, k;
    id.decode(t, kind, i, j, k);
    if (kind == 0) j = k + 1;  // C(i,k) with its merged update UA(i,k+1,k)
    t = kind | (k << 2) | (i << 10) | (j << 18);
  }
  return order;
}

// The task list of one block-column launch: the panel tiles C(i, k) below the
// chain's own L_{k+1,k} and the updates UA(i, j, k) of the block column's
// later tile columns (the chain applies the last update of the next diagonal
// tile itself), for k in [k0, k1).  As for the single launch, the list is the
// start order of a simulated list schedule (ready task with the longest
// remaining path first, beside the diagonal chain), so the few tasks the chain
// waits on next are taken before the bulk; the order is checked to be
// topological (every task after the tasks of this launch it reads) and the
// canonical order (step by step) is used if the check fails.
std::vector<int> chol_block_task_codes(int T, int k0, int k1, int workers) {
  auto code = [](int kind, int i, int j, int k) { return kind | (k << 2) | (i << 10) | (j << 18); };
  struct Task {
    int kind, i, j, k;
  };
  std::vector<Task> tasks;
  for (int k = k0; k < k1; ++k) {
    for (int i = k + 2; i < T; ++i) tasks.push_back({0, i, k, k});
    for (int j = k + 1; j < k1; ++j)
      for (int i = j; i < T; ++i)
        if (!(i == k + 1 && j == k + 1)) tasks.push_back({2, i, j, k});
  }
  const int n = (int)tasks.size();
  std::vector<int> canonical(n);
  for (int t = 0; t < n; ++t) canonical[t] = code(tasks[t].kind, tasks[t].i, tasks[t].j, tasks[t].k);
  if (n == 0 || workers < 1) return canonical;
  // ids: tasks 0..n-1; chain nodes n + 2 (k - k0) (L_kk^{-1}), + 1 (L_{k+1,k} and the next diagonal)
  const int nk = k1 - k0, N = n + 2 * nk;
  auto Li = [&](int k) { return n + 2 * (k - k0); };
  auto Ln = [&](int k) { return n + 2 * (k - k0) + 1; };
  std::vector<int> idC((size_t)T * T, -1), idUA((size_t)T * T * (nk > 0 ? nk : 1), -1);
  auto ua_at = [&](int i, int j, int k) -> int& { return idUA[((size_t)(k - k0) * T + i) * T + j]; };
  for (int t = 0; t < n; ++t) {
    const Task& x = tasks[t];
    if (x.kind == 0) idC[(size_t)x.i * T + x.k] = t; else ua_at(x.i, x.j, x.k) = t;
  }
  auto UA = [&](int i, int j, int k) { return (k >= k0 && k < k1) ? ua_at(i, j, k) : -1; };
  std::vector<std::vector<int>> deps(N);
  auto add = [&](int v, int d) {
    if (d >= 0) deps[v].push_back(d);
  };
  for (int t = 0; t < n; ++t) {
    const Task& x = tasks[t];
    if (x.kind == 0) {
      add(t, Li(x.k));
      add(t, UA(x.i, x.k, x.k - 1));
    } else {
      add(t, x.i == x.k + 1 ? Ln(x.k) : idC[(size_t)x.i * T + x.k]);
      if (x.j != x.i) add(t, x.j == x.k + 1 ? Ln(x.k) : idC[(size_t)x.j * T + x.k]);
      add(t, UA(x.i, x.j, x.k - 1));
    }
  }
  for (int k = k0; k < k1; ++k) {
    if (k > k0) add(Li(k), Ln(k - 1));
    add(Li(k), UA(k, k, k - 2));
    if (k + 1 < T) {
      add(Ln(k), Li(k));
      add(Ln(k), UA(k + 1, k, k - 1));
      if (k + 1 < k1) add(Ln(k), UA(k + 1, k + 1, k - 1));
    }
  }
  // durations (us, as the single launch): diagonal tile 10, panel tile and next diagonal 6, tile task 6
  std::vector<double> dur(N, 6.0);
  for (int k = k0; k < k1; ++k) dur[Li(k)] = 10.0;
  std::vector<std::vector<int>> succ(N);
  for (int v = 0; v < N; ++v)
    for (int d : deps[v]) succ[d].push_back(v);
  std::vector<int> cnt(N), topo, stack;
  topo.reserve(N);
  for (int v = 0; v < N; ++v)
    if ((cnt[v] = (int)deps[v].size()) == 0) stack.push_back(v);
  while (!stack.empty()) {
    const int v = stack.back();
    stack.pop_back();
    topo.push_back(v);
    for (int w : succ[v])
      if (--cnt[w] == 0) stack.push_back(w);
  }
  if ((int)topo.size() != N) return canonical;
  std::vector<double> bl(N, 0.0);
  for (int x = N - 1; x >= 0; --x) {
    const int v = topo[x];
    double m = 0.0;
    for (int w : succ[v]) m = std::max(m, bl[w]);
    bl[v] = dur[v] + m;
  }
  std::vector<int> rem(N);
  for (int v = 0; v < N; ++v) rem[v] = (int)deps[v].size();
  using RQ = std::pair<double, int>;
  std::priority_queue<RQ, std::vector<RQ>, std::greater<RQ>> ready;
  std::priority_queue<int, std::vector<int>, std::greater<int>> chain_ready;
  using EV = std::pair<double, int>;
  std::priority_queue<EV, std::vector<EV>, std::greater<EV>> ev;
  for (int v = 0; v < N; ++v)
    if (rem[v] == 0) {
      if (v >= n) chain_ready.push(v); else ready.push({-bl[v], v});
    }
  std::vector<int> out;
  out.reserve(n);
  std::vector<double> start(N, -1.0);
  double now = 0.0;
  int free_w = workers;
  bool chain_busy = false;
  for (;;) {
    while (free_w > 0 && !ready.empty()) {
      const int v = ready.top().second;
      ready.pop();
      start[v] = now;
      out.push_back(v);
      --free_w;
      ev.push({now + dur[v], v});
    }
    if (!chain_busy && !chain_ready.empty()) {
      const int v = chain_ready.top();
      chain_ready.pop();
      start[v] = now;
      chain_busy = true;
      ev.push({now + dur[v], v});
    }
    if (ev.empty()) break;
    now = ev.top().first;
    const int v = ev.top().second;
    ev.pop();
    if (v >= n) chain_busy = false; else ++free_w;
    for (int w : succ[v])
      if (--rem[w] == 0) {
        if (w >= n) chain_ready.push(w); else ready.push({-bl[w], w});
      }
  }
  if ((int)out.size() != n) return canonical;
  std::vector<char> seen(n, 0);
  for (int v : out) {
    if (v < 0 || v >= n || seen[v]) return canonical;
    seen[v] = 1;
  }
  for (int v = 0; v < N; ++v)
    for (int d : deps[v])
      if (!(start[d] >= 0.0 && start[v] >= start[d] + dur[d] - 1e-9)) return canonical;
  std::vector<int> codes(n);
  for (int q = 0; q < n; ++q) {
    const Task& x = tasks[out[q]];
    codes[q] = code(x.kind, x.i, x.j, x.k);
  }
  return codes;
}

int chol_launch_count(int P, int arith, int persistent_grid) {
  const int T = P / NB;
  if (arith == HS_CHOL_DF32) return persistent_grid > 0 ? 1 : T;
  return 1 + T + (T - 1);  // build, panels, updates (the last step has none)
}

cudaError_t chol_enqueue(const CholArgs& a, cudaStream_t s, int* launches) {
  const int T = a.P / NB;
  int n = 0;
  if (a.arith == HS_CHOL_DF32 && a.persistent_grid > 0) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)a.persistent_grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = kPersistSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = a.cooperative ? 1 : 0;
    if (launches) *launches = 1;
    return cudaLaunchKernelEx(&cfg, chol_persistent_kernel, a);
  }
  if (a.arith == HS_CHOL_DF32) {
    for (int k = 0; k < T; ++k) {
      const int m = T - k;
      step_df_kernel<<<m * (m + 1) / 2 + m * k, 256, kStepPadBytes, s>>>(a, k);
      ++n;
    }
    if (launches) *launches = n;
    return cudaGetLastError();
  }
  {
    const int64_t e = (int64_t)a.P * a.P;
    int nb = (int)((e + 255) / 256);
    if (nb > 4096) nb = 4096;
    build_kernel<<<nb, 256, 0, s>>>(a);
    ++n;
  }
  for (int k = 0; k < T; ++k) {
    panel_kernel<HS_CHOL_F64><<<T, 256, 0, s>>>(a, k);
    ++n;
    const int m = T - k - 1;
    const int nA = m * (m + 1) / 2;
    const int nB = m * (k + 1);
    if (nA + nB > 0) {
      update_kernel<HS_CHOL_F64><<<nA + nB, 256, 0, s>>>(a, k);
      ++n;
    }
  }
  if (launches) *launches = n;
  return cudaGetLastError();
}

cudaError_t tail_draw_enqueue(const TailArgs& a, cudaStream_t s, int nchains) {
  const dim3 grid((a.p * 32 + 255) / 256, nchains);
  if (a.solve) {
    if (!a.df32 || !a.L) return cudaErrorInvalidValue;
    if (a.P > kMaxTiles * NB) return cudaErrorInvalidValue;
    tail_solve_kernel<<<nchains * kSolveCTAs, kSolveThreads, 0, s>>>(a);
  } else if (a.df32) {
    // s and nu^{-1}: tail_noise_kernel, beside the factorization
    tail_w_df_kernel<<<dim3((a.p + 7) / 8, nchains), 256, 0, s>>>(a);
    tail_beta_df_kernel<<<grid, 256, 0, s>>>(a);
  } else {
    tail_w_kernel<double><<<grid, 256, 0, s>>>(a);
    tail_beta_kernel<double><<<grid, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t tail_noise_enqueue(const TailArgs& a, cudaStream_t s, int nchains) {
  if (!a.solve && !a.df32) return cudaSuccess;  // the FP64 products draw s and nu^{-1} themselves
  tail_noise_kernel<<<dim3((a.p + 255) / 256, nchains), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t commit_enqueue(const TailArgs& a, cudaStream_t s, int nchains) {
  commit_kernel<<<dim3(1, nchains), 1024, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t beta_c_launch(const double* beta, const float* colscale, int p, int ld, void* beta_c, int is_double,
                          cudaStream_t s) {
  beta_c_kernel<<<(ld + 255) / 256, 256, 0, s>>>(beta, colscale, p, ld, beta_c, is_double);
  return cudaGetLastError();
}

cudaError_t wait_timeout_launch(int* flag, int64_t max_spins, int* err, cudaStream_t s) {
  wait_timeout_kernel<<<1, 1, 0, s>>>(flag, max_spins, err);
  return cudaGetLastError();
}

}  // namespace hs

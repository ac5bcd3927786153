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
//           by a right-looking blocked Cholesky over 32 x 32 tiles, and the
//           same sweep over the tiles forms L~^{-1} by block forward
//           substitution on the identity.  L = S^{-1} L~, so
//           L^{-1} = L~^{-1} S.
//  tail     w = L^{-1} X^T z, s_j = Phi^{-1}(u_j), beta = L^{-T}(w + s)
//           (Sect. 5, beta update, steps iv to viii, with the transposes read
//           so that Cov(beta) = A^{-1}), as two parallel products with the
//           explicit inverse factor; nu_j^{-1} ~ Exp(1 + lambda_j^{-2}) and
//           xi^{-1} ~ Exp(1 + tau^{-2}) (Eq. 12, third and sixth lines); and
//           the commit of the new state, skipped when the error word is set.
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

__global__ void __launch_bounds__(kShrinkThreads) shrink_kernel(ShrinkArgs a) {
  __shared__ double s_part[kShrinkThreads / 32];
  __shared__ double s_tau;
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t sweep = (uint32_t)(*a.k_dev + 1);
  const Rng rng{a.rng.k0, a.rng.k1, a.rng.chain, a.rng.problem};
  const int j = blockIdx.x * kShrinkThreads + tid;
  double part = 0.0;
  if (j < a.p) {
    const double tau = a.scal[0];
    const uint4 w = rng.words((uint32_t)j, sweep, kPurLambda);
    double u, uc;
    unit_pair(w.x, w.y, u, uc);
    const double bj = a.beta[j];
    const double l = -log(u) / (a.nu[j] + tau * bj * bj * 0.5);
    a.lam_new[j] = l;
    part = l * bj * bj;
  }
  part = warp_sum(part);
  if (lane == 0) s_part[warp] = part;
  __syncthreads();
  if (tid == 0) {
    double bp = 0.0;
    for (int w = 0; w < kShrinkThreads / 32; ++w) bp += s_part[w];
    a.part[blockIdx.x] = bp;
    __threadfence();
    s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (warp == 0) {
    // fixed-order sum of the block partials
    double tot = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) tot += *(volatile double*)&a.part[b];
    tot = warp_sum(tot);
    // Cheng (1977) GB for shape a = (p + 1) / 2 >= 1.
    const double sh = 0.5 * (double)(a.p + 1);
    const double lam = sqrt(2.0 * sh - 1.0);
    const double bconst = sh - 1.3862943611198906;  // a - ln 4
    const double cconst = sh + lam;
    double g = sh;
    bool found = false;
    for (int r = 0; r < 64 && !found; ++r) {
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
        found = true;
      }
    }
    if (lane == 0) {
      if (!found) set_error(a.err, kErrGamma);
      const double t = g / (a.scal[1] + 0.5 * tot);
      *a.tau_new = t;
      s_tau = t;
      *a.ticket = 0u;  // ready for the next sweep
    }
  }
  __syncthreads();
  const double tn = s_tau;
  for (int jj = tid; jj < a.P; jj += kShrinkThreads) {
    double sj = 1.0;
    if (jj < a.p) {
      const double d = a.G[(size_t)jj * a.p + jj] + tn * a.lam_new[jj];
      if (!isfinite(d)) {
        set_error(a.err, kErrNonFinite);
      } else if (!(d > 0.0)) {
        set_error(a.err, kErrNotPD);
      } else {
        sj = equil_scale(d);
      }
    }
    a.S[jj] = sj;
  }
}

// ---------------------------------------------------------------------------
// Cholesky of A~ = S (G + tau Lambda) S and its inverse, FP64
// ---------------------------------------------------------------------------
__global__ void build_kernel(CholArgs a) {
  double* Ad = static_cast<double*>(a.A);
  double* Ld = static_cast<double*>(a.Linv);
  double* LTd = static_cast<double*>(a.LinvT);
  (void)Ad; (void)Ld; (void)LTd;
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

// Tile products C = As Bs over one 32 x 32 x 32 block; every thread forms
// rows {ty, ty+16} x cols {tx, tx+16} of C.  As[r][q] and Bs[q][c] are held
// in the working format of the arithmetic (FP64, or FP32 pairs).
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
template <> struct Work<HS_CHOL_DF32> {
  using E = df2;
  static __device__ __forceinline__ E from(double x) { return df_split(x); }
  static __device__ __forceinline__ void mma(const E (*As)[NB + 1], const E (*Bs)[NB + 1], int ty, int tx,
                                             double out[2][2]) {
    float h[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, l[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 4
    for (int q = 0; q < NB; ++q) {
      const df2 a0 = As[ty][q], a1 = As[ty + 16][q];
      const df2 b0 = Bs[q][tx], b1 = Bs[q][tx + 16];
      df_fma(h[0][0], l[0][0], a0, b0);
      df_fma(h[0][1], l[0][1], a0, b1);
      df_fma(h[1][0], l[1][0], a1, b0);
      df_fma(h[1][1], l[1][1], a1, b1);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) out[i][j] = df_value(h[i][j], l[i][j]);
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
template <bool kSub>
__device__ __forceinline__ void tile_mma(df2 (*C)[NB + 1], const df2 (*As)[NB + 1], const df2 (*Bt)[NB + 1]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float h[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, l[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 4
  for (int q = 0; q < NB; ++q) {
    const df2 a0 = As[ty][q], a1 = As[ty + 16][q];
    const df2 b0 = Bt[q][tx], b1 = Bt[q][tx + 16];
    df_fma(h[0][0], l[0][0], a0, b0);
    df_fma(h[0][1], l[0][1], a0, b1);
    df_fma(h[1][0], l[1][0], a1, b0);
    df_fma(h[1][1], l[1][1], a1, b1);
  }
  __syncthreads();  // all reads of As/Bt/C done before C is written (C may alias)
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const df2 v = df_renorm(h[i][j], l[i][j]);
      df2& dst = C[ty + 16 * i][tx + 16 * j];
      dst = kSub ? df_sub(dst, v) : v;
    }
  __syncthreads();
}

// Lower-triangle elements (r, q), r >= q, listed column by column (q = 0:
// rows 0..31, q = 1: rows 1..31, ...).  The trailing part of column step c
// (q > c) is a suffix of the list, (31 - c)(32 - c)/2 entries long, so every
// thread takes entries tid and tid + 256 of that suffix.
__device__ __forceinline__ void tri_entry(int idx, int& r, int& q) {
  // idx in [0, 528): column q starts at q*32 - q(q-1)/2
  int qq = (int)((65.0f - sqrtf(4225.0f - 8.0f * (float)idx)) * 0.5f);
  if (qq < 0) qq = 0;
  if (qq > 31) qq = 31;
  while (qq > 0 && qq * 32 - qq * (qq - 1) / 2 > idx) --qq;
  while (qq < 31 && (qq + 1) * 32 - (qq + 1) * qq / 2 <= idx) ++qq;
  q = qq;
  r = q + (idx - (q * 32 - q * (q - 1) / 2));
}

// Right-looking Cholesky of the lower triangle of D in place (upper set to 0),
// one block barrier per column: the trailing update uses the unscaled column,
// a_rq -= a_rc a_qc / a_cc, every thread forming 1 / a_cc itself; the columns
// are scaled by 1 / sqrt(a_cc) once at the end.  s_sq / s_rs receive the
// diagonal of the factor and its reciprocal.
__device__ void potrf_df(df2 (*D)[NB + 1], df2* s_piv, df2* s_sq, df2* s_rs, int* err, bool report) {
  const int tid = threadIdx.x;
  // this thread's two list entries, as offsets from the end of the list
  int r0, q0, r1, q1;
  tri_entry(527 - tid, r0, q0);
  const bool has1 = tid + 256 < 528;
  tri_entry(has1 ? 527 - tid - 256 : 0, r1, q1);
  for (int c = 0; c < NB; ++c) {
    __syncthreads();
    df2 d = D[c][c];
    const bool bad = !(d.hi > 0.0f) || !isfinite(d.hi);
    if (bad) d = df2{1.0f, 0.0f};
    if (tid == 0) {
      if (bad && report && *(volatile int*)err == 0) set_error(err, isfinite(D[c][c].hi) ? kErrNotPD : kErrNonFinite);
      s_piv[c] = d;
    }
    const df2 dinv = df_recip_fast(d);
    const int ntr = (31 - c) * (32 - c) / 2;  // trailing entries
    const bool e0 = tid < ntr, e1 = has1 && tid + 256 < ntr;
    df2 a0, b0, x0, a1, b1, x1;
    if (e0) {
      a0 = D[r0][c];
      b0 = D[q0][c];
      x0 = D[r0][q0];
    }
    if (e1) {
      a1 = D[r1][c];
      b1 = D[q1][c];
      x1 = D[r1][q1];
    }
    if (e0) D[r0][q0] = df_sub(x0, df_mul(a0, df_mul(b0, dinv)));
    if (e1) D[r1][q1] = df_sub(x1, df_mul(a1, df_mul(b1, dinv)));
  }
  __syncthreads();
  if (tid < NB) df_sqrt_rsqrt_fast(s_piv[tid], s_sq[tid], s_rs[tid]);
  __syncthreads();
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int r = e >> 5, c = e & 31;
    if (c > r)
      D[r][c] = df2{0.0f, 0.0f};
    else if (c == r)
      D[r][c] = s_sq[c];
    else
      D[r][c] = df_mul(D[r][c], s_rs[c]);
  }
  __syncthreads();
}

// Li = L^{-1} (lower) and LiT = its transpose by recursive doubling: with the
// inverses of the two diagonal b x b blocks of every 2b x 2b diagonal block
// known, its off-diagonal block is -Li22 (L21 Li11).  Five levels (b = 1..16),
// each two small products with at most 256 outputs.  s_rdiag = 1 / L[r][r].
// sT is a scratch tile.
__device__ void trtri_df(const df2 (*L)[NB + 1], df2 (*Li)[NB + 1], df2 (*LiT)[NB + 1], df2 (*sT)[NB + 1],
                         const df2* s_rdiag) {
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int r = e >> 5, c = e & 31;
    Li[r][c] = (r == c) ? s_rdiag[r] : df2{0.0f, 0.0f};
  }
  __syncthreads();
#pragma unroll
  for (int b = 1; b < NB; b <<= 1) {
    const int per = b * b;                 // outputs per 2b-block
    const int blk = tid / per, e = tid - blk * per;
    const bool act = blk < NB / (2 * b);
    const int ro = e / b, co = e - (e / b) * b;
    const int o = blk * 2 * b;
    if (act) {
      // T = L21 Li11: T[ro][co] = sum_{m=co}^{b-1} L[o+b+ro][o+m] Li[o+m][o+co]
      float h = 0.0f, l = 0.0f;
      for (int m = co; m < b; ++m) df_fma(h, l, L[o + b + ro][o + m], Li[o + m][o + co]);
      sT[o + ro][co] = df_renorm(h, l);
    }
    __syncthreads();
    if (act) {
      // Li21 = -Li22 T: Li[o+b+ro][o+co] = -sum_{m=0}^{ro} Li[o+b+ro][o+b+m] T[m][co]
      float h = 0.0f, l = 0.0f;
      for (int m = 0; m <= ro; ++m) df_fma(h, l, Li[o + b + ro][o + b + m], sT[o + m][co]);
      Li[o + b + ro][o + co] = df_neg(df_renorm(h, l));
    }
    __syncthreads();
  }
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int r = e >> 5, c = e & 31;
    LiT[c][r] = Li[r][c];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) step_df_kernel(CholArgs a, int k) {
  __shared__ DTile sD, sW, sX1, sX2, sLi;
  __shared__ df2 s_piv[NB], s_sq[NB], s_rs[NB];
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
  potrf_df(sD, s_piv, s_sq, s_rs, a.err, isA && i == k);
  trtri_df(sD, sLi, sX1, sX2, s_rs);  // sX1 <- (L_kk^{-1})^T, sX2 scratch
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
// tail
// ---------------------------------------------------------------------------
__device__ __forceinline__ double elem(const double* M, size_t idx) { return M[idx]; }
__device__ __forceinline__ double elem(const df2* M, size_t idx) { return df_value(M[idx]); }

// v_i = sum_{j <= i} Linv[i][j] S_j xtz_j + s_i   (one warp per row)
template <typename E>
__global__ void __launch_bounds__(256) tail_w_kernel(TailArgs a) {
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
__global__ void __launch_bounds__(256) tail_beta_kernel(TailArgs a) {
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

// Commit (single CTA): xi^{-1}, state, compute-type beta, ring, k.
__global__ void __launch_bounds__(1024) commit_kernel(TailArgs a) {
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
      a.nu[j] = a.nu_new[j];
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
    a.scal[1] = -log(u) / (1.0 + tn);
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
                       (const void*)tail_w_kernel<double>,
                       (const void*)tail_beta_kernel<double>,
                       (const void*)tail_w_kernel<df2>,
                       (const void*)tail_beta_kernel<df2>,
                       (const void*)commit_kernel,
                       (const void*)beta_c_kernel,
                       (const void*)wait_timeout_kernel};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute((const void*)step_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kStepPadBytes);
}

cudaError_t shrink_launch(const ShrinkArgs& a, cudaStream_t s) {
  shrink_kernel<<<(a.p + kShrinkThreads - 1) / kShrinkThreads, kShrinkThreads, 0, s>>>(a);
  return cudaGetLastError();
}

int chol_launch_count(int P, int arith) {
  const int T = P / NB;
  if (arith == HS_CHOL_DF32) return T;
  return 1 + T + (T - 1);  // build, panels, updates (the last step has none)
}

cudaError_t chol_enqueue(const CholArgs& a, cudaStream_t s, int* launches) {
  const int T = a.P / NB;
  int n = 0;
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

cudaError_t tail_enqueue(const TailArgs& a, cudaStream_t s, int* launches) {
  const int nb = (a.p * 32 + 255) / 256;
  if (a.df32) {
    tail_w_kernel<df2><<<nb, 256, 0, s>>>(a);
    tail_beta_kernel<df2><<<nb, 256, 0, s>>>(a);
  } else {
    tail_w_kernel<double><<<nb, 256, 0, s>>>(a);
    tail_beta_kernel<double><<<nb, 256, 0, s>>>(a);
  }
  commit_kernel<<<1, 1024, 0, s>>>(a);
  if (launches) *launches = 3;
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

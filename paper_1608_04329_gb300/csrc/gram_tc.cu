// The one-time Gram matrix G = X^T X of the stored X (Sect. 5, beta update,
// step i), to FP64 accuracy on the fifth-generation tensor cores.
//
// Method (error-free products on BF16 tensor cores): every column j of X is
// put on a fixed power-of-two grid, v_rj = x_rj 2^{-E_j} with |v| < 1 (E_j from
// the column's largest magnitude), and each v is cut into S BF16 digits
// d_1 .. d_S of weight 2^{-8t} (tc_common.cuh).  Then
//     G_ij = 2^{E_i + E_j} sum_w 2^{-8w} C_w[i][j],
//     C_w  = sum_{t+u=w} sum_r d_t(r,i) d_u(r,j),
// over every digit pair for BF16 and FP8 X (so their products are exact), and
// for FP32 and FP64 X over the pairs with t + u <= S + 1 only: each dropped
// product is below 2^14 2^{-8(S+2)} = 2^{-8S-2} of 2^{E_i + E_j}.
// Each C_w is a sum of integer products; over a window of at most 128 rows it
// stays below 2^24, so the tensor cores' FP32 accumulators hold it exactly.
// After every window the classes are combined into FP32-pair accumulators
// (error-free transformations, about 48 significant bits); every 8 windows
// the pairs are added into FP64 accumulators in shared memory, so the pairs'
// rounding stays relative to 1024 rows whatever N is.  The tile is written in
// FP64; a second kernel adds the row splits in a fixed order and applies the
// powers of two (and, for FP8 X, the column scales).
//
// Digits per storage type: FP8 e4m3 values have 4 significant bits inside a
// range of 2^18, so 3 digits represent them exactly; BF16 4, FP32 5 and FP64
// 7 digits put the remainder below 2^{-33}, 2^{-41} and 2^{-57} of the column's
// largest value (BF16 values above 2^{-24} of it are represented exactly).
//
// One CTA computes a 128 x 64 tile of G (features i of the MMA's M, features
// j of its N) over a range of rows.  Warps 0-3 load rows of X, cut them into
// digits and write the 128-byte-swizzled MN-major operand tiles into a ring of
// stages (32 rows each); warp 12 issues tcgen05.mma, one accumulator of 64
// TMEM columns per weight class; warps 4-11 read the classes back after each
// window and fold them into their registers.  Every wait is bounded (2 s).
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "hs_common.cuh"
#include "hs_internal.h"
#include "df32.cuh"
#include "hs_probit.h"
#include "tc_common.cuh"

namespace hs {
namespace {

constexpr int kBM = 128;           // features of the A operand (MMA M)
constexpr int kBN = 64;            // features of the B operand (MMA N)
constexpr int kRows = 32;          // rows per stage: two MMA K steps of 16
constexpr int kSlicerWarps = 4;    // warps 0..3
constexpr int kEpiWarps = 8;       // warps 4..11
constexpr int kMmaWarp = 12;
constexpr int kThreads = 32 * 13;
constexpr int kSlicers = 32 * kSlicerWarps;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr uint32_t kAtomBytes = kRows * 128;          // 64 features x 32 rows of BF16
constexpr uint32_t kASliceBytes = 2 * kAtomBytes;     // 128 features
constexpr uint32_t kBSliceBytes = kAtomBytes;         // 64 features

// ---- storage types: one 16-byte vector -> VE values of the compute type ------
template <int XD> struct GFmt;
template <> struct GFmt<HS_X_F64> {
  using CT = double;
  static constexpr int VE = 2, S = 7, kWindowStages = 3, kStages = 1;
  static constexpr bool kAllPairs = false;
  static __device__ __forceinline__ void cvt(const uint4& v, CT* o) {
    o[0] = __hiloint2double((int)v.y, (int)v.x);
    o[1] = __hiloint2double((int)v.w, (int)v.z);
  }
};
template <> struct GFmt<HS_X_F32> {
  using CT = float;
  static constexpr int VE = 4, S = 5, kWindowStages = 4, kStages = 2;
  static constexpr bool kAllPairs = false;
  static __device__ __forceinline__ void cvt(const uint4& v, CT* o) {
    o[0] = __uint_as_float(v.x);
    o[1] = __uint_as_float(v.y);
    o[2] = __uint_as_float(v.z);
    o[3] = __uint_as_float(v.w);
  }
};
template <> struct GFmt<HS_X_BF16> {
  using CT = float;
  static constexpr int VE = 8, S = 4, kWindowStages = 4, kStages = 3;
  static constexpr bool kAllPairs = true;
  static __device__ __forceinline__ void cvt(const uint4& v, CT* o) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      o[2 * i] = __uint_as_float(w[i] << 16);
      o[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
  }
};
template <> struct GFmt<HS_X_FP8E4M3> {
  using CT = float;
  static constexpr int VE = 16, S = 3, kWindowStages = 4, kStages = 3;
  static constexpr bool kAllPairs = true;
  static __device__ __forceinline__ void cvt(const uint4& v, CT* o) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const __nv_fp8x2_storage_t pr = (__nv_fp8x2_storage_t)((w[i] >> (16 * h)) & 0xFFFFu);
        const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(pr, __NV_E4M3);
        const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&hr));
        o[4 * i + 2 * h] = f.x;
        o[4 * i + 2 * h + 1] = f.y;
      }
    }
  }
};
// Exactness of a window: a class sum over R rows is at most R (S + 2) 2^14
// (|d_1| <= 256, other digits <= 128; classes past S + 1 hold fewer pairs),
// which must stay below 2^24.
template <int XD>
constexpr bool window_exact() {
  return GFmt<XD>::kWindowStages * kRows * (GFmt<XD>::S + 2) * 16384 <= 16777216;
}
static_assert(window_exact<HS_X_F64>() && window_exact<HS_X_F32>() && window_exact<HS_X_BF16>() &&
                  window_exact<HS_X_FP8E4M3>(),
              "class sums must stay exact in FP32 over a window");

// Weight classes w = 2 .. last_class(): one TMEM accumulator of 64 columns each.
template <int XD>
constexpr int last_class() {
  return GFmt<XD>::kAllPairs ? 2 * GFmt<XD>::S : GFmt<XD>::S + 1;
}
template <int XD>
constexpr int n_classes() {
  return last_class<XD>() - 1;
}
static_assert(n_classes<HS_X_F64>() * 64 <= 512 && n_classes<HS_X_F32>() * 64 <= 512 &&
                  n_classes<HS_X_BF16>() * 64 <= 512 && n_classes<HS_X_FP8E4M3>() * 64 <= 512,
              "the classes fit in TMEM");

template <int XD>
constexpr uint32_t stage_bytes() {
  return (uint32_t)GFmt<XD>::S * (kASliceBytes + kBSliceBytes);
}
constexpr int kAccLd = kBN + 1;        // FP64 accumulator row stride (odd: fewer bank conflicts)
constexpr int kFlushWindows = 8;        // pairs go into the FP64 accumulators every 8 windows
template <int XD>
constexpr size_t smem_bytes() {
  return 1024 + (size_t)GFmt<XD>::kStages * stage_bytes<XD>() + (size_t)kBM * kAccLd * sizeof(double);
}
static_assert(smem_bytes<HS_X_F64>() <= 227 * 1024 && smem_bytes<HS_X_F32>() <= 227 * 1024 &&
                  smem_bytes<HS_X_BF16>() <= 227 * 1024 && smem_bytes<HS_X_FP8E4M3>() <= 227 * 1024,
              "stages and accumulators fit in shared memory");

// Tile t -> (bi, bj): tiles run over bi, then bj = 0 .. min(2 bi + 1, NB - 1),
// which covers every (i, j) with j <= i exactly once.
__host__ __device__ __forceinline__ void tile_of(int t, int NB, int& bi, int& bj) {
  int b = 0;
  for (;;) {
    const int n = min(2 * b + 2, NB);
    if (t < n) break;
    t -= n;
    ++b;
  }
  bi = b;
  bj = t;
}

// Power-of-two exponent of a column from its largest magnitude (as float bits):
// |x| < 2^E for every entry.
__device__ __forceinline__ int col_exponent(unsigned int maxbits) {
  const float m = __uint_as_float(maxbits);
  if (!(m > 0.0f) || !isfinite(m)) return 0;
  int e;
  frexpf(m, &e);
  return e;
}

struct GramShared {
  uint64_t full[3], empty[3], acc_full, acc_empty, done;
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ bool gwait(uint64_t* bar, uint32_t parity, GramShared* sh, int* err) {
  if (mbar_test(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_test(bar, parity)) {
    if (*(volatile int*)&sh->abort) return false;
    if (global_ns() - t0 > 2000000000ull) {
      set_error(err, kErrTimeout);
      *(volatile int*)&sh->abort = 1;
      return false;
    }
  }
  return true;
}

// Per-column max |x| (as float bits; atomicMax on non-negative float bits orders them).
template <int XD>
__global__ void colmax_kernel(const void* __restrict__ X, int64_t N, int ld, int p, unsigned int* maxbits) {
  using F = GFmt<XD>;
  using CT = typename F::CT;
  const int nvec = ld / F::VE;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  float m[F::VE];
#pragma unroll
  for (int e = 0; e < F::VE; ++e) m[e] = 0.0f;
  const uint4* base = static_cast<const uint4*>(X);
  for (int64_t r = blockIdx.y; r < N; r += gridDim.y) {
    CT x[F::VE];
    F::cvt(__ldg(base + (size_t)r * nvec + v), x);
#pragma unroll
    for (int e = 0; e < F::VE; ++e) m[e] = fmaxf(m[e], (float)fabs(x[e]));
  }
#pragma unroll
  for (int e = 0; e < F::VE; ++e) {
    const int f = v * F::VE + e;
    if (f < p) atomicMax(maxbits + f, __float_as_uint(m[e]));
  }
}

// 13 warps: one SM sub-partition holds four of them, and each sub-partition
// has a quarter of the register file, so at most 128 registers per thread.
template <int XD>
__global__ void __launch_bounds__(kThreads, 1)
    gram_tc_kernel(const void* __restrict__ X, int64_t N, int ld, int p, const unsigned int* __restrict__ maxbits,
                   int NB, int ntiles, int splits, double* __restrict__ partial, int* err) {
  using F = GFmt<XD>;
  using CT = typename F::CT;
  constexpr int S = F::S, VE = F::VE, W = F::kWindowStages, NS = F::kStages;
  constexpr uint32_t kStage = stage_bytes<XD>();
  extern __shared__ unsigned char dyn[];
  __shared__ GramShared sh;
  __shared__ CT s_inv[kBM + kBN];  // 2^{-E_j} of the A features, then of the B features
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* base = dyn + ((1024u - (smem_u32(dyn) & 1023u)) & 1023u);  // 1024-byte aligned stages
  double* acc64 = reinterpret_cast<double*>(base + (size_t)NS * kStage);     // [kBM][kAccLd]

  const int tile = blockIdx.x % ntiles, split = blockIdx.x / ntiles;
  int bi, bj;
  tile_of(tile, NB, bi, bj);
  const int64_t r0 = N * split / splits, r1 = N * (split + 1) / splits;
  const int nst = (int)((r1 - r0 + kRows - 1) / kRows);
  const int nwin = (nst + W - 1) / W;

  if (tid < kBM + kBN) {
    const int f = tid < kBM ? kBM * bi + tid : kBN * bj + (tid - kBM);
    const int e = f < p ? col_exponent(maxbits[f]) : 0;
    s_inv[tid] = (CT)ldexp(1.0, -e);
  }
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&sh.full[s], kSlicers);
      mbar_init(&sh.empty[s], 1);
    }
    mbar_init(&sh.acc_full, 1);
    mbar_init(&sh.acc_empty, kEpiThreads);
    mbar_init(&sh.done, 1);
    sh.abort = 0;
    fence_mbar_init();
  }
  if (warp == kMmaWarp) tc::tmem_alloc(&sh.tmem, 512);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = sh.tmem;

  if (warp < kSlicerWarps) {
    // ---------------- digits of 32 rows per stage ----------------
    // thread: row r of the stage, A features [32 q, 32 q + 32), B features [16 q, 16 q + 16)
    const int r = tid >> 2, q = tid & 3;
    constexpr int NA = 32 / VE > 0 ? 32 / VE : 1;  // 16-byte vectors of the A span (VE <= 32)
    constexpr int NBV = 16 / VE > 0 ? 16 / VE : 1;
    constexpr int EA = NA * VE, EB = NBV * VE;      // values loaded (>= 32 and 16)
    const int nvec = ld / VE;
    const uint4* Xv = static_cast<const uint4*>(X);
    const int fa0 = kBM * bi + 32 * q, fb0 = kBN * bj + 16 * q;  // first A / B feature of this thread
    for (int st = 0; st < nst; ++st) {
      const int s = st % NS;
      if (st >= NS && !gwait(&sh.empty[s], ((st / NS) - 1) & 1, &sh, err)) break;
      const int64_t row = r0 + (int64_t)st * kRows + r;
      const bool live = row < r1;
      CT xa[EA], xb[EB];
#pragma unroll
      for (int k = 0; k < NA; ++k) {
        const int v = (fa0 + k * VE) / VE;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (live && fa0 + k * VE < ld) w = __ldg(Xv + (size_t)row * nvec + v);
        F::cvt(w, xa + k * VE);
      }
#pragma unroll
      for (int k = 0; k < NBV; ++k) {
        const int v = (fb0 + k * VE) / VE;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (live && fb0 + k * VE < ld) w = __ldg(Xv + (size_t)row * nvec + v);
        F::cvt(w, xb + k * VE);
      }
      unsigned char* stg = base + (size_t)s * kStage;
      // A: 4 groups of 8 features; B: 2 groups.  (VE = 16 loads 16 values for
      // the 16-wide B span and 32 for the A span, as needed.)
#pragma unroll
      for (int g = 0; g < 6; ++g) {
        const bool isA = g < 4;
        const int lf = isA ? 32 * q + 8 * g : 16 * q + 8 * (g - 4);  // feature within the A (B) block
        CT rr[8];
#pragma unroll
        for (int e = 0; e < 8; ++e)
          rr[e] = isA ? xa[8 * g + e] * s_inv[lf + e] : xb[8 * (g - 4) + e] * s_inv[kBM + lf + e];
        const uint32_t off = tc::sw128_off(r, lf & 63);
        // digit t of the eight values, written as soon as it is formed
#pragma unroll
        for (int t = 0; t < S; ++t) {
          float d8[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) d8[e] = (float)tc::digit_step(rr[e]);
          unsigned char* dst = isA ? stg + (size_t)t * kASliceBytes + (lf >> 6) * kAtomBytes + off
                                   : stg + (size_t)S * kASliceBytes + (size_t)t * kBSliceBytes + off;
          *reinterpret_cast<uint4*>(dst) = tc::pack8_bf16(d8);
        }
      }
      tc::fence_smem_to_async();
      mbar_arrive(&sh.full[s]);
    }
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16(kBM, kBN, 1, 1);  // both operands MN-major
      const uint32_t sbase = smem_u32(base);
      bool ok = true;
      for (int st = 0; st < nst && ok; ++st) {
        const int s = st % NS, win = st / W;
        const bool first = (st % W) == 0;
        if (first && win > 0 && !(ok = gwait(&sh.acc_empty, (win - 1) & 1, &sh, err))) break;
        if (!(ok = gwait(&sh.full[s], (st / NS) & 1, &sh, err))) break;
        tc::fence_after();
        const uint32_t sa = sbase + (uint32_t)s * kStage;
        const uint32_t sb = sa + S * kASliceBytes;
#pragma unroll
        for (int w = 2; w <= last_class<XD>(); ++w) {
          const uint32_t d = tmem + (uint32_t)(w - 2) * kBN;
          int n = 0;
#pragma unroll
          for (int t = 1; t <= S; ++t) {
            const int u = w - t;
            if (u < 1 || u > S) continue;
#pragma unroll
            for (int ks = 0; ks < kRows / 16; ++ks, ++n) {
              const uint64_t da = tc::sw128_desc(sa + (t - 1) * kASliceBytes + ks * 2048, kAtomBytes, 1024);
              const uint64_t db = tc::sw128_desc(sb + (u - 1) * kBSliceBytes + ks * 2048, kAtomBytes, 1024);
              tc::mma_bf16(d, da, db, idesc, (first && n == 0) ? 0 : 1);
            }
          }
        }
        tc::mma_commit(&sh.empty[s]);
        if ((st % W) == W - 1 || st == nst - 1) tc::mma_commit(&sh.acc_full);
      }
      tc::mma_commit(&sh.done);
      mbar_wait(&sh.done, 0, 2000000000ull);  // nothing in flight when the CTA leaves
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: fold each window into FP32 pairs ----------------
    const int ew = warp - kSlicerWarps;          // 0..7
    const int quad = warp & 3, half = ew >> 2;   // TMEM lanes 32 quad.., columns 32 half..
    const int i = 32 * quad + lane;              // feature of the A block = TMEM lane
    const uint32_t lane_off = (uint32_t)(32 * quad) << 16;
    float ah[32], al[32];
    double* acc_row = acc64 + (size_t)i * kAccLd + 32 * half;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      ah[c] = al[c] = 0.0f;
      acc_row[c] = 0.0;
    }
    for (int win = 0; win < nwin; ++win) {
      if (!gwait(&sh.acc_full, win & 1, &sh, err)) break;
      tc::fence_after();
      constexpr int NC = n_classes<XD>();
      constexpr int kChunk = 2;  // classes loaded per TMEM wait (register budget)
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        // f = sum_w C_w 2^{-8(w-2)} by Horner from the smallest class, in pairs
        float fh[8], fl[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) fh[e] = fl[e] = 0.0f;
#pragma unroll
        for (int top = NC; top > 0; top -= kChunk) {
          const int lo = top - kChunk > 0 ? top - kChunk : 0;  // classes lo .. top-1 (0 = class 2)
          uint32_t c[kChunk][8];
#pragma unroll
          for (int w = lo; w < top; ++w)
            tc::tmem_ld8(tmem + lane_off + (uint32_t)w * kBN + 32 * half + 8 * g, c[w - lo]);
          tc::tmem_ld_wait();
          if (g == 3 && lo == 0) {
            tc::fence_before();
            mbar_arrive(&sh.acc_empty);  // the MMA may overwrite the classes now
          }
#pragma unroll
          for (int w = top - 1; w >= lo; --w) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const float a = fh[e] * 0x1p-8f, b = __uint_as_float(c[w - lo][e]);
              const float sum = a + b;
              const float bb = sum - a;
              const float err2 = (a - (sum - bb)) + (b - bb);
              fh[e] = sum;
              fl[e] = fmaf(fl[e], 0x1p-8f, err2);
            }
          }
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const df2 v = df_add(df2{ah[8 * g + e], al[8 * g + e]}, df2{fh[e], fl[e]});
          ah[8 * g + e] = v.hi;
          al[8 * g + e] = v.lo;
        }
      }
      if ((win + 1) % kFlushWindows == 0) {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          acc_row[c] += (double)ah[c] + (double)al[c];  // the pair's value is exact in FP64
          ah[c] = al[c] = 0.0f;
        }
      }
    }
    // this CTA's part of the tile, in units of 2^{E_i + E_j}
    double* out = partial + ((size_t)split * ntiles + tile) * (kBM * kBN) + (size_t)i * kBN + 32 * half;
#pragma unroll
    for (int c = 0; c < 32; ++c) out[c] = (acc_row[c] + ((double)ah[c] + (double)al[c])) * 0x1p-16;
  }
  tc::fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc::fence_after();
    tc::tmem_free(tmem, 512);
  }
}

// G[i][j] = G[j][i] = 2^{E_i + E_j} (s_i s_j) sum over the row splits, fixed order.
__global__ void gram_reduce_kernel(const double* __restrict__ partial, int splits, int ntiles, int NB, int p,
                                   const unsigned int* __restrict__ maxbits, const float* __restrict__ colscale,
                                   double* __restrict__ G) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)p * p) return;
  const int i = (int)(e / p), j = (int)(e % p);
  if (j > i) return;
  const int bi = i / kBM, bj = j / kBN;
  int t = 0;
  for (int b = 0; b < bi; ++b) t += min(2 * b + 2, NB);
  t += bj;
  const size_t off = (size_t)(i % kBM) * kBN + (j % kBN);
  double s = 0.0;
  for (int sp = 0; sp < splits; ++sp) s += partial[((size_t)sp * ntiles + t) * (kBM * kBN) + off];
  s = ldexp(s, col_exponent(maxbits[i]) + col_exponent(maxbits[j]));
  if (colscale) s *= (double)colscale[i] * (double)colscale[j];
  G[(size_t)i * p + j] = s;
  G[(size_t)j * p + i] = s;
}

struct GramPlan {
  int NB, ntiles, splits;
};
GramPlan plan(int64_t N, int p, int num_sms) {
  GramPlan g;
  const int MB = (p + kBM - 1) / kBM;
  g.NB = (p + kBN - 1) / kBN;
  g.ntiles = 0;
  for (int b = 0; b < MB; ++b) g.ntiles += std::min(2 * b + 2, g.NB);
  int sp = num_sms / g.ntiles;
  const int64_t by_rows = N / 512;
  if (sp > by_rows) sp = (int)by_rows;
  g.splits = sp < 1 ? 1 : sp;
  return g;
}

template <int XD>
cudaError_t launch_xd(const void* X, int64_t N, int ld, int p, const float* colscale, double* G,
                      unsigned char* ws, int num_sms, int* err, cudaStream_t s) {
  const GramPlan g = plan(N, p, num_sms);
  unsigned int* maxbits = reinterpret_cast<unsigned int*>(ws);
  double* partial = reinterpret_cast<double*>(ws + ((size_t)p * sizeof(unsigned int) + 255) / 256 * 256);
  cudaError_t e = cudaMemsetAsync(maxbits, 0, (size_t)p * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  const int nvec = ld / GFmt<XD>::VE;
  const dim3 cg((nvec + 127) / 128, (unsigned)std::min<int64_t>(std::max<int64_t>(N, 1), 1024));
  colmax_kernel<XD><<<cg, 128, 0, s>>>(X, N, ld, p, maxbits);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  auto k = gram_tc_kernel<XD>;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<XD>());
  if (e != cudaSuccess) return e;
  k<<<g.ntiles * g.splits, kThreads, smem_bytes<XD>(), s>>>(X, N, ld, p, maxbits, g.NB, g.ntiles, g.splits,
                                                             partial, err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t n = (int64_t)p * p;
  gram_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(partial, g.splits, g.ntiles, g.NB, p, maxbits,
                                                                  XD == HS_X_FP8E4M3 ? colscale : nullptr, G);
  return cudaGetLastError();
}

}  // namespace

size_t gram_workspace_bytes(int64_t N, int p, int num_sms) {
  const GramPlan g = plan(N, p, num_sms);
  return ((size_t)p * sizeof(unsigned int) + 255) / 256 * 256 +
         (size_t)g.splits * g.ntiles * kBM * kBN * sizeof(double);
}

cudaError_t gram_launch(int x_dtype, const void* X, int64_t N, int ld, int p, const float* colscale, double* G,
                        void* workspace, int num_sms, int* err, cudaStream_t s) {
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  switch (x_dtype) {
    case HS_X_F64: return launch_xd<HS_X_F64>(X, N, ld, p, colscale, G, ws, num_sms, err, s);
    case HS_X_F32: return launch_xd<HS_X_F32>(X, N, ld, p, colscale, G, ws, num_sms, err, s);
    case HS_X_BF16: return launch_xd<HS_X_BF16>(X, N, ld, p, colscale, G, ws, num_sms, err, s);
    case HS_X_FP8E4M3: return launch_xd<HS_X_FP8E4M3>(X, N, ld, p, colscale, G, ws, num_sms, err, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hs

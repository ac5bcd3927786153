// Trailing updates of the blocked Cholesky factorization on the tensor cores
// (Sect. 5, beta update, step iii: the factor of X^T X + tau^{-2} Lambda^{-2},
// equilibrated to unit diagonal).
//
// The factorization runs over block columns of kTrailBlockTiles 32-wide tiles
// (four: 128 columns).  Inside a block column the FP32-pair tile tasks of
// chol_persistent_kernel factor the diagonal block and form the panel L_ib;
// everything to the right of the block column then takes the rank-128 update
//     A_ij -= sum_{k in block b} L_ik L_jk^T
// here, on the tensor cores, from exact products of BF16 digits.
//
// Digits: every entry of the equilibrated factor has |L| <= 1 (the rows of L
// have unit norm), so L sits on the fixed grid 2^0 and each FP32 pair is cut
// into six digits d_1..d_6 of weight 2^{-8t} (|d_1| <= 256, |d_t| <= 128,
// remainder below 2^{-49}); the tile tasks write them into six BF16 planes
// when they store L.  With classes C_w = sum_{t+u=w} sum_k d_t(i,k) d_u(j,k),
// w = 2..7 (pairs with t + u > 7 weigh below 2^{-56}),
//     sum_k L_ik L_jk = sum_w 2^{-8w} C_w.
// Each C_w over the (at most 128) columns of a block is an integer below 2^24:
// the pairs with a first digit are bounded through the unit row norm
// (sum_k |d_1(i,k)| <= sqrt(128) 262), the others by 128^3 each, so the FP32
// accumulators of the tensor cores hold the classes exactly.  The epilogue
// combines them into an FP32 pair (about 48 bits, absolute error near 2^{-48}
// on the unit-diagonal scale, as the pair arithmetic of the tile tasks) and
// subtracts it from the stored tile.
//
// One CTA per SM loops over work items (chain, 128-row strip, 64-column pair
// of tiles): warp 0 lane 0 loads the digit tiles of one 32-column tile of the
// block per stage by TMA into a ring of three stages (64-byte swizzle,
// K-major), warp 1 lane 0 issues
// tcgen05.mma (M 128, N 64, K 16), one TMEM accumulator of 64 columns per
// class, warp 2 owns TMEM, warps 4-11 (one per 32 x 32 output tile, each
// reading its tile's old values before the products finish) fold the classes
// and write the tiles with their update counters.  Every wait is
// bounded (2 s); a wait that runs out sets the timeout bit and the CTA winds down.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>

#include "df32.cuh"
#include "hs_common.cuh"
#include "hs_internal.h"
#include "tc_common.cuh"

namespace hs {
namespace {

constexpr int NB = 32;                  // tile
constexpr int kBlockTiles = kTrailBlockTiles;  // tiles per block column
constexpr int kDigits = 6;
constexpr int kStages = 3;
constexpr int kKc = 32;                 // columns of the block per stage (one tile; 64-byte rows)
constexpr uint32_t kADigitBytes = 128 * kKc * 2;  // 128 rows x 32 columns of BF16: 8 KB
constexpr uint32_t kBDigitBytes = 64 * kKc * 2;   // 64 rows: 4 KB
constexpr uint32_t kStageBytes = kDigits * (kADigitBytes + kBDigitBytes);  // 72 KB
constexpr size_t kSmem = 1024 + (size_t)kStages * kStageBytes;
static_assert(kSmem <= 227 * 1024, "stages fit in shared memory");
static_assert(kBlockTiles * 32 <= 128, "class sums stay exact over a block column of at most 128 columns");
constexpr int kEpiWarps = 8;            // warps 4..11: one 32 x 32 output tile each
constexpr int kThreads = 128 + 32 * kEpiWarps;
constexpr unsigned long long kEpochStride = 1024;  // as the readiness words of chol_persistent_kernel
constexpr int kSyncHeader = 8;

struct TrailShared {
  uint64_t full[kStages], empty[kStages], acc_full, acc_empty, done;
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ bool twait(uint64_t* bar, uint32_t parity, TrailShared* sh, int* err, int site) {
  if (mbar_test(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_test(bar, parity)) {
    if (*(volatile int*)&sh->abort) return false;
    if (global_ns() - t0 > 2000000000ull) {
      set_timeout(err, site);
      *(volatile int*)&sh->abort = 1;
      return false;
    }
  }
  return true;
}

// 2-D TMA load of one box into shared memory, completing on an mbarrier.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// K-major operand in the 64-byte swizzled layout TMA writes (32 BF16 per
// row, 8-row groups 512 bytes apart; descriptor layout code 4); a K step of 16
// moves the start by 32 bytes.
__device__ __forceinline__ uint64_t kmaj_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) | (1ull << 46) |
         (4ull << 61);
}

// Work items of block column b (tiles from c1 = kBlockTiles (b + 1) on are
// updated): chain m, strip s of 128 rows (tiles 4s..4s+3) reaching row tile c1,
// column pair jp (tiles 2jp, 2jp+1) with 2jp >= max(col_lo, c1), 2jp < col_hi
// and 2jp <= 4s + 3; tiles above the diagonal are not stored.
struct ItemSpace {
  int T, nstrip, s0, jp0, jp1;  // strips s0..nstrip-1, column pairs jp0..jp1-1
  __host__ __device__ ItemSpace(int T_, int b, int col_lo, int col_hi) : T(T_) {
    const int c1 = kBlockTiles * (b + 1);
    nstrip = (T + 3) / 4;
    s0 = c1 / 4;
    jp0 = max(col_lo, c1) / 2;  // only columns right of the block column
    jp1 = (min(col_hi, T) + 1) / 2;
  }
  __host__ __device__ int pairs_in_strip(int s) const {
    const int hi = min(jp1, 2 * s + 2);  // 2jp <= 4s + 3
    return hi > jp0 ? hi - jp0 : 0;
  }
  __host__ __device__ int per_chain() const {
    int n = 0;
    for (int s = s0; s < nstrip; ++s) n += pairs_in_strip(s);
    return n;
  }
  __host__ __device__ void decode(int u, int& s, int& jp) const {
    s = s0;
    for (;;) {
      const int n = pairs_in_strip(s);
      if (u < n) break;
      u -= n;
      ++s;
    }
    jp = jp0 + u;
  }
};

__global__ void __launch_bounds__(kThreads, 1)
    chol_trail_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                      TrailArgs a) {
  extern __shared__ unsigned char dyn[];
  __shared__ TrailShared sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* base = dyn + ((1024u - (smem_u32(dyn) & 1023u)) & 1023u);
  const int T = a.P / NB;
  const ItemSpace is(T, a.b, a.col_lo, a.col_hi);
  const int per_chain = is.per_chain();
  const int nitems = per_chain * a.nchains;
  const int k0 = kBlockTiles * a.b, k1 = min(k0 + kBlockTiles, T);
  const int nk = k1 - k0;  // stages per item (tile columns of the block)
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], 1);
    }
    mbar_init(&sh.acc_full, 1);
    mbar_init(&sh.acc_empty, 32 * kEpiWarps);
    mbar_init(&sh.done, 1);
    sh.abort = 0;
    fence_mbar_init();
  }
  if (warp == 2) tc::tmem_alloc(&sh.tmem, 512);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = sh.tmem;
  // the launch epoch of the factorization (chol_persistent_kernel records it)
  const unsigned long long e = *(volatile unsigned long long*)a.sync;
  const unsigned long long done_count = e * kEpochStride + (unsigned long long)k1;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    uint32_t q = 0;
    bool ok = true;
    for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
      const int m = it / per_chain;
      int s, jp;
      is.decode(it % per_chain, s, jp);
      for (int kk = 0; kk < nk && ok; ++kk, ++q) {
        const int st = q % kStages;
        if (q >= kStages && !(ok = twait(&sh.empty[st], ((q / kStages) - 1) & 1, &sh, a.err, kSiteTrailLoad))) break;
        unsigned char* stg = base + (size_t)st * kStageBytes;
        mbar_arrive_expect_tx(&sh.full[st], kStageBytes);
        const int x = NB * (k0 + kk);
#pragma unroll
        for (int t = 0; t < kDigits; ++t) {
          const int plane = (m * kDigits + t) * a.P;
          tma_load_2d(stg + t * kADigitBytes, &mapA, x, plane + 128 * s, &sh.full[st]);
          tma_load_2d(stg + kDigits * kADigitBytes + t * kBDigitBytes, &mapB, x, plane + 64 * jp, &sh.full[st]);
        }
      }
    }
    // every issued load lands before the CTA may leave
    const uint32_t nd = q < (uint32_t)kStages ? q : (uint32_t)kStages;
    for (uint32_t d = 1; d <= nd; ++d) {
      const uint32_t qq = q - d;
      mbar_wait(&sh.full[qq % kStages], (qq / kStages) & 1, 2000000000ull);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    const uint32_t idesc = tc::idesc_bf16(128, 64, 0, 0);
    const uint32_t sbase = smem_u32(base);
    uint32_t q = 0;
    int n_item = 0;
    bool ok = true;
    for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++n_item) {
      if (n_item > 0 && !(ok = twait(&sh.acc_empty, (n_item - 1) & 1, &sh, a.err, kSiteTrailMma))) break;
      tc::fence_after();
      for (int kk = 0; kk < nk && ok; ++kk, ++q) {
        const int st = q % kStages;
        if (!(ok = twait(&sh.full[st], (q / kStages) & 1, &sh, a.err, kSiteTrailMma))) break;
        tc::fence_after();
        const uint32_t sa = sbase + (uint32_t)st * kStageBytes;
        const uint32_t sb = sa + kDigits * kADigitBytes;
        const int nks = kKc / 16;  // K steps of 16
#pragma unroll
        for (int w = 2; w <= kDigits + 1; ++w) {
          int n = 0;
#pragma unroll
          for (int t = 1; t <= kDigits; ++t) {
            const int u = w - t;
            if (u < 1 || u > kDigits) continue;
            for (int ks = 0; ks < nks; ++ks, ++n)
              tc::mma_bf16(tmem + (uint32_t)(w - 2) * 64, kmaj_desc(sa + (t - 1) * kADigitBytes + ks * 32),
                           kmaj_desc(sb + (u - 1) * kBDigitBytes + ks * 32), idesc, (kk > 0 || n > 0) ? 1 : 0);
          }
        }
        tc::mma_commit(&sh.empty[st]);
      }
      if (ok) tc::mma_commit(&sh.acc_full);
    }
    tc::mma_commit(&sh.done);
    mbar_wait(&sh.done, 0, 2000000000ull);  // nothing in flight when the CTA leaves
  } else if (warp >= 4) {
    // ---------------- epilogue: one 32 x 32 output tile per warp ----------------
    const int quad = warp & 3, jj = (warp - 4) >> 2;  // tile row 4s + quad, tile column 2jp + jj
    const uint32_t lane_off = (uint32_t)(32 * quad) << 16;
    int n_item = 0;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x, ++n_item) {
      const int m = it / per_chain;
      int s, jp;
      is.decode(it % per_chain, s, jp);
      const int i = 4 * s + quad;            // tile row of this warp
      const int j = 2 * jp + jj;             // tile column
      const int r = NB * i + lane;           // matrix row of this thread
      const bool live = i < T && j < T && j <= i;  // warp-uniform
      df2* const A = static_cast<df2*>(a.A) + (size_t)m * a.P * a.P;
      // the tile's current values (independent of the products: read before they
      // finish); before the first block column they are the equilibrated
      // precision matrix that precision_pairs_kernel wrote
      df2 old[NB];
      if (live) {
        const float4* src = reinterpret_cast<const float4*>(A + (size_t)r * a.P + NB * j);
#pragma unroll
        for (int h = 0; h < NB / 2; ++h) {
          const float4 v = __ldcg(src + h);
          old[2 * h] = df2{v.x, v.y};
          old[2 * h + 1] = df2{v.z, v.w};
        }
      }
      if (!twait(&sh.acc_full, n_item & 1, &sh, a.err, kSiteTrailEpi)) break;
      tc::fence_after();
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        uint32_t c[kDigits][8];
#pragma unroll
        for (int w = 0; w < kDigits; ++w) tc::tmem_ld8(tmem + lane_off + (uint32_t)w * 64 + 32 * jj + 8 * g, c[w]);
        tc::tmem_ld_wait();
        if (g == 3) {
          tc::fence_before();
          mbar_arrive(&sh.acc_empty);  // the MMA may overwrite the classes now
        }
        if (!live) continue;
        float4 outv[4];
#pragma unroll
        for (int e2 = 0; e2 < 8; ++e2) {
          // sum_w C_w 2^{-8(w-2)} by Horner from the smallest class, in pairs; times 2^-16
          float fh = __uint_as_float(c[kDigits - 1][e2]), fl = 0.0f;
#pragma unroll
          for (int w = kDigits - 2; w >= 0; --w) {
            const float x = fh * 0x1p-8f, y = __uint_as_float(c[w][e2]);
            const float sum = x + y, bb = sum - x;
            const float er = (x - (sum - bb)) + (y - bb);
            fh = sum;
            fl = fmaf(fl, 0x1p-8f, er);
          }
          const df2 v = df_sub(old[8 * g + e2], df2{fh * 0x1p-16f, fl * 0x1p-16f});
          if (e2 & 1) {
            outv[e2 >> 1].z = v.hi;
            outv[e2 >> 1].w = v.lo;
          } else {
            outv[e2 >> 1].x = v.hi;
            outv[e2 >> 1].y = v.lo;
          }
        }
        float4* dst = reinterpret_cast<float4*>(A + (size_t)r * a.P + NB * j + 8 * g);
#pragma unroll
        for (int h = 0; h < 4; ++h) __stcg(dst + h, outv[h]);
      }
      // the tile has taken every update of this block column
      if (live) {
        // the warp's stores, ordered by the warp barrier before lane 0's release
        __syncwarp();
        if (lane == 0) {
          unsigned long long* const cntA = a.sync + (size_t)m * a.sync_words + kSyncHeader;
          asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(cntA + (size_t)i * T + j), "l"(done_count)
                       : "memory");
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 2) {
    tc::fence_after();
    tc::tmem_free(tmem, 512);
  }
}

// The lower tiles of the equilibrated precision matrix of every chain,
// A~ = S (G + tau^{-2} Lambda^{-2}) S as FP32 pairs (identity past p), from the
// Gram matrix in pairs: the work matrix the block-column factorization starts
// from.  blockIdx.y is the chain.
__global__ void precision_pairs_kernel(TrailArgs a) {
  const int m = blockIdx.y;
  const int64_t n = (int64_t)a.P * a.P;
  df2* const A = static_cast<df2*>(a.A) + (size_t)m * n;
  const df2* const G2 = static_cast<const df2*>(a.G2);
  const double* const S = a.S + (size_t)m * a.P;
  const double tau = a.tau_new[m];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / a.P), c = (int)(e % a.P);
    if ((c >> 5) > (r >> 5)) continue;  // tiles right of the diagonal tile are never read
    df2 v{0.0f, 0.0f};
    if (r < a.p && c < a.p) {
      v = df_mul(df_mul(G2[e], df2{(float)S[r], 0.0f}), df2{(float)S[c], 0.0f});
      if (r == c) v = df_add(v, df_split(S[r] * S[r] * tau * a.lam_new[(size_t)m * a.p + r]));
    } else if (r == c) {
      v = df2{1.0f, 0.0f};
    }
    A[e] = v;
  }
}

// G2 = G as FP32 pairs, P x P with zero padding (read by the first block column).
__global__ void gram_pairs_kernel(const double* __restrict__ G, int p, int P, df2* __restrict__ G2) {
  const int64_t n = (int64_t)P * P;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / P), c = (int)(e % P);
    G2[e] = (r < p && c < p) ? df_split(G[(size_t)r * p + c]) : df2{0.0f, 0.0f};
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult qr;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &qr) == cudaSuccess &&
        qr == cudaDriverEntryPointSuccess && f)
      fn = reinterpret_cast<EncodeFn>(f);
  }
  return fn;
}

}  // namespace

size_t chol_trail_smem_bytes() { return kSmem; }

cudaError_t chol_trail_prepare() {
  return cudaFuncSetAttribute((const void*)chol_trail_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kSmem);
}

// Tensor maps of the digit planes (nchains x 6 planes of P x P BF16, row-major,
// one after another): 32-column boxes of 128 rows (A) and 64 rows (B), 64-byte
// swizzle.  0 on success.
int chol_trail_make_maps(const void* digits, int P, int nchains, void* mapA, void* mapB) {
  EncodeFn enc = encode_fn();
  if (!enc) return -1;
  const cuuint64_t dims[2] = {(cuuint64_t)P, (cuuint64_t)P * kDigits * (cuuint64_t)nchains};
  const cuuint64_t strides[1] = {(cuuint64_t)P * 2};
  const cuuint32_t estr[2] = {1, 1};
  const cuuint32_t boxA[2] = {kKc, 128}, boxB[2] = {kKc, 64};
  CUresult r = enc(reinterpret_cast<CUtensorMap*>(mapA), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(digits),
                   dims, strides, boxA, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return -1;
  r = enc(reinterpret_cast<CUtensorMap*>(mapB), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(digits), dims,
          strides, boxB, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

int chol_trail_items(int P, int b, int col_lo, int col_hi, int nchains) {
  const ItemSpace is(P / NB, b, col_lo, col_hi);
  return is.per_chain() * nchains;
}

cudaError_t chol_trail_launch(const void* mapA, const void* mapB, const TrailArgs& a, int grid, cudaStream_t s) {
  if (chol_trail_items(a.P, a.b, a.col_lo, a.col_hi, a.nchains) == 0) return cudaSuccess;
  CUtensorMap ma, mb;
  memcpy(&ma, mapA, sizeof(ma));
  memcpy(&mb, mapB, sizeof(mb));
  chol_trail_kernel<<<grid, kThreads, kSmem, s>>>(ma, mb, a);
  return cudaGetLastError();
}

cudaError_t precision_pairs_launch(const TrailArgs& a, cudaStream_t s) {
  precision_pairs_kernel<<<dim3(256, a.nchains), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t gram_pairs_launch(const double* G, int p, int P, void* G2, cudaStream_t s) {
  gram_pairs_kernel<<<512, 256, 0, s>>>(G, p, P, static_cast<df2*>(G2));
  return cudaGetLastError();
}

}  // namespace hs

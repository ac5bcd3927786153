// Batched X-stream on the fifth-generation tensor cores: K chains that share
// one BF16 design matrix X (Sect. 5 schedule, step (i) latent draw and the
// X^T z of the beta update, for K chains at once).
//
// For a tile of 128 rows of X:
//   pass 1   eta'  = X_tile [B_hi | B_lo]            (128 x 2K, tcgen05, TMEM)
//            eta   = eta'_hi + eta'_lo               (per row and chain)
//            z     ~ TN(eta, 1) truncated by y (Eq. 12, first line), branch-free
//                    inverse CDF on the chain's own Philox counters
//   pass 2   XtZ  += X_tile^T Z_hi + X_tile^T Z_lo   (p x K, tcgen05, TMEM)
// with pass 1 of the next tile issued before pass 2 of this one (eta has two
// TMEM buffers), so the tensor cores and the loads keep running while the
// epilogue draws z.
// where beta (FP64) is split into two BF16 parts B_hi + B_lo and so is z, so
// that the products carry about 16 significant bits of beta and z; X itself
// is exact in BF16 and the tensor cores accumulate in FP32.
//
// Data movement: X tiles arrive by TMA (box 64 features x 128 rows, 128-byte
// swizzle) in a ring of S stages of 16 KB + the matching B^T chunk: in pass 1
// each stage also receives the 64-feature chunk of B^T (both parts,
// pre-swizzled in global memory, L2-resident) by a bulk copy.  Pass 2 reads the same tile again, which the
// 129 MB L2 still holds, so HBM sees X once per sweep.  Each CTA owns a
// contiguous range of row tiles and keeps its X^T Z partial in TMEM; at the
// end it writes the partial (p x KC, FP32) and a second kernel sums the
// partials in a fixed order in FP64.
//
// Launch shape: KC chain columns per tile (32, or 16 for K <= 16: the narrow
// form, half the B^T and Z^T traffic through shared memory and half the TMEM
// columns per feature group, so p up to 3584 fits), and S ring stages (4, 6
// or 8); a tuner picks them (and the grid) per workload.
//
// Warp roles (128 + 32 KC / 2 threads): warp 0 lane 0 issues TMA, warp 1
// lane 0 issues tcgen05.mma, warp 2 owns the TMEM allocation, warps 4.. read
// eta, draw z and write Z^T: warp w serves TMEM lane quadrant w % 4 (thread =
// tile row) and chains 8 (w - 4) / 4 .. +7 (several warps per SM
// sub-partition hide the latency of the draw's dependent arithmetic).  Every wait is
// bounded (2 s); a wait that runs out sets the timeout bit and all roles wind
// down through a shared abort flag.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>

#include "hs_common.cuh"
#include "hs_internal.h"

namespace hs {
namespace {

constexpr int kTR = 128;         // rows per tile (MMA M of pass 1; K of pass 2)
constexpr int kCF = 64;          // features per chunk (one 128-byte swizzle row)
constexpr uint32_t kXChunkBytes = kTR * kCF * 2;      // 16 KB: 128 rows x 64 features of X
constexpr int kEpiChains = 8;                         // chains per epilogue warp (8-column TMEM loads)

// The launch shape: KC chain columns (padded; K <= KC), S ring stages (even:
// pass 2 takes them in pairs).
template <int KC, int S>
struct XKShape {
  static_assert(KC == 16 || KC == 32, "chain columns");
  static_assert(S >= 4 && S % 2 == 0, "ring stages");
  static constexpr int kKc = KC;
  static constexpr int kStages = S;
  static constexpr uint32_t kBChunkBytes = 2 * KC * kCF * 2;      // 2 KC rows (hi chains, lo chains) x 128 B of B^T
  static constexpr uint32_t kStageBytes = kXChunkBytes + kBChunkBytes;  // X chunk, then (pass 1) its B^T chunk
  static constexpr uint32_t kZBlock = KC * 128;                  // KC chains x 64 rows x 2 B
  static constexpr int kEpiWarps = 4 * (KC / kEpiChains);
  static constexpr int kEpiThreads = 32 * kEpiWarps;
  static constexpr int kThreads = 128 + kEpiThreads;  // 4 role warps + the epilogue warps
  static constexpr size_t kSmem = 1024 + (size_t)S * kStageBytes + 4 * (size_t)kZBlock;
};
__host__ __device__ constexpr uint32_t bchunk_bytes(int kc) { return 2u * kc * kCF * 2; }

// ---- tcgen05 helpers (shared-memory descriptors, 128-byte swizzle) ---------
// Descriptor: start address >> 4 in bits 0-13, leading byte offset >> 4 in
// 16-29, stride byte offset >> 4 in 32-45, version 1 in 46-47, layout in
// 61-63 (2 = 128-byte swizzle).  K-major operand: 8-row groups of 128-byte
// rows SBO apart.  MN-major operand: 64-element atoms LBO apart along M/N and
// 8-row K groups SBO apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46) | (2ull << 61);
}
// Instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A and B bf16
// (bits 7-9, 10-12 = 1), A/B major (bits 15, 16; 1 = MN-major), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on an mbarrier once every tcgen05.mma issued so far has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 32 consecutive columns of TMEM into 32 registers per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
// 32 lanes x 16 consecutive columns of TMEM into 16 registers per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// 32 lanes x 8 consecutive columns of TMEM into 8 registers per thread.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
// FP32 uniform pair from two Philox words: u = (2m + 1) 2^-53 and 1 - u with
// m = (hi << 20) | (lo >> 12).  With m = hi 2^20 + l (l < 2^20),
// u = hi 2^-32 + (2l + 1) 2^-53: the second term is exact in FP32 and one FMA
// adds it to the rounded first, so u is within an ulp of (2m + 1) 2^-53
// (exactly rounded when hi < 2^24) using 32-bit conversions only; 1 - u is
// the same with the complemented words (2^52 - 1 - m = ~hi 2^20 + (2^20 - 1 - l)).
__device__ __forceinline__ void unit_pair_f(uint32_t hi, uint32_t lo, float& u, float& uc) {
  const uint32_t l = lo >> 12;
  u = fmaf(__uint2float_rn(2u * l + 1u), 0x1p-53f, __uint2float_rn(hi) * 0x1p-32f);
  uc = fmaf(__uint2float_rn(2u * (0xFFFFFu - l) + 1u), 0x1p-53f, __uint2float_rn(~hi) * 0x1p-32f);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 2-D TMA load of one box into shared memory, completing on an mbarrier, with
// an L2 eviction-priority policy (createpolicy).
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Byte offset of element (row n, column k < 64) in a 128-byte-swizzled K-major
// block whose 8-row groups are 1024 bytes apart (the layout TMA writes).
__host__ __device__ __forceinline__ uint32_t sw128_off(int n, int k) {
  const uint32_t byte = (uint32_t)k * 2;
  return (uint32_t)(n >> 3) * 1024u + (uint32_t)(n & 7) * 128u + ((((byte >> 4) ^ (uint32_t)(n & 7)) & 7u) << 4) +
         (byte & 15u);
}

// ---- the latent draw of the batched form --------------------------------------
// Phi^{-1}(p) for 0 < p <= 1/2: Wichura (1988), Applied Statistics 37,
// Algorithm AS 241, PPND7 (rational approximations, about 7 significant
// digits; 1.2e-7 mixed relative error against scipy's ndtri for p down to
// 1e-37).  Both arms are evaluated and selected, so lanes do not diverge.
__device__ __forceinline__ float ppnd7_lower(float p) {
  const float q = p - 0.5f;
  const float r1 = 0.180625f - q * q;
  const float num1 = fmaf(fmaf(fmaf(59.109374720f, r1, 159.29113202f), r1, 50.434271938f), r1, 3.3871327179f);
  const float den1 = fmaf(fmaf(fmaf(67.187563600f, r1, 78.757757664f), r1, 17.895169469f), r1, 1.0f);
  const float central = q * __fdividef(num1, den1);
  const float r = sqrtf(-__logf(p));
  const bool near = r <= 5.0f;
  const float rr = near ? r - 1.6f : r - 5.0f;
  const float c3 = near ? 0.17023821103f : 0.017337203997f, c2 = near ? 1.3067284816f : 0.42868294337f;
  const float c1 = near ? 2.7568153900f : 3.0812263860f, c0 = near ? 1.4234372777f : 6.6579051150f;
  const float d2 = near ? 0.12021132975f : 0.012258202635f, d1 = near ? 0.73700164250f : 0.24197894225f;
  const float tail = -__fdividef(fmaf(fmaf(fmaf(c3, rr, c2), rr, c1), rr, c0), fmaf(fmaf(d2, rr, d1), rr, 1.0f));
  return fabsf(q) <= 0.425f ? central : tail;
}
// z+ = ms - Phi^{-1}(u Phi(ms)) (Eq. 12, first line; the main arm of
// tn_main): Phi(ms) and Phi(-ms) come from one erfc of |ms| (the smaller is
// the tail, the other 1 - tail), and Phi^{-1} is taken on the smaller of q
// and 1 - q = (1 - u) + u Phi(-ms).
__device__ __forceinline__ float tn_main_k(float ms, float u, float uc) {
  const float t = 0.5f * erfcf(fabsf(ms) * 0.70710678118654752f);  // Phi(-|ms|)
  const float pm = ms < 0.0f ? t : 1.0f - t;
  const float pc = ms < 0.0f ? 1.0f - t : t;
  const float q = u * pm;
  const float qc = fmaf(u, pc, uc);
  const bool lower = q <= qc;
  const float w0 = ppnd7_lower(lower ? q : qc);
  return ms - (lower ? w0 : -w0);
}

template <int S>
struct XKShared {
  uint64_t full[S], empty[S];
  uint64_t eta_full[2], eta_empty[2], z_ready, zt_empty, acc_done;
  uint32_t tmem;
  int abort;
};

// Bounded wait; on timeout records the error and raises the CTA's abort flag.
__device__ __forceinline__ bool xk_wait(uint64_t* bar, uint32_t parity, int* abort, int* err) {
  if (mbar_test(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_test(bar, parity)) {
    if (*(volatile int*)abort) return false;
    if (global_ns() - t0 > 2000000000ull) {
      set_error(err, kErrTimeout);
      *(volatile int*)abort = 1;
      return false;
    }
  }
  return true;
}

// TMEM columns of a CTA: two eta' buffers of 2 KC columns, then KC per
// 128-feature group, rounded up to a power of two (at least 32).
__host__ __device__ constexpr uint32_t xk_tmem_cols(int kc, int nch) {
  const uint32_t need = (uint32_t)(4 * kc + kc * (nch / 2));
  uint32_t c = 32;
  while (c < need) c <<= 1;
  return c;
}

template <int KC, int S, int MINB>
__global__ void __launch_bounds__(XKShape<KC, S>::kThreads, MINB)
    xstream_k_kernel(const __grid_constant__ CUtensorMap xmap, XKArgs a) {
  using Sh = XKShape<KC, S>;
  constexpr int kXStages = S;
  constexpr uint32_t kStageBytes = Sh::kStageBytes;
  constexpr uint32_t kBChunkBytes = Sh::kBChunkBytes;
  constexpr uint32_t kZBlock = Sh::kZBlock;
  constexpr int kEpiWarps = Sh::kEpiWarps;
  constexpr int kEpiThreads = Sh::kEpiThreads;
  extern __shared__ unsigned char dyn[];
  __shared__ XKShared<S> sh;
  int* const abort_flag = &sh.abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* base = dyn + ((1024u - (smem_u32(dyn) & 1023u)) & 1023u);  // 1024-byte aligned
  unsigned char* sX = base;                                   // S stages
  unsigned char* sZ = sX + (size_t)kXStages * kStageBytes;    // [hi/lo][rows 0-63 | 64-127] x KC x 128 B
  const int64_t ntiles = (a.N + kTR - 1) / kTR;
  const int64_t t0 = ntiles * blockIdx.x / gridDim.x;
  const int64_t t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
  const int nch = a.nch;       // even
  const int ngrp = nch / 2;    // 128-feature groups of pass 2

  if (tid == 0) {
    if (a.sm_mark) {
      // tell the factorization, running beside this kernel, which SMs are busy here
      unsigned int smid;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
      if (smid < (unsigned)kSmMarks) a.sm_mark[smid] = (unsigned int)(*a.k_dev + 1);
    }
    for (int s = 0; s < kXStages; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.eta_full[b], 1);
      mbar_init(&sh.eta_empty[b], kEpiThreads);
    }
    mbar_init(&sh.z_ready, kEpiThreads);
    mbar_init(&sh.zt_empty, 1);
    mbar_init(&sh.acc_done, 1);
    sh.abort = 0;
    fence_mbar_init();
  }
  const uint32_t tcols = xk_tmem_cols(KC, nch);
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;
  const uint32_t tm_eta = tmem;             // columns [2 KC b, 2 KC (b + 1)): eta' of buffer b (hi chains, lo chains)
  const uint32_t tm_xtz = tmem + 4 * KC;    // columns [4 KC + KC g, +KC): X^T Z of feature group g

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    // load order (as the MMA issuer consumes): pass 1 of t0; then for each
    // tile t, pass 1 of t + 1 and pass 2 of t
    uint32_t q = 0;
    // pass 1 keeps the tile in L2 for pass 2 (which reads it for the last time)
    const uint64_t pol_keep = l2_policy_evict_last(), pol_done = l2_policy_evict_first();
    auto load_pass = [&](int64_t t, bool with_b) -> bool {
      for (int c = 0; c < nch; ++c, ++q) {
        const int s = q % kXStages;
        if (!xk_wait(&sh.empty[s], ((q / kXStages) & 1) ^ 1, abort_flag, a.err)) return false;
        unsigned char* st = sX + (size_t)s * kStageBytes;
        mbar_arrive_expect_tx(&sh.full[s], with_b ? kStageBytes : kXChunkBytes);
        tma_load_2d(st, &xmap, c * kCF, (int)(t * kTR), &sh.full[s], with_b ? pol_keep : pol_done);
        if (with_b)
          bulk_g2s(st + kXChunkBytes, static_cast<const unsigned char*>(a.bsw) + (size_t)c * kBChunkBytes,
                   kBChunkBytes, &sh.full[s]);
      }
      return true;
    };
    bool okp = t0 < t1 ? load_pass(t0, true) : true;
    for (int64_t t = t0; t < t1 && okp; ++t) {
      if (t + 1 < t1 && !(okp = load_pass(t + 1, true))) break;
      okp = load_pass(t, false);
    }
    // drain: every issued load must land before the CTA may exit
    const uint32_t nd = q < (uint32_t)kXStages ? q : (uint32_t)kXStages;
    for (uint32_t d = 1; d <= nd; ++d) {
      const uint32_t qq = q - d;
      mbar_wait(&sh.full[qq % kXStages], (qq / kXStages) & 1, 2000000000ull);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    const uint32_t id_eta = idesc_bf16(kTR, 2 * KC, 0, 0);   // M 128 rows, N 2 KC (hi, lo), both K-major
    const uint32_t id_xtz = idesc_bf16(128, KC, 1, 0);       // M 128 features (MN-major A), N KC chains
    // Descriptors are built once: moving a descriptor by b bytes adds b >> 4 to
    // its address field (shared addresses stay below 256 KB, so it cannot carry).
    // This warp shares its sub-partition with four epilogue warps, so every
    // instruction it saves shortens the issue loop.
    const uint64_t dX0 = sw128_desc(smem_u32(sX), 16, 1024);                  // pass 1: X chunk of stage 0
    const uint64_t dB0 = sw128_desc(smem_u32(sX) + kXChunkBytes, 16, 1024);   // pass 1: B^T chunk of stage 0
    const uint64_t dA0 = sw128_desc(smem_u32(sX), kStageBytes, 1024);         // pass 2: X pair from stage 0
    uint64_t dZ[2][8];                                                         // pass 2: Z part hl, rows 16 kk ..
#pragma unroll
    for (int hl = 0; hl < 2; ++hl)
#pragma unroll
      for (int kk = 0; kk < 8; ++kk)
        dZ[hl][kk] = sw128_desc(smem_u32(sZ + (size_t)(hl * 2 + kk / 4) * kZBlock) + (kk % 4) * 32, 16, 1024);
    constexpr uint64_t kStageStep = kStageBytes >> 4;
    bool ok = true;
    uint32_t q = 0;
    // pass 1 of tile number n (within this CTA) into eta buffer n % 2
    auto pass1 = [&](int n) -> bool {
      const int b = n & 1;
      if (!xk_wait(&sh.eta_empty[b], ((n >> 1) & 1) ^ 1, abort_flag, a.err)) return false;  // the epilogue read it
      tc_fence_after();
      for (int c = 0; c < nch; ++c, ++q) {
        const int s = q % kXStages;
        if (!xk_wait(&sh.full[s], (q / kXStages) & 1, abort_flag, a.err)) return false;
        tc_fence_after();
        const uint64_t dx = dX0 + kStageStep * s, db = dB0 + kStageStep * s;
#pragma unroll
        for (int kk = 0; kk < kCF / 16; ++kk)
          mma_bf16(tm_eta + 2 * KC * b, dx + 2 * kk, db + 2 * kk, id_eta, (c > 0 || kk > 0) ? 1 : 0);
        mma_commit(&sh.empty[s]);
      }
      mma_commit(&sh.eta_full[b]);
      return true;
    };
    const int ntl = (int)(t1 - t0);
    if (ok && ntl > 0) ok = pass1(0);
    for (int it = 0; it < ntl && ok; ++it) {
      // pass 1 of the next tile runs while the epilogue draws z of this one
      if (it + 1 < ntl && !(ok = pass1(it + 1))) break;
      // pass 2: X^T Z once the epilogue has written Z^T of this tile
      if (!(ok = xk_wait(&sh.z_ready, it & 1, abort_flag, a.err))) break;
      tc_fence_after();
      for (int g = 0; g < ngrp && ok; ++g) {
        const int s0 = q % kXStages;  // even: chunks 2g and 2g+1 sit in stages s0, s0+1
        if (!(ok = xk_wait(&sh.full[s0], (q / kXStages) & 1, abort_flag, a.err))) break;
        if (!(ok = xk_wait(&sh.full[s0 + 1], ((q + 1) / kXStages) & 1, abort_flag, a.err))) break;
        tc_fence_after();
        const uint64_t da = dA0 + kStageStep * s0;
        const int acc0 = it > 0 ? 1 : 0;
#pragma unroll
        for (int kk = 0; kk < kTR / 16; ++kk) {
          // rows 16kk.., features of both stages (the second 64-feature atom of A
          // is the next stage's X chunk, kStageBytes further)
          const uint64_t ad = da + 128 * kk;
          mma_bf16(tm_xtz + KC * g, ad, dZ[0][kk], id_xtz, kk > 0 ? 1 : acc0);
          mma_bf16(tm_xtz + KC * g, ad, dZ[1][kk], id_xtz, 1);
        }
        mma_commit(&sh.empty[s0]);
        mma_commit(&sh.empty[s0 + 1]);
        q += 2;
      }
      if (!ok) break;
      mma_commit(&sh.zt_empty);
    }
    mma_commit(&sh.acc_done);
  } else if (warp >= 4) {
    // ---------------- epilogue: z draws and Z^T ----------------
    const int quad = warp & 3, part = (warp - 4) >> 2;  // TMEM lane quadrant; chains kEpiChains part ..
    const int er = 32 * quad + lane;                      // row within the tile = TMEM lane
    const uint32_t lane_off = (uint32_t)(32 * quad) << 16;
    const int m0 = kEpiChains * part;
    const uint32_t sweep = (uint32_t)(*a.k_dev + 1);
    int it = 0;
    // y of this thread's row, one tile ahead (its load latency off the draw's path)
    int y_next = (t0 < t1 && t0 * kTR + er < a.N) ? a.y[t0 * kTR + er] : 1;
    for (int64_t t = t0; t < t1; ++t, ++it) {
      const int eb = it & 1;  // eta buffer of this tile
      const int yi_t = y_next;
      if (t + 1 < t1 && (t + 1) * kTR + er < a.N) y_next = a.y[(t + 1) * kTR + er];
      if (!xk_wait(&sh.eta_full[eb], (it >> 1) & 1, abort_flag, a.err)) break;
      tc_fence_after();
      uint32_t hi[kEpiChains], lo[kEpiChains];
      tmem_ld8(tm_eta + 2 * KC * eb + lane_off + m0, hi);
      tmem_ld8(tm_eta + 2 * KC * eb + lane_off + KC + m0, lo);
      tmem_ld_wait();
      tc_fence_before();
      mbar_arrive(&sh.eta_empty[eb]);
      const int64_t i = t * kTR + er;
      const bool active = i < a.N;
      const int yi = active ? yi_t : 1;
      // Z^T (both parts) for pass 2, once pass 2 of the previous tile is done with it
      if (!xk_wait(&sh.zt_empty, (it & 1) ^ 1, abort_flag, a.err)) break;
      const int katom = er >> 6, kr = er & 63;
      if (m0 >= a.K) {
        // every chain of this warp is padding (K < 32): zeros, no draws (the branch is warp-uniform)
#pragma unroll
        for (int mm = 0; mm < kEpiChains; ++mm) {
          const uint32_t o = sw128_off(m0 + mm, kr);
          *reinterpret_cast<uint16_t*>(sZ + (size_t)(0 * 2 + katom) * kZBlock + o) = 0;
          *reinterpret_cast<uint16_t*>(sZ + (size_t)(1 * 2 + katom) * kZBlock + o) = 0;
        }
      } else {
#pragma unroll
      for (int mm = 0; mm < kEpiChains; ++mm) {
        const int m = m0 + mm;
        const float eta = __uint_as_float(hi[mm]) + __uint_as_float(lo[mm]);
        const bool on = active && m < a.K;
        float u = 0.5f, uc = 0.5f;
        if (on) {
          const Rng r{a.rng.k0, a.rng.k1, a.rng.chain + (uint32_t)m, a.rng.problem};
          const uint4 wd = r.words((uint32_t)i, sweep, kPurZ);
          unit_pair_f(wd.x, wd.y, u, uc);
        }
        const float ms = on ? (yi ? eta : -eta) : 0.0f;
        float zp = tn_main_k(ms, u, uc);
        const bool tail = on && ms < TnMath<float>::kTail;
        if (tail) zp = tn_tail<float>(ms, u, uc);
        zp = zp > TnMath<float>::tiny() ? zp : TnMath<float>::tiny();
        float zz = on ? (yi ? zp : -zp) : 0.0f;
        if (on && !isfinite(zz)) {
          set_error(a.err, kErrNonFinite);
          zz = 0.0f;
        }
        if (on && a.z_out) a.z_out[(size_t)m * a.N + i] = (double)zz;
        const __nv_bfloat16 zh = __float2bfloat16_rn(zz);
        const __nv_bfloat16 zl = __float2bfloat16_rn(zz - __bfloat162float(zh));
        const uint32_t o = sw128_off(m, kr);
        *reinterpret_cast<__nv_bfloat16*>(sZ + (size_t)(0 * 2 + katom) * kZBlock + o) = zh;
        *reinterpret_cast<__nv_bfloat16*>(sZ + (size_t)(1 * 2 + katom) * kZBlock + o) = zl;
      }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core reads
      mbar_arrive(&sh.z_ready);
    }
    // the CTA's X^T Z partial: row = feature 128 g + er, KC chains; groups split between the parts
    if (xk_wait(&sh.acc_done, 0, abort_flag, a.err)) {
      tc_fence_after();
      for (int g = part; g < ngrp; g += kEpiWarps / 4) {
        uint32_t r[KC];
        if constexpr (KC == 32) tmem_ld32(tm_xtz + KC * g + lane_off, r);
        else tmem_ld16(tm_xtz + KC * g + lane_off, r);
        tmem_ld_wait();
        const int f = 128 * g + er;
        float* out = a.partials + ((size_t)blockIdx.x * a.fpad + f) * KC;
#pragma unroll
        for (int m = 0; m < KC; m += 4)
          *reinterpret_cast<float4*>(out + m) = make_float4(__uint_as_float(r[m]), __uint_as_float(r[m + 1]),
                                                            __uint_as_float(r[m + 2]), __uint_as_float(r[m + 3]));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
  }
}

// ---- the split form: pass 1 and pass 2 as two kernels ------------------------
// Pass 1 (xk_eta_kernel): per 128-row tile eta' = X [B_hi | B_lo] on the
// tensor cores, the z draws as in the fused kernel, and Z^T (both BF16 parts,
// in the swizzled layout pass 2 reads) stored to global memory by one bulk
// copy per tile.  Pass 2 (xk_xtz_kernel): X^T Z_hi + X^T Z_lo over the same
// tiles into TMEM, which then holds only the feature groups (KC columns
// each).  For FP8 X each 64-feature chunk lands by TMA as codes (8 KB, 64-byte
// rows) and four converter warps rewrite it as BF16 (exact: e4m3 values have
// 4 significant bits) in the 128-byte-swizzled layout before the MMA reads it;
// the column scales sit in B^T (pass 1) and in the reduce (pass 2).
constexpr uint32_t kFp8PairBytes = kTR * 2 * kCF;  // 16 KB: 128 rows x 128 codes (two chunks)

template <int KC, int F8>
struct XKSplit {
  static_assert(KC == 16 || KC == 32, "chain columns");
  static constexpr int kStages = KC == 16 ? 6 : 4;  // BF16 X: one ring (even: pass 2 takes stages in pairs)
  static constexpr uint32_t kBChunkBytes = 2 * KC * kCF * 2;
  static constexpr uint32_t kZBlock = KC * 128;
  static constexpr uint32_t kZTile = 4 * kZBlock;  // [hi/lo][rows 0-63 | 64-127]
  static constexpr uint32_t kStageEta = kXChunkBytes + kBChunkBytes;
  static constexpr uint32_t kStageXtz = kXChunkBytes;
  // FP8 X: a ring of code stages, each two chunks (128 features: TMA boxes
  // of 128-byte rows; pass 1 also puts the two B^T chunks there), and a ring
  // of BF16 stages (even: a code stage fills two) the converter warps fill
  static constexpr uint32_t kCodeEta = kFp8PairBytes + 2 * kBChunkBytes;
  static constexpr uint32_t kCodeXtz = kFp8PairBytes;
  static constexpr int kCodeStagesEta = KC == 16 ? 6 : 4;
  static constexpr int kBfStagesEta = 4;
  static constexpr int kCodeStagesXtz = KC == 16 ? 7 : 8;
  static constexpr int kBfStagesXtz = KC == 16 ? 6 : 4;
  static constexpr int kEpiWarps = 4 * (KC / kEpiChains);
  static constexpr int kCvtWarps = F8 ? 4 : 0;
  static constexpr int kThreads = 128 + 32 * (kEpiWarps + kCvtWarps);
  static constexpr size_t kRingEta = F8 ? (size_t)kCodeStagesEta * kCodeEta + (size_t)kBfStagesEta * kXChunkBytes
                                        : (size_t)kStages * kStageEta;
  static constexpr size_t kRingXtz = F8 ? (size_t)kCodeStagesXtz * kCodeXtz + (size_t)kBfStagesXtz * kXChunkBytes
                                        : (size_t)kStages * kStageXtz;
  static constexpr size_t kSmemEta = 1024 + kRingEta + 2 * (size_t)kZTile;
  static constexpr size_t kSmemXtz = 1024 + kRingXtz + 2 * (size_t)kZTile;
  static_assert(kSmemEta <= 227 * 1024 && kSmemXtz <= 227 * 1024, "stages fit in shared memory");
  static_assert(kStageEta % 1024 == 0 && kCodeEta % 1024 == 0 && kCodeXtz % 1024 == 0,
                "stages keep the 1024-byte swizzle alignment");
};

// FP8 e4m3 codes of two chunks (128 rows of 128 bytes) -> BF16 in the
// 128-byte-swizzled K-major layout of the MMA, features 0-63 into dst0 and
// 64-127 into dst1.  Thread t (0..127) takes the 16-byte granules t + 128 j
// (row G / 8, features 16 (G % 8) ..), so eight consecutive lanes read one
// 128-byte row.  Each granule gives two 16-byte outputs; the lanes writing
// dst1 store theirs in the opposite order, so the eight lanes of a quarter
// warp hit eight different swizzled granules (dst0 and dst1 are 16 KB apart,
// on the same banks) and no store conflicts.
__device__ __forceinline__ void cvt_pair_fp8(const unsigned char* src, unsigned char* dst0, unsigned char* dst1,
                                             int t) {
#pragma unroll
  for (int jg = 0; jg < 8; ++jg) {
    const int G = t + 128 * jg;
    const int row = G >> 3, c16 = G & 7;
    unsigned char* dst = c16 < 4 ? dst0 : dst1;
    const int f0 = 16 * (c16 & 3);
    const uint4 v = *reinterpret_cast<const uint4*>(src + (size_t)G * 16);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t o[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const __nv_fp8x2_storage_t pr = (__nv_fp8x2_storage_t)((w[i] >> (16 * h)) & 0xFFFFu);
        const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(pr, __NV_E4M3);
        const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&hr));
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(f.x, f.y);
        o[2 * i + h] = *reinterpret_cast<const uint32_t*>(&b2);
      }
    }
    const uint4 lo = make_uint4(o[0], o[1], o[2], o[3]), hi = make_uint4(o[4], o[5], o[6], o[7]);
    const bool up = c16 >= 4;
    *reinterpret_cast<uint4*>(dst + sw128_off(row, up ? f0 + 8 : f0)) = up ? hi : lo;
    *reinterpret_cast<uint4*>(dst + sw128_off(row, up ? f0 : f0 + 8)) = up ? lo : hi;
  }
}

// Shared-memory to global bulk copy of one tile's Z^T (bulk-group completion).
__device__ __forceinline__ void bulk_s2g(void* gdst, const void* ssrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(ssrc)),
               "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

template <int KC, int F8>
__global__ void __launch_bounds__(XKSplit<KC, F8>::kThreads, 1)
    xk_eta_kernel(const __grid_constant__ CUtensorMap xmap, XKArgs a) {
  using Sp = XKSplit<KC, F8>;
  // BF16 X: one ring of S stages (X chunk, B^T chunk).  FP8 X: CS code
  // stages (codes, B^T chunk) and BS BF16 stages.
  constexpr int S = Sp::kStages, CS = Sp::kCodeStagesEta, BS = Sp::kBfStagesEta;
  constexpr int NF = F8 ? CS : S, NB = F8 ? BS : 1;  // barrier array sizes
  constexpr uint32_t kStage = Sp::kStageEta, kCode = Sp::kCodeEta, kBChunkBytes = Sp::kBChunkBytes,
                     kZBlock = Sp::kZBlock, kZTile = Sp::kZTile;
  constexpr int kEpiWarps = Sp::kEpiWarps, kEpiThreads = 32 * kEpiWarps;
  extern __shared__ unsigned char dyn[];
  __shared__ uint64_t full[NF], empty[NF], bfull[NB], bempty[NB], eta_full[2], eta_empty[2], z_ready[2],
      zt_empty[2], mma_done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_v;
  int* const abort_flag = &abort_v;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* base = dyn + ((1024u - (smem_u32(dyn) & 1023u)) & 1023u);
  unsigned char* bf = base + (size_t)CS * kCode;  // FP8: the BF16 ring after the code ring
  unsigned char* sZ = base + Sp::kRingEta;        // two tiles of Z^T
  const int64_t ntiles = (a.N + kTR - 1) / kTR;
  const int64_t t0 = ntiles * blockIdx.x / gridDim.x;
  const int64_t t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
  const int nch = a.nch;
  const uint32_t nq = (uint32_t)((t1 - t0) * nch);  // chunks this CTA loads

  if (tid == 0) {
    if (a.sm_mark) {
      unsigned int smid;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
      if (smid < (unsigned)kSmMarks) a.sm_mark[smid] = (unsigned int)(*a.k_dev + 1);
    }
    for (int s = 0; s < NF; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < NB; ++s) {
      mbar_init(&bfull[s], 128);
      mbar_init(&bempty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&eta_full[b], 1);
      mbar_init(&eta_empty[b], kEpiThreads);
      mbar_init(&z_ready[b], kEpiThreads);
      mbar_init(&zt_empty[b], 1);
    }
    mbar_init(&mma_done, 1);
    abort_v = 0;
    fence_mbar_init();
  }
  constexpr uint32_t tcols = 4 * KC < 32 ? 32 : 4 * KC;  // two eta' buffers of 2 KC columns
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm_eta = tmem_base;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer: X chunk and its B^T chunk (FP8: two of each) ----------------
    const uint64_t pol = l2_policy_evict_first();  // X is read once by this kernel
    uint32_t q = 0;  // stage fills
    bool ok = true;
    for (int64_t t = t0; t < t1 && ok; ++t) {
      for (int c = 0; c < nch; c += F8 ? 2 : 1, ++q) {
        const int s = q % NF;
        if (!(ok = xk_wait(&empty[s], ((q / NF) & 1) ^ 1, abort_flag, a.err))) break;
        const unsigned char* bsw = static_cast<const unsigned char*>(a.bsw) + (size_t)c * kBChunkBytes;
        if constexpr (F8) {
          unsigned char* st = base + (size_t)s * kCode;
          mbar_arrive_expect_tx(&full[s], kFp8PairBytes + 2 * kBChunkBytes);
          tma_load_2d(st, &xmap, c * kCF, (int)(t * kTR), &full[s], pol);  // 128 codes x 128 rows
          bulk_g2s(st + kFp8PairBytes, bsw, 2 * kBChunkBytes, &full[s]);
        } else {
          unsigned char* st = base + (size_t)s * kStage;
          mbar_arrive_expect_tx(&full[s], kXChunkBytes + kBChunkBytes);
          tma_load_2d(st, &xmap, c * kCF, (int)(t * kTR), &full[s], pol);
          bulk_g2s(st + kXChunkBytes, bsw, kBChunkBytes, &full[s]);
        }
      }
    }
    const uint32_t nd = q < (uint32_t)NF ? q : (uint32_t)NF;
    for (uint32_t d = 1; d <= nd; ++d) {
      const uint32_t qq = q - d;
      mbar_wait(&full[qq % NF], (qq / NF) & 1, 2000000000ull);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer: pass 1 ----------------
    const uint32_t id_eta = idesc_bf16(kTR, 2 * KC, 0, 0);
    uint32_t q = 0;  // chunks
    bool ok = true;
    for (int64_t n = 0; t0 + n < t1 && ok; ++n) {
      const int b = (int)(n & 1);
      if (!(ok = xk_wait(&eta_empty[b], ((n >> 1) & 1) ^ 1, abort_flag, a.err))) break;
      tc_fence_after();
      for (int c = 0; c < nch; ++c, ++q) {
        uint32_t xa, ba;  // shared addresses of the BF16 X chunk and of the B^T chunk
        if constexpr (F8) {
          const int sb = q % NB;
          if (!(ok = xk_wait(&bfull[sb], (q / NB) & 1, abort_flag, a.err))) break;
          xa = smem_u32(bf) + (uint32_t)sb * kXChunkBytes;
          ba = smem_u32(base) + (uint32_t)((q / 2) % NF) * kCode + kFp8PairBytes + (q & 1) * kBChunkBytes;
        } else {
          if (!(ok = xk_wait(&full[q % NF], (q / NF) & 1, abort_flag, a.err))) break;
          xa = smem_u32(base) + (uint32_t)(q % NF) * kStage;
          ba = xa + kXChunkBytes;
        }
        tc_fence_after();
        const uint64_t dx = sw128_desc(xa, 16, 1024), db = sw128_desc(ba, 16, 1024);
#pragma unroll
        for (int kk = 0; kk < kCF / 16; ++kk)
          mma_bf16(tm_eta + 2 * KC * b, dx + 2 * kk, db + 2 * kk, id_eta, (c > 0 || kk > 0) ? 1 : 0);
        if constexpr (F8) {
          mma_commit(&bempty[q % NB]);
          if (q & 1) mma_commit(&empty[(q / 2) % NF]);  // both chunks of the code stage read
        } else {
          mma_commit(&empty[q % NF]);
        }
      }
      if (!ok) break;
      mma_commit(&eta_full[b]);
    }
    mma_commit(&mma_done);
    mbar_wait(&mma_done, 0, 2000000000ull);  // nothing in flight when the CTA leaves
  } else if (warp == 3 && lane == 0) {
    // ---------------- Z^T storer: one bulk copy per tile ----------------
    for (int64_t n = 0; t0 + n < t1; ++n) {
      const int zb = (int)(n & 1);
      if (!xk_wait(&z_ready[zb], (n >> 1) & 1, abort_flag, a.err)) break;
      bulk_s2g(static_cast<unsigned char*>(a.zt) + (size_t)(t0 + n) * kZTile, sZ + (size_t)zb * kZTile, kZTile);
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // the source may be rewritten
      mbar_arrive(&zt_empty[zb]);
    }
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // the writes are done before the CTA leaves
  } else if (F8 && warp >= 4 + kEpiWarps) {
    // ---------------- converter warps: codes -> BF16 ----------------
    const int ct = tid - 32 * (4 + kEpiWarps);
    for (uint32_t r = 0; r < nq / 2; ++r) {  // code stage r: chunks 2r, 2r + 1
      const int s = r % NF, sb = (2 * r) % NB;   // NB even: the pair is sb, sb + 1
      if (!xk_wait(&full[s], (r / NF) & 1, abort_flag, a.err)) break;
      if (!xk_wait(&bempty[sb], (((2 * r) / NB) & 1) ^ 1, abort_flag, a.err)) break;
      if (!xk_wait(&bempty[sb + 1], (((2 * r + 1) / NB) & 1) ^ 1, abort_flag, a.err)) break;
      cvt_pair_fp8(base + (size_t)s * kCode, bf + (size_t)sb * kXChunkBytes, bf + (size_t)(sb + 1) * kXChunkBytes,
                   ct);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core reads
      mbar_arrive(&bfull[sb]);
      mbar_arrive(&bfull[sb + 1]);
    }
  } else if (warp >= 4 && warp < 4 + kEpiWarps) {
    // ---------------- epilogue: z draws and Z^T, as in the fused kernel ----------------
    const int quad = warp & 3, part = (warp - 4) >> 2;
    const int er = 32 * quad + lane;
    const uint32_t lane_off = (uint32_t)(32 * quad) << 16;
    const int m0 = kEpiChains * part;
    const uint32_t sweep = (uint32_t)(*a.k_dev + 1);
    int it = 0;
    int y_next = (t0 < t1 && t0 * kTR + er < a.N) ? a.y[t0 * kTR + er] : 1;
    for (int64_t t = t0; t < t1; ++t, ++it) {
      const int eb = it & 1;
      const int yi_t = y_next;
      if (t + 1 < t1 && (t + 1) * kTR + er < a.N) y_next = a.y[(t + 1) * kTR + er];
      if (!xk_wait(&eta_full[eb], (it >> 1) & 1, abort_flag, a.err)) break;
      tc_fence_after();
      uint32_t hi[kEpiChains], lo[kEpiChains];
      tmem_ld8(tm_eta + 2 * KC * eb + lane_off + m0, hi);
      tmem_ld8(tm_eta + 2 * KC * eb + lane_off + KC + m0, lo);
      tmem_ld_wait();
      tc_fence_before();
      mbar_arrive(&eta_empty[eb]);
      const int64_t i = t * kTR + er;
      const bool active = i < a.N;
      const int yi = active ? yi_t : 1;
      if (!xk_wait(&zt_empty[eb], ((it >> 1) & 1) ^ 1, abort_flag, a.err)) break;
      unsigned char* zt = sZ + (size_t)eb * kZTile;
      const int katom = er >> 6, kr = er & 63;
      if (m0 >= a.K) {
#pragma unroll
        for (int mm = 0; mm < kEpiChains; ++mm) {
          const uint32_t o = sw128_off(m0 + mm, kr);
          *reinterpret_cast<uint16_t*>(zt + (size_t)(0 * 2 + katom) * kZBlock + o) = 0;
          *reinterpret_cast<uint16_t*>(zt + (size_t)(1 * 2 + katom) * kZBlock + o) = 0;
        }
      } else {
#pragma unroll
        for (int mm = 0; mm < kEpiChains; ++mm) {
          const int m = m0 + mm;
          const float eta = __uint_as_float(hi[mm]) + __uint_as_float(lo[mm]);
          const bool on = active && m < a.K;
          float u = 0.5f, uc = 0.5f;
          if (on) {
            const Rng r{a.rng.k0, a.rng.k1, a.rng.chain + (uint32_t)m, a.rng.problem};
            const uint4 wd = r.words((uint32_t)i, sweep, kPurZ);
            unit_pair_f(wd.x, wd.y, u, uc);
          }
          const float ms = on ? (yi ? eta : -eta) : 0.0f;
          float zp = tn_main_k(ms, u, uc);
          const bool tail = on && ms < TnMath<float>::kTail;
          if (tail) zp = tn_tail<float>(ms, u, uc);
          zp = zp > TnMath<float>::tiny() ? zp : TnMath<float>::tiny();
          float zz = on ? (yi ? zp : -zp) : 0.0f;
          if (on && !isfinite(zz)) {
            set_error(a.err, kErrNonFinite);
            zz = 0.0f;
          }
          if (on && a.z_out) a.z_out[(size_t)m * a.N + i] = (double)zz;
          const __nv_bfloat16 zh = __float2bfloat16_rn(zz);
          const __nv_bfloat16 zl = __float2bfloat16_rn(zz - __bfloat162float(zh));
          const uint32_t o = sw128_off(m, kr);
          *reinterpret_cast<__nv_bfloat16*>(zt + (size_t)(0 * 2 + katom) * kZBlock + o) = zh;
          *reinterpret_cast<__nv_bfloat16*>(zt + (size_t)(1 * 2 + katom) * kZBlock + o) = zl;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> bulk copy reads
      mbar_arrive(&z_ready[eb]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm_eta), "r"(tcols));
  }
}

template <int KC, int F8>
__global__ void __launch_bounds__(XKSplit<KC, F8>::kThreads, 1)
    xk_xtz_kernel(const __grid_constant__ CUtensorMap xmap, XKArgs a) {
  using Sp = XKSplit<KC, F8>;
  // BF16 X: one ring of S stages (X chunks).  FP8 X: CS code stages and BS
  // BF16 stages (BS even: pass 2 takes BF16 stages in pairs).
  constexpr int S = Sp::kStages, CS = Sp::kCodeStagesXtz, BS = Sp::kBfStagesXtz;
  constexpr int NF = F8 ? CS : S, NB = F8 ? BS : 1;
  constexpr int NP = F8 ? BS : S;  // the ring the MMA reads in pairs
  constexpr uint32_t kStage = Sp::kStageXtz, kCode = Sp::kCodeXtz, kZBlock = Sp::kZBlock, kZTile = Sp::kZTile;
  constexpr int kEpiWarps = Sp::kEpiWarps;
  extern __shared__ unsigned char dyn[];
  __shared__ uint64_t full[NF], empty[NF], bfull[NB], bempty[NB], zfull[2], zempty[2], acc_done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_v;
  int* const abort_flag = &abort_v;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* base = dyn + ((1024u - (smem_u32(dyn) & 1023u)) & 1023u);
  unsigned char* bf = base + (size_t)CS * kCode;  // FP8: the BF16 ring after the code ring
  unsigned char* sZ = base + Sp::kRingXtz;
  const int64_t ntiles = (a.N + kTR - 1) / kTR;
  const int64_t t0 = ntiles * blockIdx.x / gridDim.x;
  const int64_t t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
  const int nch = a.nch;
  const int ngrp = nch / 2;
  const uint32_t nq = (uint32_t)((t1 - t0) * nch);

  if (tid == 0) {
    for (int s = 0; s < NF; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], F8 ? 128 : 1);  // FP8: the converter frees a code stage once it has read it
    }
    for (int s = 0; s < NB; ++s) {
      mbar_init(&bfull[s], 128);
      mbar_init(&bempty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&zfull[b], 1);
      mbar_init(&zempty[b], 1);
    }
    mbar_init(&acc_done, 1);
    abort_v = 0;
    fence_mbar_init();
  }
  uint32_t tcols = 32;
  while (tcols < (uint32_t)(KC * ngrp)) tcols <<= 1;
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm_xtz = tmem_base;  // columns [KC g, KC (g + 1)): X^T Z of feature group g

  if (warp == 0 && lane == 0) {
    // ---------------- producer: the tile's Z^T, then its X chunks ----------------
    const uint64_t pol = l2_policy_evict_first();
    uint32_t q = 0;
    int64_t nz = 0;
    bool ok = true;
    for (int64_t t = t0; t < t1 && ok; ++t, ++nz) {
      const int zb = (int)(nz & 1);
      if (!(ok = xk_wait(&zempty[zb], ((nz >> 1) & 1) ^ 1, abort_flag, a.err))) break;
      mbar_arrive_expect_tx(&zfull[zb], kZTile);
      bulk_g2s(sZ + (size_t)zb * kZTile, static_cast<const unsigned char*>(a.zt) + (size_t)t * kZTile, kZTile,
               &zfull[zb]);
      for (int c = 0; c < nch; c += F8 ? 2 : 1, ++q) {  // FP8: a code stage holds two chunks
        const int s = q % NF;
        if (!(ok = xk_wait(&empty[s], ((q / NF) & 1) ^ 1, abort_flag, a.err))) break;
        mbar_arrive_expect_tx(&full[s], F8 ? kFp8PairBytes : kXChunkBytes);
        tma_load_2d(base + (size_t)s * (F8 ? kCode : kStage), &xmap, c * kCF, (int)(t * kTR), &full[s], pol);
      }
    }
    const uint32_t nd = q < (uint32_t)NF ? q : (uint32_t)NF;
    for (uint32_t d = 1; d <= nd; ++d) {
      const uint32_t qq = q - d;
      mbar_wait(&full[qq % NF], (qq / NF) & 1, 2000000000ull);
    }
    for (int64_t d = nz - 1; d >= 0 && d >= nz - 2; --d) mbar_wait(&zfull[d & 1], (d >> 1) & 1, 2000000000ull);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer: pass 2 ----------------
    const uint32_t id_xtz = idesc_bf16(128, KC, 1, 0);
    // the two 64-feature atoms of A are consecutive stages of the ring read in pairs
    const uint32_t pbase = F8 ? smem_u32(bf) : smem_u32(base);
    constexpr uint32_t pstride = F8 ? kXChunkBytes : kStage;
    const uint64_t dA0 = sw128_desc(pbase, pstride, 1024);
    constexpr uint64_t kStep = pstride >> 4;
    uint32_t q = 0;
    bool ok = true;
    for (int64_t n = 0; t0 + n < t1 && ok; ++n) {
      const int zb = (int)(n & 1);
      if (!(ok = xk_wait(&zfull[zb], (n >> 1) & 1, abort_flag, a.err))) break;
      tc_fence_after();
      const uint32_t zbase = smem_u32(sZ + (size_t)zb * kZTile);
      for (int g = 0; g < ngrp && ok; ++g) {
        const int s0 = q % NP;  // even: chunks 2g and 2g+1 sit in stages s0, s0+1
        uint64_t* const w0 = F8 ? &bfull[s0] : &full[s0];
        uint64_t* const w1 = F8 ? &bfull[s0 + 1] : &full[s0 + 1];
        if (!(ok = xk_wait(w0, (q / NP) & 1, abort_flag, a.err))) break;
        if (!(ok = xk_wait(w1, ((q + 1) / NP) & 1, abort_flag, a.err))) break;
        tc_fence_after();
        const uint64_t da = dA0 + kStep * s0;
        const int acc0 = n > 0 ? 1 : 0;
#pragma unroll
        for (int kk = 0; kk < kTR / 16; ++kk) {
          const uint64_t ad = da + 128 * kk;
          const uint32_t zo = (uint32_t)(kk / 4) * kZBlock + (uint32_t)(kk % 4) * 32;
          mma_bf16(tm_xtz + KC * g, ad, sw128_desc(zbase + zo, 16, 1024), id_xtz, kk > 0 ? 1 : acc0);
          mma_bf16(tm_xtz + KC * g, ad, sw128_desc(zbase + 2 * kZBlock + zo, 16, 1024), id_xtz, 1);
        }
        if constexpr (F8) {
          mma_commit(&bempty[s0]);
          mma_commit(&bempty[s0 + 1]);
        } else {
          mma_commit(&empty[s0]);
          mma_commit(&empty[s0 + 1]);
        }
        q += 2;
      }
      if (!ok) break;
      mma_commit(&zempty[zb]);
    }
    mma_commit(&acc_done);
    mbar_wait(&acc_done, 0, 2000000000ull);  // nothing in flight when the CTA leaves
  } else if (F8 && warp >= 4 + kEpiWarps) {
    // ---------------- converter warps: codes -> BF16 ----------------
    const int ct = tid - 32 * (4 + kEpiWarps);
    for (uint32_t r = 0; r < nq / 2; ++r) {  // code stage r: chunks 2r, 2r + 1
      const int s = r % NF, sb = (2 * r) % NB;   // NB even: the pair is sb, sb + 1
      if (!xk_wait(&full[s], (r / NF) & 1, abort_flag, a.err)) break;
      if (!xk_wait(&bempty[sb], (((2 * r) / NB) & 1) ^ 1, abort_flag, a.err)) break;
      if (!xk_wait(&bempty[sb + 1], (((2 * r + 1) / NB) & 1) ^ 1, abort_flag, a.err)) break;
      cvt_pair_fp8(base + (size_t)s * kCode, bf + (size_t)sb * kXChunkBytes, bf + (size_t)(sb + 1) * kXChunkBytes,
                   ct);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic accesses before async-proxy ones
      mbar_arrive(&empty[s]);  // the codes have been read
      mbar_arrive(&bfull[sb]);
      mbar_arrive(&bfull[sb + 1]);
    }
  } else if (warp >= 4 && warp < 4 + kEpiWarps) {
    // ---------------- the CTA's X^T Z partial ----------------
    const int quad = warp & 3, part = (warp - 4) >> 2;
    const int er = 32 * quad + lane;
    const uint32_t lane_off = (uint32_t)(32 * quad) << 16;
    if (xk_wait(&acc_done, 0, abort_flag, a.err)) {
      tc_fence_after();
      for (int g = part; g < ngrp; g += kEpiWarps / 4) {
        uint32_t r[KC];
        if constexpr (KC == 32) tmem_ld32(tm_xtz + KC * g + lane_off, r);
        else tmem_ld16(tm_xtz + KC * g + lane_off, r);
        tmem_ld_wait();
        const int f = 128 * g + er;
        float* out = a.partials + ((size_t)blockIdx.x * a.fpad + f) * KC;
#pragma unroll
        for (int m = 0; m < KC; m += 4)
          *reinterpret_cast<float4*>(out + m) = make_float4(__uint_as_float(r[m]), __uint_as_float(r[m + 1]),
                                                            __uint_as_float(r[m + 2]), __uint_as_float(r[m + 3]));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm_xtz), "r"(tcols));
  }
}

// B^T in the shared-memory layout of pass 1: chunk c holds features 64c..64c+63
// of 2 KC rows (rows 0..KC-1: BF16 high parts of the K chains' beta (times
// the column scale of FP8 X, so that the codes multiply it), rows
// KC..2KC-1: the low parts beta - hi), 128-byte swizzled.
__global__ void bsw_prep_kernel(const double* __restrict__ beta, int64_t beta_stride, int K, int p, int nch, int kc,
                                const float* __restrict__ colscale, unsigned char* __restrict__ bsw) {
  const int rows = 2 * kc;
  const int64_t n_el = (int64_t)nch * rows * kCF;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / (rows * kCF)), rem = (int)(e % (rows * kCF));
    const int n = rem / kCF, k = rem % kCF;
    const int m = n % kc, f = c * kCF + k;
    float v = 0.0f;
    if (m < K && f < p) {
      const double b = beta[(int64_t)m * beta_stride + f] * (colscale ? (double)colscale[f] : 1.0);
      const __nv_bfloat16 h = __float2bfloat16_rn((float)b);
      v = n < kc ? __bfloat162float(h) : (float)(b - (double)__bfloat162float(h));
    }
    *reinterpret_cast<__nv_bfloat16*>(bsw + (size_t)c * bchunk_bytes(kc) + sw128_off(n, k)) = __float2bfloat16_rn(v);
  }
}

// X^T z of chain m, feature j: fixed-order FP64 sum over the CTAs' partials.
// One block per feature, 256 threads = KC chains x (256 / KC) groups: thread
// (g, m) adds the partial rows of CTAs g, g + G, g + 2G, ... (each warp reads
// whole lines of consecutive chains) in four interleaved accumulators, then
// the G group sums are added in group order, so the result is the same every
// sweep.
template <int KC>
__global__ void __launch_bounds__(256) reduce_k_kernel(const float* __restrict__ part, int grid, int fpad, int p, int K,
                                                       const float* __restrict__ colscale, double* __restrict__ xtz,
                                                       int64_t xtz_stride) {
  constexpr int G = 256 / KC;
  __shared__ double s_grp[G][KC];
  const int j = blockIdx.x;
  const int m = threadIdx.x % KC, g = threadIdx.x / KC;
  const float* col = part + (size_t)j * KC + m;
  const size_t cs = (size_t)fpad * KC;
  // four accumulators (the group's CTAs taken round-robin), added in a fixed order
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int c = g;
  for (; c + 3 * G < grid; c += 4 * G) {
    a0 += (double)__ldg(col + (size_t)c * cs);
    a1 += (double)__ldg(col + (size_t)(c + G) * cs);
    a2 += (double)__ldg(col + (size_t)(c + 2 * G) * cs);
    a3 += (double)__ldg(col + (size_t)(c + 3 * G) * cs);
  }
  for (; c < grid; c += G) a0 += (double)__ldg(col + (size_t)c * cs);
  s_grp[g][m] = (a0 + a1) + (a2 + a3);
  __syncthreads();
  if (g == 0 && m < K) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < G; ++q) t += s_grp[q][m];
    xtz[(int64_t)m * xtz_stride + j] = t * (colscale ? (double)colscale[j] : 1.0);
  }
}

}  // namespace

int xstream_k_chunks(int p) {
  const int nch = (p + kCF - 1) / kCF;
  return (nch + 1) & ~1;
}

namespace {
// f(KC, S, MINB) as std::integral_constant values for the instantiated launch
// shapes (chain columns, ring stages, CTAs per SM); false for any other.
// Two CTAs per SM only for the narrow tile with four stages: 89 KB of shared
// memory and at most 85 registers a thread each.
template <class F>
bool with_shape(int kc, int stages, int per_sm, F&& f) {
#define HS_XK_SHAPE(KC, S, M)                                                                  \
  if (kc == KC && stages == S && per_sm == M) {                                                \
    f(std::integral_constant<int, KC>{}, std::integral_constant<int, S>{}, std::integral_constant<int, M>{}); \
    return true;                                                                               \
  }
  HS_XK_SHAPE(16, 4, 1) HS_XK_SHAPE(16, 6, 1) HS_XK_SHAPE(16, 8, 1) HS_XK_SHAPE(16, 4, 2)
  HS_XK_SHAPE(32, 4, 1) HS_XK_SHAPE(32, 6, 1) HS_XK_SHAPE(32, 8, 1)
#undef HS_XK_SHAPE
  return false;
}
}  // namespace

size_t xstream_k_smem_bytes(int kc, int stages) {
  size_t b = 0;
  with_shape(kc, stages, 1, [&](auto KC, auto S, auto) { b = XKShape<decltype(KC)::value, decltype(S)::value>::kSmem; });
  return b;
}

bool xstream_k_supported(int p, int kc, int stages, int per_sm) {
  const int nch = xstream_k_chunks(p);
  bool inst = false;
  with_shape(kc, stages, per_sm, [&](auto, auto, auto) { inst = true; });
  const size_t smem = xstream_k_smem_bytes(kc, stages);
  // TMEM: two eta' buffers of 2 KC columns + KC per 128-feature group; with
  // two CTAs per SM each must fit in half of the 512 columns (an allocation
  // never waits for the other CTA)
  return p >= 1 && inst && smem > 0 && 4 * kc + kc * (nch / 2) <= 512 / per_sm &&
         smem * per_sm <= (per_sm == 1 ? 227 * 1024 : 228 * 1024 - 2048);
}

int xstream_k_default_kc(int K) { return K <= 16 ? 16 : 32; }

cudaError_t xstream_k_prepare(int kc, int stages, int per_sm) {
  cudaError_t e = cudaErrorInvalidValue;
  with_shape(kc, stages, per_sm, [&](auto KC, auto S, auto M) {
    constexpr int c = decltype(KC)::value, st = decltype(S)::value, mb = decltype(M)::value;
    e = cudaFuncSetAttribute((const void*)xstream_k_kernel<c, st, mb>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)XKShape<c, st>::kSmem);
  });
  return e;
}

size_t xstream_k_bsw_bytes(int p, int kc) { return (size_t)xstream_k_chunks(p) * bchunk_bytes(kc); }

// The tensor map of X (ld columns, N rows, BF16, row stride ld * 2 bytes):
// boxes of 64 x 128 with 128-byte swizzle; reads outside X return zeros.
int xstream_k_make_map(const void* X, int64_t N, int ld, void* map_out) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult qr;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
        qr != cudaDriverEntryPointSuccess || !fn)
      return -1;
    encode = reinterpret_cast<EncodeFn>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)N};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kCF, (cuuint32_t)kTR};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                            const_cast<void*>(X), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

namespace {
template <class F>
bool with_split(int kc, int fp8, F&& f) {
  if (kc == 16 && !fp8) f(std::integral_constant<int, 16>{}, std::integral_constant<int, 0>{});
  else if (kc == 16 && fp8) f(std::integral_constant<int, 16>{}, std::integral_constant<int, 1>{});
  else if (kc == 32 && !fp8) f(std::integral_constant<int, 32>{}, std::integral_constant<int, 0>{});
  else if (kc == 32 && fp8) f(std::integral_constant<int, 32>{}, std::integral_constant<int, 1>{});
  else return false;
  return true;
}
}  // namespace

bool xstream_k_split_supported(int p, int kc) {
  // pass 2's TMEM: KC columns per 128-feature group
  return p >= 1 && (kc == 16 || kc == 32) && kc * (xstream_k_chunks(p) / 2) <= 512;
}

cudaError_t xstream_k_split_prepare(int kc, int fp8) {
  cudaError_t e = cudaErrorInvalidValue;
  with_split(kc, fp8, [&](auto KC, auto F) {
    constexpr int c = decltype(KC)::value, f8 = decltype(F)::value;
    using Sp = XKSplit<c, f8>;
    e = cudaFuncSetAttribute((const void*)xk_eta_kernel<c, f8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Sp::kSmemEta);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)xk_xtz_kernel<c, f8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)Sp::kSmemXtz);
  });
  return e;
}

int xstream_k_split_stages(int kc) { return kc == 16 ? XKSplit<16, 0>::kStages : XKSplit<32, 0>::kStages; }

size_t xstream_k_zt_bytes(int64_t N, int kc) { return (size_t)((N + kTR - 1) / kTR) * 4 * (size_t)kc * 128; }

cudaError_t xstream_k_split_enqueue(const void* map, const XKArgs& a, const double* beta, int64_t beta_stride,
                                    unsigned char* bsw, int grid, cudaStream_t s) {
  if (a.K > a.kc || !a.zt) return cudaErrorInvalidValue;
  bsw_prep_kernel<<<64, 256, 0, s>>>(beta, beta_stride, a.K, a.p, a.nch, a.kc, a.colscale, bsw);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap m;
  memcpy(&m, map, sizeof(m));
  e = cudaErrorInvalidValue;
  with_split(a.kc, a.fp8, [&](auto KC, auto F) {
    constexpr int c = decltype(KC)::value, f8 = decltype(F)::value;
    using Sp = XKSplit<c, f8>;
    xk_eta_kernel<c, f8><<<grid, Sp::kThreads, Sp::kSmemEta, s>>>(m, a);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
      xk_xtz_kernel<c, f8><<<grid, Sp::kThreads, Sp::kSmemXtz, s>>>(m, a);
      e = cudaGetLastError();
    }
  });
  return e;
}

int xstream_k_make_map_fp8(const void* X, int64_t N, int ld, void* map_out) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult qr;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
        qr != cudaDriverEntryPointSuccess || !fn)
      return -1;
    encode = reinterpret_cast<EncodeFn>(fn);
  }
  // rows of ld one-byte codes (ld a multiple of 16); boxes of 128 codes x 128
  // rows (two 64-feature chunks, whole 128-byte lines of each row), no
  // swizzle (the converter warps read the rows); reads outside X return zeros
  const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)N};
  const cuuint64_t strides[1] = {(cuuint64_t)ld};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * kCF), (cuuint32_t)kTR};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                            const_cast<void*>(X), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

int xstream_k_grid(int64_t N, int num_sms) {
  const int64_t ntiles = (N + kTR - 1) / kTR;
  int64_t g = num_sms > 1 ? (int64_t)num_sms - 1 : 1;
  if (g > ntiles) g = ntiles;
  return (int)(g < 1 ? 1 : g);
}

int64_t xstream_k_tiles(int64_t N) { return (N + kTR - 1) / kTR; }

size_t xstream_k_partial_floats(int p, int grid, int kc) {
  return (size_t)grid * (size_t)(xstream_k_chunks(p) * kCF) * kc;
}

cudaError_t xstream_k_enqueue(const void* map, const XKArgs& a, const double* beta, int64_t beta_stride,
                              unsigned char* bsw, int grid, cudaStream_t s) {
  if (a.K > a.kc) return cudaErrorInvalidValue;
  bsw_prep_kernel<<<64, 256, 0, s>>>(beta, beta_stride, a.K, a.p, a.nch, a.kc, nullptr, bsw);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap m;
  memcpy(&m, map, sizeof(m));
  e = cudaErrorInvalidValue;
  with_shape(a.kc, a.stages, a.per_sm, [&](auto KC, auto S, auto M) {
    using Sh = XKShape<decltype(KC)::value, decltype(S)::value>;
    xstream_k_kernel<Sh::kKc, Sh::kStages, decltype(M)::value><<<grid, Sh::kThreads, Sh::kSmem, s>>>(m, a);
    e = cudaGetLastError();
  });
  return e;
}

cudaError_t xstream_k_reduce(const XKArgs& a, int grid, double* xtz, int64_t xtz_stride, cudaStream_t s) {
  if (a.kc == 16)
    reduce_k_kernel<16><<<a.p, 256, 0, s>>>(a.partials, grid, a.fpad, a.p, a.K, a.colscale, xtz, xtz_stride);
  else if (a.kc == 32)
    reduce_k_kernel<32><<<a.p, 256, 0, s>>>(a.partials, grid, a.fpad, a.p, a.K, a.colscale, xtz, xtz_stride);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace hs

// The X-stream of one Gibbs sweep and its companions.
//
// For every row i the sweep needs eta_i = x_i beta (Sect. 5, z update, step i),
// a draw z_i ~ TN(eta_i, 1, y_i) (Eq. 12, first line; Sect. 5, z update,
// step ii) and the accumulation of X^T z (Sect. 5, beta update, step vi).
// All three need the same row, so one persistent kernel reads X exactly once
// per sweep:
//   * one producer warp streams tiles of R contiguous rows into a ring of
//     shared-memory stages with cp.async.bulk (one bulk copy per tile, its
//     completion counted on an mbarrier);
//   * eight consumer warps own fixed 16-byte column slices of every row,
//     keep their slice of beta in registers, form the row dot products,
//     reduce them across the warp with a transpose-reduction (one lane ends up
//     with each row's warp sum) and across warps through shared memory;
//   * a sampler warp draws the R latents of the tile with the branch-free
//     inverse-CDF sampler on counter-based Philox (the sign of y folded in as
//     in the paper's y*_i = 2 y_i - 1); it holds none of the tile's X
//     registers, which keeps the kernel's register count low enough for the
//     Cholesky branch to run beside it on every SM;
//   * every consumer thread then folds x_ij z_i into its register
//     accumulators of X^T z for its own columns.
// Each CTA owns a contiguous range of row tiles and writes one row of
// partial sums; a second kernel adds the rows in a fixed order in FP64.
#include <cuda_fp8.h>

#include "hs_common.cuh"
#include "hs_internal.h"
#include "hs_probit.h"

namespace hs {
namespace {

constexpr int kConsumerWarps = 8;
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kSamplerWarp = kConsumerWarps;          // draws z for the tile
constexpr int kProducerWarp = kConsumerWarps + 1;     // issues the bulk copies
constexpr int kBarThreads = kConsumers + 32;          // consumers + sampler
constexpr int kThreads = kConsumers + 64;

// ---- storage formats: one 16-byte vector -> VE compute-type values ---------
template <int XD> struct XFmt;
template <> struct XFmt<HS_X_F64> {
  using CT = double;
  static constexpr int VE = 2;
  static constexpr int kElemBytes = 8;
  static __device__ __forceinline__ void cvt(const uint4& v, CT* o) {
    o[0] = __hiloint2double((int)v.y, (int)v.x);
    o[1] = __hiloint2double((int)v.w, (int)v.z);
  }
};
template <> struct XFmt<HS_X_F32> {
  using CT = float;
  static constexpr int VE = 4;
  static constexpr int kElemBytes = 4;
  static __device__ __forceinline__ void cvt(const uint4& v, CT* o) {
    o[0] = __uint_as_float(v.x);
    o[1] = __uint_as_float(v.y);
    o[2] = __uint_as_float(v.z);
    o[3] = __uint_as_float(v.w);
  }
};
template <> struct XFmt<HS_X_BF16> {
  using CT = float;
  static constexpr int VE = 8;
  static constexpr int kElemBytes = 2;
  static __device__ __forceinline__ void cvt(const uint4& v, CT* o) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      o[2 * i] = __uint_as_float(w[i] << 16);
      o[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
  }
};
template <> struct XFmt<HS_X_FP8E4M3> {
  using CT = float;
  static constexpr int VE = 16;
  static constexpr int kElemBytes = 1;
  static __device__ __forceinline__ void cvt(const uint4& v, CT* o) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const __nv_fp8x2_storage_t pair = (__nv_fp8x2_storage_t)((w[i] >> (16 * h)) & 0xFFFFu);
        const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(pair, __NV_E4M3);
        const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&hr));
        o[4 * i + 2 * h] = f.x;
        o[4 * i + 2 * h + 1] = f.y;
      }
    }
  }
};

// ---- warp transpose-reduction --------------------------------------------
// d[0..V) per lane -> after log2(V) halving exchanges each lane holds one
// partially reduced row; butterflies over the remaining lane bits finish the
// sum.  Lane l ends with the full warp sum of row (l >> (5 - log2 R)) & (R-1).
template <int H, int OFF, typename T>
__device__ __forceinline__ void halve(T* d, int lane) {
  const bool up = (lane & OFF) != 0;
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const T send = up ? d[i] : d[i + H];
    const T keep = up ? d[i + H] : d[i];
    d[i] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
  }
}
template <int V, int OFF, typename T>
__device__ __forceinline__ T treduce(T* d, int lane) {
  if constexpr (V > 1) {
    halve<V / 2, OFF>(d, lane);
    return treduce<V / 2, OFF / 2>(d, lane);
  } else {
    T v = d[0];
#pragma unroll
    for (int off = OFF; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
  }
}
template <int R> struct RowOfLane {
  static constexpr int kShift = (R == 1) ? 5 : (R == 2) ? 4 : (R == 4) ? 3 : (R == 8) ? 2 : 1;
  static __device__ __forceinline__ int row(int lane) { return (lane >> kShift) & (R - 1); }
  static __device__ __forceinline__ bool writer(int lane) { return (lane & ((1 << kShift) - 1)) == 0; }
};

struct SmemPlan {
  int nstage;
  uint32_t stage_bytes;
  size_t total;
};

template <int XD, int R>
SmemPlan plan_smem(int ld) {
  using F = XFmt<XD>;
  SmemPlan s;
  const size_t row_bytes = (size_t)ld * F::kElemBytes;
  s.stage_bytes = (uint32_t)(((size_t)R * row_bytes + 127) / 128 * 128);
  const size_t extras = 2 * 8 * 8 + (size_t)(kConsumerWarps * R + R) * sizeof(typename F::CT) + 256;
  // One CTA per SM with about 130 KB of stages: enough bytes in flight to
  // cover HBM latency, while leaving shared memory, registers and threads on
  // every SM for the concurrent Cholesky branch of the sweep.
  const size_t budget = 132 * 1024;
  int n = (int)((budget - extras) / s.stage_bytes);
  if (n < 2) n = 2;
  if (n > 8) n = 8;
  s.nstage = n;
  s.total = (size_t)n * s.stage_bytes + extras;
  return s;
}

template <int XD, int S, int R>
__global__ void __launch_bounds__(kThreads, 1)
    xstream_kernel(XStreamArgs a, int nstage, uint32_t stage_bytes) {
  using F = XFmt<XD>;
  using CT = typename F::CT;
  constexpr int VE = F::VE;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_cabort;  // written by consumers before barrier 1 only
  __shared__ int s_pabort;  // written by the producer only
  __shared__ int64_t s_issued, s_consumed;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)nstage * stage_bytes);
  uint64_t* empty = full + nstage;
  CT* red = reinterpret_cast<CT*>(empty + nstage);  // [warps][R]
  CT* zs = red + kConsumerWarps * R;                // [R]

  const int64_t ntiles = (a.N + R - 1) / R;
  const int64_t t0 = ntiles * blockIdx.x / gridDim.x;
  const int64_t t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
  const size_t row_bytes = (size_t)a.ld * F::kElemBytes;
  const int nvec = a.ld / VE;

  if (tid == 0) {
    if (a.sm_mark) {
      // tell the factorization, running beside this kernel, which SMs are busy here
      unsigned int smid;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
      if (smid < (unsigned)kSmMarks) a.sm_mark[smid] = (unsigned int)(*a.k_dev + 1);
    }
    for (int s = 0; s < nstage; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    fence_mbar_init();
    s_cabort = 0;
    s_pabort = 0;
    s_issued = 0;
    s_consumed = 0;
  }
  __syncthreads();
  const uint32_t sweep = (uint32_t)(*a.k_dev + 1);

  if (warp == kProducerWarp) {
    // ---------------- producer ----------------
    if (lane == 0) {
      const unsigned char* X = static_cast<const unsigned char*>(a.X);
      // X is read once per sweep: keep the factorization's tiles (running
      // beside this kernel) in L2 instead
      const uint64_t policy = l2_evict_first_policy();
      int64_t it = 0;
      for (int64_t t = t0; t < t1; ++t, ++it) {
        const int s = (int)(it % nstage);
        const uint32_t use = (uint32_t)(it / nstage);
        if (use > 0) {
          // Wait for the consumers to release this stage: 100 x 20 ms at most,
          // giving up early if the consumers have stopped.
          bool ok = false;
          for (int tries = 0; tries < 100 && !ok; ++tries) {
            ok = mbar_wait(&empty[s], (use - 1) & 1u, 20000000ull);
            if (!ok && *(volatile int*)&s_cabort) break;
          }
          if (!ok) {
            if (!*(volatile int*)&s_cabort) set_error(a.err, kErrTimeout);
            s_pabort = 1;
            break;
          }
        }
        if (*(volatile int*)&s_cabort) break;
        const int rows = (int)min((int64_t)R, a.N - t * R);
        const uint32_t bytes = (uint32_t)(rows * row_bytes);
        mbar_arrive_expect_tx(&full[s], bytes);
        bulk_g2s_hint(smem + (size_t)s * stage_bytes, X + (size_t)t * R * row_bytes, bytes, &full[s], policy);
      }
      s_issued = it;
    }
  } else if (warp == kSamplerWarp) {
    // ---------------- sampler ----------------
    const Rng rng{a.rng.k0, a.rng.k1, a.rng.chain, a.rng.problem};
    int64_t it = 0;
    for (int64_t t = t0; t < t1; ++t, ++it) {
      const int rows = (int)min((int64_t)R, a.N - t * R);
      const bool active = lane < R && lane < rows;
      const int64_t i = t * R + lane;
      // counters and y do not depend on eta: fetch them while the consumers reduce
      double u = 0.5, uc = 0.5;
      int yi = 1;
      if (active) {
        yi = a.y[i];
        const uint4 wd = rng.words((uint32_t)i, sweep, kPurZ);
        unit_pair(wd.x, wd.y, u, uc);
      }
      named_bar_sync(1, kBarThreads);
      if (*(volatile int*)&s_cabort) break;
      CT eta = CT(0);
      if (lane < R) {
#pragma unroll
        for (int w = 0; w < kConsumerWarps; ++w) eta += red[w * R + lane];
      }
      const CT ms = active ? (yi ? eta : -eta) : CT(0);
      CT zp = tn_main<CT>(ms, (CT)u, (CT)uc);
      const bool tail = active && ms < TnMath<CT>::kTail;
      if (__any_sync(0xffffffffu, tail)) {
        const CT zt = tn_tail<CT>(tail ? ms : CT(-1), (CT)u, (CT)uc);
        zp = tail ? zt : zp;
      }
      zp = zp > TnMath<CT>::tiny() ? zp : TnMath<CT>::tiny();
      CT z = active ? (yi ? zp : -zp) : CT(0);
      if (active && !isfinite(z)) {
        set_error(a.err, kErrNonFinite);
        z = CT(0);
      }
      if (active && a.z_out) a.z_out[i] = (double)z;
      if (lane < R) zs[lane] = z;
      named_bar_sync(1, kBarThreads);
    }
  } else {
    // ---------------- consumers ----------------
    CT b[S][VE];
    CT acc[S][VE];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int v = tid + s * kConsumers;
#pragma unroll
      for (int e = 0; e < VE; ++e) {
        b[s][e] = (v < nvec) ? static_cast<const CT*>(a.beta_c)[v * VE + e] : CT(0);
        acc[s][e] = CT(0);
      }
    }
    int64_t it = 0;
    for (int64_t t = t0; t < t1; ++t, ++it) {
      const int st = (int)(it % nstage);
      const uint32_t ph = (uint32_t)((it / nstage) & 1);
      const bool ok = mbar_wait(&full[st], ph);
      if (!ok) {
        set_error(a.err, kErrTimeout);
        *(volatile int*)&s_cabort = 1;
      }
      const int rows = (int)min((int64_t)R, a.N - t * R);
      const unsigned char* base = smem + (size_t)st * stage_bytes;
      uint4 xr[R][S];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const int v = tid + s * kConsumers;
          xr[r][s] = (ok && r < rows && v < nvec)
                         ? *reinterpret_cast<const uint4*>(base + (size_t)r * row_bytes + (size_t)v * 16)
                         : make_uint4(0u, 0u, 0u, 0u);
        }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);

      CT d[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        d[r] = CT(0);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          CT xv[VE];
          F::cvt(xr[r][s], xv);
#pragma unroll
          for (int e = 0; e < VE; ++e) d[r] = fma(xv[e], b[s][e], d[r]);
        }
      }
      const CT rsum = treduce<R, 16>(d, lane);
      if (RowOfLane<R>::writer(lane)) red[warp * R + RowOfLane<R>::row(lane)] = rsum;
      named_bar_sync(1, kBarThreads);
      // s_cabort is only written before this barrier, so every consumer and
      // the sampler read the same value here and all of them leave together.
      if (*(volatile int*)&s_cabort) break;
      named_bar_sync(1, kBarThreads);  // z of the tile is in zs

#pragma unroll
      for (int r = 0; r < R; ++r) {
        const CT zr = zs[r];
#pragma unroll
        for (int s = 0; s < S; ++s) {
          CT xv[VE];
          F::cvt(xr[r][s], xv);
#pragma unroll
          for (int e = 0; e < VE; ++e) acc[s][e] = fma(xv[e], zr, acc[s][e]);
        }
      }
    }
    if (tid == 0) s_consumed = it;
    CT* part = static_cast<CT*>(a.partials) + (size_t)blockIdx.x * a.ld;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int v = tid + s * kConsumers;
      if (v < nvec) {
#pragma unroll
        for (int e = 0; e < VE; ++e) part[v * VE + e] = acc[s][e];
      }
    }
  }
  __syncthreads();
  // After an abort, wait (bounded) for the bulk copies still landing in
  // shared memory before the CTA exits.
  if (tid == 0 && (s_cabort || s_pabort)) {
    for (int64_t it = s_consumed; it < s_issued; ++it) {
      const int st = (int)(it % nstage);
      if (!mbar_wait(&full[st], (uint32_t)((it / nstage) & 1))) break;
    }
  }
}

template <int XD, int S, int R>
cudaError_t launch_one(const XStreamArgs& a, int grid, cudaStream_t s) {
  const SmemPlan pl = plan_smem<XD, R>(a.ld);
  auto k = xstream_kernel<XD, S, R>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.total);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  k<<<grid, kThreads, pl.total, s>>>(a, pl.nstage, pl.stage_bytes);
  return cudaGetLastError();
}

template <int XD>
int vec_elems() {
  return XFmt<XD>::VE;
}

// Rows per tile for one 16-byte slice per thread: FP64/FP32 take 16 rows;
// the narrow formats unpack 8 or 16 values per slice and take fewer rows to
// stay within the register budget.  FP8 takes 8 (measured at p = 4000: with 4
// rows, 16 KB tiles, the per-tile barriers and draws held the kernel to a
// third of HBM bandwidth).
template <int XD> constexpr int rows_s1() { return XD == HS_X_FP8E4M3 ? 8 : XD == HS_X_BF16 ? 8 : 16; }

template <int XD>
cudaError_t launch_dtype(const XStreamArgs& a, int grid, cudaStream_t s) {
  const int nvec = a.ld / XFmt<XD>::VE;
  const int S = (nvec + kConsumers - 1) / kConsumers;
  if (S <= 1) return launch_one<XD, 1, rows_s1<XD>()>(a, grid, s);
  if (S <= 2) return launch_one<XD, 2, 4>(a, grid, s);
  if (S <= 4) return launch_one<XD, 4, 2>(a, grid, s);
  if (S <= 8) return launch_one<XD, 8, 1>(a, grid, s);
  return cudaErrorInvalidValue;
}

template <int XD>
int grid_dtype(int ld, int64_t N, int num_sms) {
  const int nvec = ld / XFmt<XD>::VE;
  const int S = (nvec + kConsumers - 1) / kConsumers;
  const int R = S <= 1 ? rows_s1<XD>() : S <= 2 ? 4 : S <= 4 ? 2 : 1;
  const int64_t ntiles = (N + R - 1) / R;
  // One persistent CTA per SM but one: the SM left free runs the diagonal
  // chain of the factorization beside this kernel (the same grid whatever the
  // factorization schedule, so every entry point partitions X alike).
  int64_t g = num_sms > 1 ? (int64_t)num_sms - 1 : 1;
  if (g > ntiles) g = ntiles;
  if (g < 1) g = 1;
  return (int)g;
}

// ---- second stage: fixed-order FP64 sum of the per-CTA partials -------------
// Block of 32 columns x 8 groups: thread (g, c) adds the partial rows
// g, g + 8, g + 16, ... of its column, then group 0 adds the 8 group sums in
// order, so the sum is the same every sweep and the loads of a column are in
// flight 8 at a time.
constexpr int kRedCols = 32, kRedGroups = 8;
template <typename CT>
__global__ void __launch_bounds__(kRedCols * kRedGroups)
    reduce_partials_kernel(const CT* __restrict__ part, int grid, int ld, int p, const float* __restrict__ colscale,
                           double* __restrict__ xtz) {
  __shared__ double s_grp[kRedGroups][kRedCols];
  const int c = threadIdx.x % kRedCols, g = threadIdx.x / kRedCols;
  const int j = blockIdx.x * kRedCols + c;
  double s0 = 0.0, s1 = 0.0;
  if (j < p) {
    int b = g;
    for (; b + kRedGroups < grid; b += 2 * kRedGroups) {
      s0 += (double)part[(size_t)b * ld + j];
      s1 += (double)part[(size_t)(b + kRedGroups) * ld + j];
    }
    if (b < grid) s0 += (double)part[(size_t)b * ld + j];
  }
  s_grp[g][c] = s0 + s1;
  __syncthreads();
  if (g == 0 && j < p) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kRedGroups; ++q) s += s_grp[q][c];
    if (colscale) s *= (double)colscale[j];
    xtz[j] = s;
  }
}

__global__ void check_y_kernel(const uint8_t* __restrict__ y, int64_t N, int* err) {
  int bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    bad |= (y[i] > 1);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, kErrBadY);
}

}  // namespace

int partial_elem_bytes(int x_dtype) { return x_dtype == HS_X_F64 ? 8 : 4; }

cudaError_t xstream_prepare() {
  const void* fns[] = {(const void*)reduce_partials_kernel<double>, (const void*)reduce_partials_kernel<float>,
                       (const void*)check_y_kernel};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int xstream_grid(int x_dtype, int p, int ld, int64_t N, int num_sms) {
  (void)p;
  switch (x_dtype) {
    case HS_X_F64: return grid_dtype<HS_X_F64>(ld, N, num_sms);
    case HS_X_F32: return grid_dtype<HS_X_F32>(ld, N, num_sms);
    case HS_X_BF16: return grid_dtype<HS_X_BF16>(ld, N, num_sms);
    case HS_X_FP8E4M3: return grid_dtype<HS_X_FP8E4M3>(ld, N, num_sms);
  }
  return 1;
}

cudaError_t xstream_launch(int x_dtype, const XStreamArgs& a, int grid, cudaStream_t s) {
  switch (x_dtype) {
    case HS_X_F64: return launch_dtype<HS_X_F64>(a, grid, s);
    case HS_X_F32: return launch_dtype<HS_X_F32>(a, grid, s);
    case HS_X_BF16: return launch_dtype<HS_X_BF16>(a, grid, s);
    case HS_X_FP8E4M3: return launch_dtype<HS_X_FP8E4M3>(a, grid, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t reduce_partials_launch(int x_dtype, const void* partials, int grid, int ld, int p,
                                   const float* colscale, double* xtz, cudaStream_t s) {
  const int nb = (p + kRedCols - 1) / kRedCols;
  if (x_dtype == HS_X_F64)
    reduce_partials_kernel<double><<<nb, kRedCols * kRedGroups, 0, s>>>(static_cast<const double*>(partials), grid,
                                                                         ld, p, colscale, xtz);
  else
    reduce_partials_kernel<float><<<nb, kRedCols * kRedGroups, 0, s>>>(static_cast<const float*>(partials), grid, ld,
                                                                        p, colscale, xtz);
  return cudaGetLastError();
}

cudaError_t check_y_launch(const uint8_t* y, int64_t N, int* err, cudaStream_t s) {
  int64_t nb = (N + 255) / 256;
  if (nb > 4096) nb = 4096;
  if (nb < 1) nb = 1;
  check_y_kernel<<<(int)nb, 256, 0, s>>>(y, N, err);
  return cudaGetLastError();
}

}  // namespace hs

// Host runtime and C ABI of the Horseshoe-probit Gibbs sweep.
//
// One handle holds the data (X in its storage type with 16-byte aligned rows,
// y, optional column scales), the one-time Gram matrix, the sampler state
// (beta, lambda^{-2}, nu^{-1}, tau^{-2}, xi^{-1}, sweep count k) and the work
// buffers, all in device memory it owns.  A sweep is a fork/join DAG on two
// streams: the X-stream (and the reduce of its partial sums) on the main
// stream runs concurrently with the lambda/tau kernel and the Cholesky branch
// on a side stream, which depend only on the previous state (Sect. 5,
// schedule (i)-(ii): z and lambda first, tau next, then beta, nu, xi).  The
// beta tail joins both.  The DAG can be captured once as a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "hs_internal.h"
#include "hs_probit.h"

namespace {

thread_local int g_last_error = HS_OK;

constexpr int kMaxP = 8192;
constexpr int kProfGroups = 6;

struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = (cudaSetDevice(dev) == cudaSuccess);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int elem_bytes_of(int dt) {
  switch (dt) {
    case HS_X_F64: return 8;
    case HS_X_F32: return 4;
    case HS_X_BF16: return 2;
    case HS_X_FP8E4M3: return 1;
  }
  return 0;
}

}  // namespace

struct hs_probit {
  hs_probit_config cfg{};
  int device = 0;
  int x_dtype = HS_X_F32;
  int64_t N = 0;
  int p = 0, ld = 0, P = 0, T = 0;
  int elem = 4;
  hs::RngKey rng{};
  cudaStream_t s0 = nullptr, s1 = nullptr;
  bool own_s0 = false;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_shrink = nullptr, ev_xs = nullptr;
  std::vector<void*> allocs;

  void* X = nullptr;
  uint8_t* y = nullptr;
  float* colscale = nullptr;
  double *beta = nullptr, *lam = nullptr, *nu = nullptr, *scal = nullptr;
  int64_t* k_dev = nullptr;
  double *lam_new = nullptr, *tau_new = nullptr, *beta_new = nullptr, *nu_new = nullptr;
  void* beta_c = nullptr;
  double *G = nullptr, *S = nullptr, *A = nullptr, *Linv = nullptr, *LinvT = nullptr;
  double *xtz = nullptr, *v = nullptr;
  double* shrink_part = nullptr;
  unsigned int* shrink_ticket = nullptr;
  unsigned long long* chol_sync = nullptr;  // readiness words of the single-launch factorization
  unsigned int* sm_mark = nullptr;          // SM occupancy marks of the X-stream (single launch only)
  int chol_grid = 0;                        // its blocks; 0: one launch per block column
  size_t chol_words = 0;                    // scheduling words per chain
  int* chol_order = nullptr;                // worker task list of the single-launch factorization
  int chol_ntasks = 0;                      // its length
  // HS_SCHED_TENSOR: block-column launches and tensor-core trailing updates
  bool tensor_sched = false;
  void* digits = nullptr;                   // K x 6 digit planes of P x P BF16
  unsigned long long* sm_role = nullptr;    // per-SM claim and role words of the block-column launches
  void* G2 = nullptr;                       // P x P FP32 pairs of the Gram matrix
  int* blk_order = nullptr;                 // the block columns' task lists, one after another
  std::vector<int> blk_off, blk_len;
  int trail_grid = 0;
  alignas(64) unsigned char tmapA[128];     // tensor maps of the digit planes (128- and 64-row boxes)
  alignas(64) unsigned char tmapB[128];
  // K chains sharing X: every per-chain buffer holds K slices (chain m at offset m * size)
  int K = 1;
  int64_t* k_scratch = nullptr;             // K: commits of chains 0..K-2 record the sweep here
  int kgrid = 0;                            // batched X-stream CTAs
  bool xk = false;                          // K chains on the tensor-core X-stream (else one pass per chain)
  int xk_kc = 32, xk_stages = 8, xk_per_sm = 1;  // its launch shape (chain columns, ring stages, CTAs per SM)
  bool xk_split = false;                    // as two kernels (FP8 X, or p past the fused kernel's TMEM)
  void* zt = nullptr;                       // the split form's Z^T tiles
  bool beside = false;                      // K chains: the factorization beside the X-stream (else after it)
  int grid_max = 0, kgrid_max = 0, trail_max = 0, chol_max = 0;  // launch sizes the buffers were made for
  // draws copied on a side stream while later sweeps compute
  cudaStream_t s_dl = nullptr;
  cudaEvent_t ev_mark = nullptr, ev_dl = nullptr;
  int64_t dl_oldest = -1;                   // oldest draw index a copy may still read, or -1
  // launch shapes set by a batch (hs_probit_batch_*): no cooperative launch, no
  // chain SM isolation, and the factorization's grid chosen by the batch's tuner
  bool batch_member = false;
  uint64_t shape_epoch = 0;                 // bumped by every launch-shape change (a batch recaptures)
  unsigned char* bsw = nullptr;             // B^T of the batched X-stream
  float* kpartials = nullptr;
  alignas(64) unsigned char xmap[128];      // tensor map of X (batched X-stream)
  void* partials = nullptr;
  int grid = 1;
  double* z = nullptr;
  double *ring_beta = nullptr, *ring_lam = nullptr, *ring_tau = nullptr;
  int ring_size = 1, thin = 1;
  int* err = nullptr;
  int* hook_err = nullptr;
  int* hook_flag = nullptr;
  int* h_err = nullptr;      // pinned
  int64_t* h_k = nullptr;    // pinned

  int sticky = HS_OK;
  int last_err_word = 0;     // device error word seen by the last synchronization
  int64_t k_host = 0;
  std::vector<int64_t> drained;  // per chain: draws (index k/thin) already handed out
  int64_t launches = 0;
  bool chol_inverse = true;  // the factorization forms L~^{-1} (HS_BETA_INVERSE)

  bool graph_ready = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  // Event-record nodes of the captured graph (start/end of each kernel group),
  // re-pointed at fresh events before each launch while profiling.
  bool capturing = false;
  cudaEvent_t placeholder[kProfGroups][2] = {};
  cudaGraphNode_t prof_node[kProfGroups][2] = {};

  int profiling = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  double prof_ms[kProfGroups] = {0};
  int64_t prof_n[kProfGroups] = {0};

  template <typename T>
  cudaError_t alloc(T** p, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes < 16 ? 16 : bytes);
    if (e == cudaSuccess) {
      allocs.push_back(q);
      *p = static_cast<T*>(q);
    }
    return e;
  }
  cudaEvent_t take_event() {
    if (!ev_pool.empty()) {
      cudaEvent_t e = ev_pool.back();
      ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};

namespace {

int fail(int status) {
  g_last_error = status;
  return status;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return HS_OK;
  if (e == cudaErrorMemoryAllocation) return HS_ENOMEM;
  return HS_ECUDA;
}

int status_from_err_bits(int bits) {
  if (bits & hs::kErrNonFinite) return HS_ENONFINITE;
  if (bits & hs::kErrNotPD) return HS_ENOTPD;
  if (bits & hs::kErrTimeout) return HS_ETIMEOUT;
  if (bits & hs::kErrGamma) return HS_ENONFINITE;
  if (bits & hs::kErrBadY) return HS_EINVAL;
  return HS_ECUDA;
}

// Worker task list of the single-launch factorization: two task slots per
// worker block, shared by the chains.
std::vector<int> single_task_list(const hs_probit* h) {
  const int slots = 2 * (h->chol_grid - h->K) / h->K;
  return hs::chol_task_codes(h->T, slots > 1 ? slots : 1, h->chol_inverse);
}

// The block columns' task lists, one after another (fills blk_off, blk_len).
std::vector<int> block_task_lists(hs_probit* h) {
  std::vector<int> all;
  h->blk_off.clear();
  h->blk_len.clear();
  for (int b = 0; hs::kTrailBlockTiles * b < h->T; ++b) {
    const int slots = std::max(1, 2 * (h->chol_grid - h->K) / h->K);
    const std::vector<int> c = hs::chol_block_task_codes(
        h->T, hs::kTrailBlockTiles * b, std::min(hs::kTrailBlockTiles * (b + 1), h->T), slots);
    h->blk_off.push_back((int)all.size());
    h->blk_len.push_back((int)c.size());
    all.insert(all.end(), c.begin(), c.end());
  }
  return all;
}

hs::XStreamArgs xstream_args(hs_probit* h) {
  hs::XStreamArgs a{};
  a.X = h->X;
  a.y = h->y;
  a.N = h->N;
  a.ld = h->ld;
  a.p = h->p;
  a.beta_c = h->beta_c;
  a.partials = h->partials;
  a.z_out = h->cfg.debug ? h->z : nullptr;
  a.k_dev = h->k_dev;
  a.rng = h->rng;
  a.err = h->err;
  a.sm_mark = h->sm_mark;
  return a;
}

hs::XKArgs xk_args(hs_probit* h) {
  hs::XKArgs a{};
  a.y = h->y;
  a.N = h->N;
  a.p = h->p;
  a.nch = hs::xstream_k_chunks(h->p);
  a.fpad = a.nch * 64;
  a.K = h->K;
  a.kc = h->xk_kc;
  a.stages = h->xk_stages;
  a.per_sm = h->xk_per_sm;
  a.fp8 = h->x_dtype == HS_X_FP8E4M3 ? 1 : 0;
  a.colscale = h->colscale;
  a.zt = h->zt;
  a.bsw = h->bsw;
  a.partials = h->kpartials;
  a.z_out = h->cfg.debug ? h->z : nullptr;
  a.k_dev = h->k_dev;
  a.rng = h->rng;
  a.err = h->err;
  a.sm_mark = h->sm_mark;
  return a;
}

hs::RngKey chain_rng(const hs_probit* h, int m) {
  hs::RngKey r = h->rng;
  r.chain += (uint32_t)m;
  return r;
}

size_t shrink_blocks(const hs_probit* h) { return (size_t)((h->p + 127) / 128); }

int update_mask(const hs_probit* h) {
  return h->cfg.update_mask ? h->cfg.update_mask : (HS_UPD_LAMBDA | HS_UPD_TAU | HS_UPD_NU | HS_UPD_XI);
}

hs::ShrinkArgs shrink_args(hs_probit* h, int m) {
  const size_t p = (size_t)h->p;
  hs::ShrinkArgs a{};
  a.update_mask = update_mask(h);
  a.p = h->p;
  a.P = h->P;
  a.rng = chain_rng(h, m);
  a.k_dev = h->k_dev;
  a.beta = h->beta + m * p;
  a.lam = h->lam + m * p;
  a.nu = h->nu + m * p;
  a.scal = h->scal + 2 * m;
  a.lam_new = h->lam_new + m * p;
  a.tau_new = h->tau_new + m;
  a.G = h->G;
  a.S = h->S + (size_t)m * h->P;
  a.part = h->shrink_part + m * (shrink_blocks(h) + 1);
  a.ticket = h->shrink_ticket + m;
  a.err = h->err;
  a.unit_diag = h->tensor_sched ? 1 : 0;
  return a;
}

hs::CholArgs chol_args(hs_probit* h, int m) {
  const size_t p = (size_t)h->p, P2 = (size_t)h->P * h->P;
  hs::CholArgs a{};
  a.p = h->p;
  a.P = h->P;
  a.G = h->G;
  a.S = h->S + (size_t)m * h->P;
  a.lam_new = h->lam_new + m * p;
  a.tau_new = h->tau_new + m;
  a.A = h->A + m * P2;
  a.Linv = h->Linv + m * P2;
  a.LinvT = h->LinvT + m * P2;
  a.err = h->err;
  a.arith = h->cfg.chol_arith;
  a.sync = h->chol_sync ? h->chol_sync + m * h->chol_words : nullptr;
  a.persistent_grid = h->chol_grid;
  a.sm_mark = h->sm_mark;
  a.k_dev = h->k_dev;
  a.nchains = 1;
  a.sync_words = h->chol_words;
  a.order = h->chol_order;
  a.ntasks = h->chol_ntasks;
  a.inverse = h->chol_inverse ? 1 : 0;
  a.cooperative = h->batch_member ? 0 : 1;
  return a;
}

hs::TailArgs tail_args(hs_probit* h, int m) {
  const size_t p = (size_t)h->p, P2 = (size_t)h->P * h->P, rp = (size_t)h->ring_size * p;
  hs::TailArgs a{};
  a.update_mask = update_mask(h);
  a.p = h->p;
  a.P = h->P;
  a.ld = h->ld;
  a.rng = chain_rng(h, m);
  a.k_dev = h->k_dev;
  a.xtz = h->xtz + m * p;
  a.S = h->S + (size_t)m * h->P;
  a.Linv = h->Linv + m * P2;
  a.LinvT = h->LinvT + m * P2;
  a.df32 = (h->cfg.chol_arith == HS_CHOL_DF32);
  a.solve = h->chol_inverse ? 0 : 1;
  a.L = h->A + m * P2;
  a.v = h->v + (size_t)m * h->P;
  a.beta_new = h->beta_new + m * p;
  a.nu_new = h->nu_new + m * p;
  a.lam_new = h->lam_new + m * p;
  a.tau_new = h->tau_new + m;
  a.beta = h->beta + m * p;
  a.lam = h->lam + m * p;
  a.nu = h->nu + m * p;
  a.scal = h->scal + 2 * m;
  // the shared sweep count moves with the last chain's commit, after every chain's draws
  a.k_dev_rw = (m == h->K - 1) ? h->k_dev : h->k_scratch + m;
  a.beta_c = static_cast<unsigned char*>(h->beta_c) + (size_t)m * h->ld * (h->x_dtype == HS_X_F64 ? 8 : 4);
  a.beta_c_is_double = (h->x_dtype == HS_X_F64);
  a.colscale = h->colscale;
  a.ring_beta = h->ring_beta + m * rp;
  a.ring_lam = h->ring_lam + m * rp;
  a.ring_tau = h->ring_tau + (size_t)m * h->ring_size;
  a.ring_size = h->ring_size;
  a.thin = h->thin;
  a.err = h->err;
  return a;
}

hs::TrailArgs trail_args(hs_probit* h) {
  hs::TrailArgs ta{};
  ta.p = h->p;
  ta.P = h->P;
  ta.nchains = h->K;
  ta.col_lo = 0;
  ta.col_hi = h->T;
  ta.A = h->A;
  ta.G2 = h->G2;
  ta.S = h->S;
  ta.lam_new = h->lam_new;
  ta.tau_new = h->tau_new;
  ta.sync = h->chol_sync;
  ta.sync_words = h->chol_words;
  ta.err = h->err;
  return ta;
}

// Record a profiling event pair around a group on a stream.  While a graph is
// being captured the group's placeholder events are recorded instead, which
// become event-record nodes of the graph.
struct ProfSpan {
  hs_probit* h;
  int group;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr;
  ProfSpan(hs_probit* hh, int g, cudaStream_t ss) : h(hh), group(g), s(ss) {
    if (h->capturing) {
      // External records become event-record nodes of the captured graph.
      cudaEventRecordWithFlags(h->placeholder[group][0], s, cudaEventRecordExternal);
    } else if (h->profiling) {
      e0 = h->take_event();
      cudaEventRecord(e0, s);
    }
  }
  ~ProfSpan() {
    if (h->capturing) {
      cudaEventRecordWithFlags(h->placeholder[group][1], s, cudaEventRecordExternal);
    } else if (h->profiling && e0) {
      cudaEvent_t e1 = h->take_event();
      cudaEventRecord(e1, s);
      h->pending.push_back({group, {e0, e1}});
    }
  }
};

// Enqueue one sweep (eager launches).  Returns a CUDA error or success.
cudaError_t enqueue_sweep(hs_probit* h) {
  cudaError_t e;
  if ((e = cudaEventRecord(h->ev_fork, h->s0)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(h->s1, h->ev_fork, 0)) != cudaSuccess) return e;
  {
    ProfSpan sp(h, 2, h->s1);
    if ((e = hs::shrink_launch(shrink_args(h, 0), h->s1, h->K)) != cudaSuccess) return e;
  }
  // s and nu^{-1} (substitution form, and the FP32-pair products) are drawn beside the factorization
  const bool noise_beside = !h->chol_inverse || h->cfg.chol_arith == HS_CHOL_DF32;
  if (noise_beside && (e = cudaEventRecord(h->ev_shrink, h->s1)) != cudaSuccess) return e;
  // the work matrix of the factorization, beside the X-stream (outside the
  // timed spans: one span per kernel group and sweep)
  if (h->tensor_sched && (e = hs::precision_pairs_launch(trail_args(h), h->s1)) != cudaSuccess) return e;
  // One chain: the factorization runs beside the X-stream (its blocks are
  // small enough to share the SMs).  Several chains on the single-launch
  // schedule: both fill the GPU, so the factorization follows the X-stream
  // explicitly (same total time, and each group's events time only itself).
  const bool after_xstream = h->K > 1 && h->chol_grid > 0 && !h->beside;
  auto factorize = [&]() -> cudaError_t {
    cudaError_t ee;
    {
      ProfSpan sp(h, 3, h->s1);
      if (h->tensor_sched) {
        // block column b: its tile tasks (one launch), then the rank-128 update
        // of everything to its right on the tensor cores (one launch)
        hs::CholArgs ca = chol_args(h, 0);
        ca.nchains = h->K;
        ca.digits = h->digits;
        ca.prebuilt = 1;  // precision_pairs_kernel wrote A~ beside the X-stream
        const hs::TrailArgs ta = trail_args(h);
        const int slots = 2 * (h->chol_grid - h->K);
        for (int b = 0; b < (int)h->blk_off.size(); ++b) {
          ca.k0 = hs::kTrailBlockTiles * b;
          ca.k1 = std::min(hs::kTrailBlockTiles * (b + 1), h->T);
          ca.order = h->blk_order + h->blk_off[b];
          ca.ntasks = h->blk_len[b];
          // chains on SMs of their own where the block column's chain, not its
          // task list, bounds the launch (measured: fewer than about five tasks
          // per worker slot)
          ca.sm_role = (h->K == 1 || (double)h->blk_len[b] * h->K < 5.0 * slots) ? h->sm_role : nullptr;
          if (h->batch_member) ca.sm_role = nullptr;  // the batch's tuner sizes the grid instead
          if ((ee = hs::chol_enqueue(ca, h->s1, nullptr)) != cudaSuccess) return ee;
          hs::TrailArgs tb = ta;
          tb.b = b;
          if ((ee = hs::chol_trail_launch(h->tmapA, h->tmapB, tb, h->trail_grid, h->s1)) != cudaSuccess) return ee;
        }
      } else if (after_xstream) {
        // every chain's factorization in one launch
        hs::CholArgs ca = chol_args(h, 0);
        ca.nchains = h->K;
        if ((ee = hs::chol_enqueue(ca, h->s1, nullptr)) != cudaSuccess) return ee;
      } else {
        for (int m = 0; m < h->K; ++m)
          if ((ee = hs::chol_enqueue(chol_args(h, m), h->s1, nullptr)) != cudaSuccess) return ee;
      }
    }
    return cudaEventRecord(h->ev_join, h->s1);
  };
  if (!after_xstream && (e = factorize()) != cudaSuccess) return e;
  if (h->K == 1) {
    {
      ProfSpan sp(h, 0, h->s0);
      if ((e = hs::xstream_launch(h->x_dtype, xstream_args(h), h->grid, h->s0)) != cudaSuccess) return e;
    }
    {
      ProfSpan sp(h, 1, h->s0);
      if ((e = hs::reduce_partials_launch(h->x_dtype, h->partials, h->grid, h->ld, h->p, h->colscale, h->xtz,
                                          h->s0)) != cudaSuccess)
        return e;
    }
  } else if (h->xk) {
    const hs::XKArgs xa = xk_args(h);
    {
      ProfSpan sp(h, 0, h->s0);
      e = h->xk_split ? hs::xstream_k_split_enqueue(h->xmap, xa, h->beta, h->p, h->bsw, h->kgrid, h->s0)
                      : hs::xstream_k_enqueue(h->xmap, xa, h->beta, h->p, h->bsw, h->kgrid, h->s0);
      if (e != cudaSuccess) return e;
    }
    {
      ProfSpan sp(h, 1, h->s0);
      if ((e = hs::xstream_k_reduce(xa, h->kgrid, h->xtz, h->p, h->s0)) != cudaSuccess) return e;
    }
  } else {
    // K chains beyond the tensor-core X-stream (not BF16, or p past its TMEM
    // budget): one pass of the one-chain X-stream per chain
    const size_t part = (size_t)h->grid * h->ld * hs::partial_elem_bytes(h->x_dtype);
    const size_t bc = (size_t)h->ld * (h->x_dtype == HS_X_F64 ? 8 : 4);
    {
      ProfSpan sp(h, 0, h->s0);
      for (int m = 0; m < h->K && e == cudaSuccess; ++m) {
        hs::XStreamArgs a = xstream_args(h);
        a.beta_c = static_cast<const unsigned char*>(h->beta_c) + m * bc;
        a.partials = static_cast<unsigned char*>(h->partials) + m * part;
        a.z_out = h->cfg.debug ? h->z + (size_t)m * h->N : nullptr;
        a.rng.chain += (uint32_t)m;
        a.sm_mark = nullptr;
        e = hs::xstream_launch(h->x_dtype, a, h->grid, h->s0);
      }
      if (e != cudaSuccess) return e;
    }
    {
      ProfSpan sp(h, 1, h->s0);
      for (int m = 0; m < h->K && e == cudaSuccess; ++m)
        e = hs::reduce_partials_launch(h->x_dtype, static_cast<unsigned char*>(h->partials) + m * part, h->grid,
                                       h->ld, h->p, h->colscale, h->xtz + (size_t)m * h->p, h->s0);
      if (e != cudaSuccess) return e;
    }
  }
  if (noise_beside) {
    // the s and nu draws need lambda^{-2} only: beside the factorization
    if ((e = cudaStreamWaitEvent(h->s0, h->ev_shrink, 0)) != cudaSuccess) return e;
    if ((e = hs::tail_noise_enqueue(tail_args(h, 0), h->s0, h->K)) != cudaSuccess) return e;
  }
  if (after_xstream) {
    if ((e = cudaEventRecord(h->ev_xs, h->s0)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(h->s1, h->ev_xs, 0)) != cudaSuccess) return e;
    if ((e = factorize()) != cudaSuccess) return e;
  }
  if ((e = cudaStreamWaitEvent(h->s0, h->ev_join, 0)) != cudaSuccess) return e;
  {
    ProfSpan sp(h, 4, h->s0);
    if ((e = hs::tail_draw_enqueue(tail_args(h, 0), h->s0, h->K)) != cudaSuccess) return e;
    // every chain's commit reads the sweep count before the last one advances it
    if (h->K > 1 && (e = hs::commit_enqueue(tail_args(h, 0), h->s0, h->K - 1)) != cudaSuccess) return e;
    if ((e = hs::commit_enqueue(tail_args(h, h->K - 1), h->s0, 1)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t build_graph(hs_probit* h) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < kProfGroups && e == cudaSuccess; ++i)
    for (int j = 0; j < 2 && e == cudaSuccess; ++j)
      if (!h->placeholder[i][j]) e = cudaEventCreate(&h->placeholder[i][j]);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCapture(h->s0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  h->capturing = true;
  cudaError_t e2 = enqueue_sweep(h);
  h->capturing = false;
  e = cudaStreamEndCapture(h->s0, &g);
  if (e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return e2;
  }
  if (e != cudaSuccess) return e;
  // locate the event-record nodes of the profiling spans
  size_t n = 0;
  e = cudaGraphGetNodes(g, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  if (e == cudaSuccess && n) e = cudaGraphGetNodes(g, nodes.data(), &n);
  for (size_t q = 0; q < n && e == cudaSuccess; ++q) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nodes[q], &ty) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord) continue;
    cudaEvent_t ev = nullptr;
    if (cudaGraphEventRecordNodeGetEvent(nodes[q], &ev) != cudaSuccess) continue;
    for (int i = 0; i < kProfGroups; ++i)
      for (int j = 0; j < 2; ++j)
        if (ev == h->placeholder[i][j]) h->prof_node[i][j] = nodes[q];
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return e;
  }
  h->graph = g;
  h->graph_ready = true;
  return cudaSuccess;
}

// Before a graph launch while profiling: point the span nodes at fresh events.
cudaError_t arm_graph_events(hs_probit* h) {
  for (int i = 0; i < kProfGroups; ++i) {
    if (!h->prof_node[i][0] || !h->prof_node[i][1]) continue;
    cudaEvent_t e0 = h->take_event(), e1 = h->take_event();
    cudaError_t e = cudaGraphExecEventRecordNodeSetEvent(h->gexec, h->prof_node[i][0], e0);
    if (e == cudaSuccess) e = cudaGraphExecEventRecordNodeSetEvent(h->gexec, h->prof_node[i][1], e1);
    if (e != cudaSuccess) return e;
    h->pending.push_back({i, {e0, e1}});
  }
  return cudaSuccess;
}

void collect_profile(hs_probit* h) {
  for (auto& pe : h->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) {
      h->prof_ms[pe.first] += ms;
      h->prof_n[pe.first] += 1;
    }
    h->ev_pool.push_back(pe.second.first);
    h->ev_pool.push_back(pe.second.second);
  }
  h->pending.clear();
  (void)cudaGetLastError();
}

void destroy(hs_probit* h) {
  if (!h) return;
  if (h->s0) cudaStreamSynchronize(h->s0);
  if (h->s1) cudaStreamSynchronize(h->s1);
  if (h->s_dl) cudaStreamSynchronize(h->s_dl);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  for (int i = 0; i < kProfGroups; ++i)
    for (int j = 0; j < 2; ++j)
      if (h->placeholder[i][j]) cudaEventDestroy(h->placeholder[i][j]);
  for (auto& pe : h->pending) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_shrink) cudaEventDestroy(h->ev_shrink);
  if (h->ev_xs) cudaEventDestroy(h->ev_xs);
  if (h->ev_mark) cudaEventDestroy(h->ev_mark);
  if (h->ev_dl) cudaEventDestroy(h->ev_dl);
  if (h->s_dl) cudaStreamDestroy(h->s_dl);
  for (void* p : h->allocs) cudaFree(p);
  if (h->h_err) cudaFreeHost(h->h_err);
  if (h->h_k) cudaFreeHost(h->h_k);
  if (h->s1) cudaStreamDestroy(h->s1);
  if (h->own_s0 && h->s0) cudaStreamDestroy(h->s0);
  (void)cudaGetLastError();
  delete h;
}

// Before n_iter more sweeps are enqueued on stream s: if they would write a
// ring slot that a side-stream copy may still be reading, s waits for the
// copies first.
cudaError_t guard_ring(hs_probit* h, int64_t n_iter, cudaStream_t s) {
  if (h->dl_oldest < 0) return cudaSuccess;
  if (cudaEventQuery(h->ev_dl) == cudaSuccess) {
    h->dl_oldest = -1;
    return cudaSuccess;
  }
  (void)cudaGetLastError();  // cudaErrorNotReady
  const int64_t newest_after = (h->k_host + n_iter) / h->thin;
  if (newest_after - h->dl_oldest + 1 <= h->ring_size) return cudaSuccess;
  return cudaStreamWaitEvent(s, h->ev_dl, 0);
}

int sync_and_check(hs_probit* h) {
  cudaError_t e = cudaMemcpyAsync(h->h_err, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->s0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_k, h->k_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, h->s0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s0);
  if (e != cudaSuccess) return cuda_status(e);
  h->k_host = *h->h_k;
  h->last_err_word = *h->h_err;
  if (*h->h_err) return status_from_err_bits(*h->h_err);
  return HS_OK;
}

}  // namespace

extern "C" {

void hs_probit_config_default(hs_probit_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->x_dtype = HS_X_F32;
  cfg->x_is_device = 0;
  cfg->thin = 1;
  cfg->ring_size = 1024;
  cfg->debug = 0;
  cfg->use_graph = 0;
  cfg->chol_arith = HS_CHOL_DF32;
  cfg->chol_sched = HS_SCHED_AUTO;
  cfg->num_chains = 1;
  cfg->device = 0;
}

int hs_probit_last_error(void) { return g_last_error; }

const char* hs_probit_status_string(int status) {
  switch (status) {
    case HS_OK: return "ok";
    case HS_EINVAL: return "invalid argument";
    case HS_ENOMEM: return "out of memory";
    case HS_ECUDA: return "CUDA runtime error";
    case HS_ENOTPD: return "precision matrix not positive definite";
    case HS_ENONFINITE: return "non-finite value in the sweep";
    case HS_ETIMEOUT: return "bounded device wait ran out";
    case HS_ESTATE: return "handle in error state (call hs_probit_set_state)";
    case HS_EUNSUPPORTED: return "unsupported option";
  }
  return "unknown status";
}

static hs_probit* init_ex_impl(const hs_probit_config* cfg_in, const void* X, const uint8_t* y, int64_t N,
                               int64_t p, uint64_t seed) {
  g_last_error = HS_OK;
  hs_probit_config cfg;
  if (cfg_in)
    cfg = *cfg_in;
  else
    hs_probit_config_default(&cfg);
  // ---- argument checks (host only, before any CUDA call) ----
  if (!X || !y || N < 2 || p < 1 || p > kMaxP || cfg.thin < 1 || cfg.ring_size < 1 ||
      cfg.chain >= (1u << 24) || (cfg.x_dtype < HS_X_F64 || cfg.x_dtype > HS_X_FP8E4M3) ||
      (cfg.chol_arith != HS_CHOL_F64 && cfg.chol_arith != HS_CHOL_DF32) || N > (int64_t)0xFFFFFFFF ||
      cfg.chol_sched < HS_SCHED_AUTO || cfg.chol_sched > HS_SCHED_TENSOR || cfg.beta_solve < HS_BETA_AUTO ||
      cfg.beta_solve > HS_BETA_SUBST) {
    fail(HS_EINVAL);
    return nullptr;
  }
  if (cfg.x_dtype == HS_X_FP8E4M3 && !cfg.x_scales) {
    fail(HS_EINVAL);
    return nullptr;
  }
  // K chains (num_chains > 1): BF16 X on the tensor-core X-stream, chain ids chain .. chain+K-1
  const int Kc = cfg.num_chains > 1 ? cfg.num_chains : 1;
  if (cfg.num_chains < 0 || Kc > 32 || (uint64_t)cfg.chain + (uint64_t)Kc > (1u << 24)) {
    fail(HS_EINVAL);
    return nullptr;
  }

  {
    // The X-stream takes at most 2048 16-byte slices per row (p <= 4096 for FP64 X).
    const int64_t eb = cfg.x_dtype == HS_X_F64 ? 8 : cfg.x_dtype == HS_X_F32 ? 4 : cfg.x_dtype == HS_X_BF16 ? 2 : 1;
    const int64_t ve = 16 / eb;
    if ((p + ve - 1) / ve > 2048) {
      fail(HS_EINVAL);
      return nullptr;
    }
    // an adopted X is the library's row layout as it stands: rows of whole
    // 16-byte slices (no pad columns) from a 16-byte aligned base
    if (cfg.x_is_device < 0 || cfg.x_is_device > HS_X_ADOPT ||
        (cfg.x_is_device == HS_X_ADOPT && ((p * eb) % 16 != 0 || (reinterpret_cast<uintptr_t>(X) & 15u) != 0)) ||
        (cfg.update_mask & ~(HS_UPD_LAMBDA | HS_UPD_TAU | HS_UPD_NU | HS_UPD_XI)) != 0) {
      fail(HS_EINVAL);
      return nullptr;
    }
  }
  if (!cfg.x_is_device) {
    for (int64_t i = 0; i < N; ++i)
      if (y[i] > 1) {
        fail(HS_EINVAL);
        return nullptr;
      }
    if (cfg.x_dtype == HS_X_FP8E4M3)
      for (int64_t j = 0; j < p; ++j)
        if (!(std::isfinite(cfg.x_scales[j]) && cfg.x_scales[j] > 0.f)) {
          fail(HS_EINVAL);
          return nullptr;
        }
  }
  DeviceGuard dg(cfg.device);
  if (!dg.ok) {
    fail(HS_ECUDA);
    return nullptr;
  }
  hs_probit* h = new (std::nothrow) hs_probit();
  if (!h) {
    fail(HS_ENOMEM);
    return nullptr;
  }
  h->cfg = cfg;
  h->K = Kc;
  h->xk_kc = hs::xstream_k_default_kc(Kc);
  h->xk_stages = hs::kXkDefaultStages;
  {
    // K chains on the tensor cores: the fused kernel for BF16 X within its
    // TMEM budget, else the split form (BF16 or FP8 X)
    const bool fused = cfg.x_dtype == HS_X_BF16 && hs::xstream_k_supported((int)p, h->xk_kc, h->xk_stages, 1);
    const bool split = (cfg.x_dtype == HS_X_BF16 || cfg.x_dtype == HS_X_FP8E4M3) &&
                       hs::xstream_k_split_supported((int)p, h->xk_kc);
    h->xk = Kc > 1 && (fused || split);
    h->xk_split = h->xk && !fused;
    if (h->xk_split) h->xk_stages = hs::xstream_k_split_stages(h->xk_kc);
  }
  h->drained.assign((size_t)Kc, 0);
  h->device = cfg.device;
  h->x_dtype = cfg.x_dtype;
  h->N = N;
  h->p = (int)p;
  h->elem = elem_bytes_of(cfg.x_dtype);
  const int ve = 16 / h->elem;
  h->ld = (int)((p + ve - 1) / ve * ve);
  h->T = (int)((p + 31) / 32);
  h->P = h->T * 32;
  h->rng = hs::RngKey{(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32), cfg.chain, cfg.problem};
  h->ring_size = cfg.ring_size;
  h->thin = cfg.thin;

  cudaError_t e = cudaSuccess;
  auto check = [&](cudaError_t ee) {
    if (e == cudaSuccess && ee != cudaSuccess) e = ee;
    return e == cudaSuccess;
  };
  int num_sms = 0;
  check(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, h->device));
  check(hs::xstream_prepare());
  check(hs::linalg_prepare());
  if (e == cudaSuccess && cfg.chol_arith == HS_CHOL_DF32 && cfg.chol_sched != HS_SCHED_COLUMNS) {
    h->chol_grid = hs::chol_persistent_grid(h->device, Kc);
    if (h->chol_grid == 0 && (cfg.chol_sched == HS_SCHED_SINGLE || cfg.chol_sched == HS_SCHED_TENSOR)) {
      destroy(h);
      fail(HS_EUNSUPPORTED);
      return nullptr;
    }
  }
  // beta by substitution needs the single-launch schedule's inverse-free mode
  if (e == cudaSuccess && cfg.beta_solve == HS_BETA_SUBST && h->chol_grid == 0) {
    destroy(h);
    fail(HS_EUNSUPPORTED);
    return nullptr;
  }
  // AUTO: the factorization is throughput-bound for several chains or a large p
  // (measured: one chain at p = 4000, N = 5e5: 65 -> 108 sweeps/s with substitution;
  // at p = 1000 its diagonal chain bounds it and the inverse products win)
  h->chol_inverse = !(h->chol_grid > 0 && (cfg.beta_solve == HS_BETA_SUBST ||
                                          (cfg.beta_solve == HS_BETA_AUTO && (h->K > 1 || h->T >= 64))));
  // the tensor-core trailing updates: where the factorization is throughput-bound
  // (several chains, or a large p), factor only
  h->tensor_sched = h->chol_grid > 0 && cfg.chol_arith == HS_CHOL_DF32 &&
                    (cfg.chol_sched == HS_SCHED_TENSOR ||
                     (cfg.chol_sched == HS_SCHED_AUTO && !h->chol_inverse && (h->K > 1 || h->T >= 64)));
  if (h->tensor_sched && h->chol_inverse) {
    if (cfg.beta_solve == HS_BETA_INVERSE) {
      destroy(h);
      fail(HS_EUNSUPPORTED);
      return nullptr;
    }
    h->chol_inverse = false;
  }
  if (cfg.stream) {
    h->s0 = static_cast<cudaStream_t>(cfg.stream);
  } else {
    check(cudaStreamCreateWithFlags(&h->s0, cudaStreamNonBlocking));
    h->own_s0 = true;
  }
  check(cudaStreamCreateWithFlags(&h->s1, cudaStreamNonBlocking));
  check(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  check(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  check(cudaEventCreateWithFlags(&h->ev_shrink, cudaEventDisableTiming));
  check(cudaEventCreateWithFlags(&h->ev_xs, cudaEventDisableTiming));
  const size_t P2 = (size_t)h->P * h->P;
  const size_t pd = (size_t)p * sizeof(double);
  const size_t K = (size_t)h->K;
  const size_t bc_bytes = (size_t)h->ld * (h->x_dtype == HS_X_F64 ? 8 : 4);
  h->grid = hs::xstream_grid(h->x_dtype, h->p, h->ld, N, num_sms > 0 ? num_sms : 1);
  if (h->xk_split) {
    check(hs::xstream_k_split_prepare(h->xk_kc, cfg.x_dtype == HS_X_FP8E4M3 ? 1 : 0));
    // both widths, so that a tuner may switch
    if (hs::xstream_k_split_supported((int)p, 32))
      check(hs::xstream_k_split_prepare(32, cfg.x_dtype == HS_X_FP8E4M3 ? 1 : 0));
    h->kgrid = hs::xstream_k_grid(N, num_sms > 0 ? num_sms : 1);
  } else if (h->xk) {
    check(hs::xstream_k_prepare(h->xk_kc, h->xk_stages, 1));
    h->kgrid = hs::xstream_k_grid(N, num_sms > 0 ? num_sms : 1);
  }
  h->chol_words = hs::chol_sync_words(h->P);
  if (cfg.x_is_device == HS_X_ADOPT)
    h->X = const_cast<void*>(X);  // the caller's buffer, never freed here
  else
    check(h->alloc(&h->X, (size_t)N * h->ld * h->elem));
  check(h->alloc(&h->y, (size_t)N));
  if (cfg.x_dtype == HS_X_FP8E4M3) check(h->alloc(&h->colscale, (size_t)p * sizeof(float)));
  check(h->alloc(&h->beta, K * pd));
  check(h->alloc(&h->lam, K * pd));
  check(h->alloc(&h->nu, K * pd));
  check(h->alloc(&h->scal, K * 2 * sizeof(double)));
  check(h->alloc(&h->k_dev, sizeof(int64_t)));
  check(h->alloc(&h->k_scratch, K * sizeof(int64_t)));
  check(h->alloc(&h->lam_new, K * pd));
  check(h->alloc(&h->tau_new, K * sizeof(double)));
  check(h->alloc(&h->beta_new, K * pd));
  check(h->alloc(&h->nu_new, K * pd));
  check(h->alloc(&h->beta_c, K * bc_bytes));
  check(h->alloc(&h->G, (size_t)p * p * sizeof(double)));
  check(h->alloc(&h->S, K * (size_t)h->P * sizeof(double)));
  check(h->alloc(&h->A, K * P2 * sizeof(double)));
  check(h->alloc(&h->Linv, K * P2 * sizeof(double)));
  check(h->alloc(&h->LinvT, K * P2 * sizeof(double)));
  check(h->alloc(&h->xtz, K * pd));
  check(h->alloc(&h->v, K * (size_t)h->P * sizeof(double)));
  check(h->alloc(&h->shrink_part, K * (shrink_blocks(h) + 1) * sizeof(double)));
  check(h->alloc(&h->shrink_ticket, K * sizeof(unsigned int)));
  std::vector<int> order;
  if (h->chol_grid > 0) {
    check(h->alloc(&h->chol_sync, K * h->chol_words * sizeof(unsigned long long)));
    check(h->alloc(&h->sm_mark, hs::kSmMarks * sizeof(unsigned int)));
    order = single_task_list(h);
    h->chol_ntasks = (int)order.size();
    if (!order.empty()) check(h->alloc(&h->chol_order, order.size() * sizeof(int)));
  }
  if (h->tensor_sched) {
    check(hs::chol_trail_prepare());
    check(h->alloc(&h->digits, K * 6 * P2 * sizeof(uint16_t)));
    check(h->alloc(&h->sm_role, 2 * hs::kSmMarks * sizeof(unsigned long long)));
    if (e == cudaSuccess) check(cudaMemset(h->sm_role, 0, 2 * hs::kSmMarks * sizeof(unsigned long long)));
    check(h->alloc(&h->G2, P2 * 2 * sizeof(float)));
    const std::vector<int> all = block_task_lists(h);
    check(h->alloc(&h->blk_order, std::max<size_t>(all.size(), 1) * sizeof(int)));
    if (e == cudaSuccess && !all.empty())
      check(cudaMemcpy(h->blk_order, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (e == cudaSuccess && hs::chol_trail_make_maps(h->digits, h->P, h->K, h->tmapA, h->tmapB) != 0)
      e = cudaErrorInvalidValue;
    h->trail_grid = num_sms > 0 ? num_sms : 1;
  }
  if (!h->xk) {
    check(h->alloc(&h->partials, K * h->grid * h->ld * hs::partial_elem_bytes(h->x_dtype)));
  } else {
    // sized for the widest launch shape (32 chain columns), so a tuner may switch
    check(h->alloc(&h->bsw, hs::xstream_k_bsw_bytes(h->p, 32)));
    if (h->xk_split)
      check(h->alloc(&h->zt, hs::xstream_k_zt_bytes(N, hs::xstream_k_split_supported(h->p, 32) ? 32 : h->xk_kc)));
    check(h->alloc(&h->kpartials, hs::xstream_k_partial_floats(h->p, h->kgrid, 32) * sizeof(float)));
  }
  if (cfg.debug) check(h->alloc(&h->z, K * (size_t)N * sizeof(double)));
  check(h->alloc(&h->ring_beta, K * (size_t)h->ring_size * pd));
  check(h->alloc(&h->ring_lam, K * (size_t)h->ring_size * pd));
  check(h->alloc(&h->ring_tau, K * (size_t)h->ring_size * sizeof(double)));
  check(h->alloc(&h->err, sizeof(int)));
  check(h->alloc(&h->hook_err, sizeof(int)));
  check(h->alloc(&h->hook_flag, sizeof(int)));
  if (e == cudaSuccess) check(cudaMallocHost(&h->h_err, sizeof(int)));
  if (e == cudaSuccess) check(cudaMallocHost(&h->h_k, sizeof(int64_t)));
  if (e != cudaSuccess) {
    int st = cuda_status(e);
    destroy(h);
    fail(st);
    return nullptr;
  }
  // ---- data ----
  const cudaMemcpyKind kind = cfg.x_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (cfg.x_is_device != HS_X_ADOPT) {
    check(cudaMemsetAsync(h->X, 0, (size_t)N * h->ld * h->elem, h->s0));
    check(cudaMemcpy2DAsync(h->X, (size_t)h->ld * h->elem, X, (size_t)p * h->elem, (size_t)p * h->elem, (size_t)N,
                            kind, h->s0));
  }
  check(cudaMemcpyAsync(h->y, y, (size_t)N, kind, h->s0));
  if (h->colscale) check(cudaMemcpyAsync(h->colscale, cfg.x_scales, (size_t)p * sizeof(float), kind, h->s0));
  check(cudaMemsetAsync(h->err, 0, sizeof(int), h->s0));
  check(cudaMemsetAsync(h->hook_err, 0, sizeof(int), h->s0));
  check(cudaMemsetAsync(h->shrink_ticket, 0, K * sizeof(unsigned int), h->s0));
  if (h->chol_order && e == cudaSuccess)
    check(cudaMemcpy(h->chol_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (h->chol_sync) {
    check(cudaMemsetAsync(h->chol_sync, 0, K * h->chol_words * sizeof(unsigned long long), h->s0));
    check(cudaMemsetAsync(h->sm_mark, 0, hs::kSmMarks * sizeof(unsigned int), h->s0));
  }
  if (h->xk && e == cudaSuccess &&
      (h->x_dtype == HS_X_FP8E4M3 ? hs::xstream_k_make_map_fp8(h->X, N, h->ld, h->xmap)
                                  : hs::xstream_k_make_map(h->X, N, h->ld, h->xmap)) != 0)
    e = cudaErrorInvalidValue;
  if (cfg.x_is_device) check(hs::check_y_launch(h->y, N, h->err, h->s0));
  // ---- cold start (Sect. 6.1): beta = 0, lambda = nu = tau = xi = 1, k = 0, every chain ----
  {
    std::vector<double> ones(K * (size_t)p, 1.0), sc(2 * K, 1.0);
    const int64_t k0 = 0;
    check(cudaMemsetAsync(h->beta, 0, K * pd, h->s0));
    check(cudaMemcpyAsync(h->lam, ones.data(), K * pd, cudaMemcpyHostToDevice, h->s0));
    check(cudaMemcpyAsync(h->nu, ones.data(), K * pd, cudaMemcpyHostToDevice, h->s0));
    check(cudaMemcpyAsync(h->scal, sc.data(), 2 * K * sizeof(double), cudaMemcpyHostToDevice, h->s0));
    check(cudaMemcpyAsync(h->k_dev, &k0, sizeof(k0), cudaMemcpyHostToDevice, h->s0));
    check(cudaMemsetAsync(h->beta_c, 0, K * bc_bytes, h->s0));
    check(cudaStreamSynchronize(h->s0));  // host staging buffers go out of scope
  }
  // ---- one-time Gram matrix (Sect. 5, beta update, step i), tensor cores ----
  void* gram_ws = nullptr;
  check(cudaMalloc(&gram_ws, hs::gram_workspace_bytes(N, h->p, num_sms > 0 ? num_sms : 1)));
  {
    ProfSpan sp(h, 5, h->s0);
    check(hs::gram_launch(h->x_dtype, h->X, N, h->ld, h->p, h->colscale, h->G, gram_ws, num_sms > 0 ? num_sms : 1,
                          h->err, h->s0));
  }
  if (h->tensor_sched) check(hs::gram_pairs_launch(h->G, h->p, h->P, h->G2, h->s0));
  if (e == cudaSuccess) {
    const int st = sync_and_check(h);
    cudaFree(gram_ws);
    gram_ws = nullptr;
    if (st != HS_OK) {
      destroy(h);
      fail(st);
      return nullptr;
    }
  }
  if (gram_ws) {
    cudaStreamSynchronize(h->s0);
    cudaFree(gram_ws);
  }
  if (e != cudaSuccess) {
    int st = cuda_status(e);
    destroy(h);
    fail(st);
    return nullptr;
  }
  // per chain: shrink, the factorization, two draws, commit; then the X-stream and its reduce
  int64_t chol_l = hs::chol_launch_count(h->P, h->cfg.chol_arith, h->chol_grid);
  if (h->tensor_sched) {
    chol_l = 1;  // the precision matrix in pairs

    for (int b = 0; b < (int)h->blk_off.size(); ++b)
      chol_l += 1 + (hs::chol_trail_items(h->P, b, 0, h->T, h->K) > 0 ? 1 : 0);
  }
  // shrink, factorization (one launch for every chain when single-launch), two draws, commits
  h->launches = 1 + ((h->K > 1 && h->chol_grid > 0) ? chol_l : h->K * chol_l) + 2 +
                (h->K > 1 ? 2 : 1) +
                (h->K == 1 ? 2 : h->xk_split ? 4 : h->xk ? 3 : 2 * h->K);
  h->grid_max = h->grid;
  h->kgrid_max = h->kgrid;
  h->trail_max = h->trail_grid;
  h->chol_max = h->chol_grid;
  return h;
}

hs_probit* hs_probit_init(const float* X, const uint8_t* y, int64_t N, int64_t p, uint64_t seed) {
  hs_probit_config cfg;
  hs_probit_config_default(&cfg);
  return hs_probit_init_ex(&cfg, X, y, N, p, seed);
}

// No C++ exception leaves the C ABI: the host-side containers that can throw
// std::bad_alloc are caught here and reported as HS_ENOMEM.
hs_probit* hs_probit_init_ex(const hs_probit_config* cfg_in, const void* X, const uint8_t* y, int64_t N,
                             int64_t p, uint64_t seed) {
  try {
    return init_ex_impl(cfg_in, X, y, N, p, seed);
  } catch (...) {
    g_last_error = HS_ENOMEM;
    return nullptr;
  }
}

static int sweep_impl(hs_probit* h, int64_t n_iter) {
  if (!h || n_iter < 0) return HS_EINVAL;
  if (h->sticky != HS_OK) return HS_ESTATE;
  if (n_iter == 0) return HS_OK;
  DeviceGuard dg(h->device);
  if (!dg.ok) return HS_ECUDA;
  cudaError_t e = cudaSuccess;
  const bool graph = h->cfg.use_graph != 0;
  if (graph && !h->graph_ready) {
    e = build_graph(h);
    if (e != cudaSuccess) return cuda_status(e);
  }
  e = guard_ring(h, n_iter, h->s0);
  for (int64_t i = 0; i < n_iter && e == cudaSuccess; ++i) {
    if (graph) {
      if (h->profiling) e = arm_graph_events(h);
      if (e == cudaSuccess) e = cudaGraphLaunch(h->gexec, h->s0);
    } else {
      e = enqueue_sweep(h);
    }
  }
  if (e != cudaSuccess) {
    cudaStreamSynchronize(h->s0);
    return cuda_status(e);
  }
  const int st = sync_and_check(h);
  if (h->profiling) {
    cudaStreamSynchronize(h->s1);
    collect_profile(h);
  }
  if (st != HS_OK) h->sticky = st;
  return st;
}

int64_t hs_probit_draws_available_chain(const hs_probit* h, int chain) {
  if (!h || chain < 0 || chain >= h->K) return HS_EINVAL;
  const int64_t newest = h->k_host / h->thin;
  int64_t first = h->drained[chain] + 1;
  if (newest - first + 1 > h->ring_size) first = newest - h->ring_size + 1;
  return newest >= first ? newest - first + 1 : 0;
}

int64_t hs_probit_draws_available(const hs_probit* h) { return hs_probit_draws_available_chain(h, 0); }

int64_t hs_probit_draws_chain(hs_probit* h, int chain, double* beta, double* lambda_inv2, double* tau_inv2,
                              int64_t max_draws) {
  if (!h || max_draws < 0 || chain < 0 || chain >= h->K) return HS_EINVAL;
  DeviceGuard dg(h->device);
  if (!dg.ok) return HS_ECUDA;
  if (cudaStreamSynchronize(h->s0) != cudaSuccess) return HS_ECUDA;
  const int64_t newest = h->k_host / h->thin;
  int64_t first = h->drained[chain] + 1;
  if (newest - first + 1 > h->ring_size) first = newest - h->ring_size + 1;
  int64_t count = newest >= first ? newest - first + 1 : 0;
  if (count > max_draws) count = max_draws;
  const size_t p = (size_t)h->p;
  const double* rb = h->ring_beta + (size_t)chain * h->ring_size * p;
  const double* rl = h->ring_lam + (size_t)chain * h->ring_size * p;
  const double* rt = h->ring_tau + (size_t)chain * h->ring_size;
  for (int64_t d = 0; d < count;) {
    const int64_t slot = (first + d - 1) % h->ring_size;
    int64_t run = h->ring_size - slot;
    if (run > count - d) run = count - d;
    cudaError_t e = cudaSuccess;
    if (beta) e = cudaMemcpy(beta + d * p, rb + slot * p, run * p * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && lambda_inv2)
      e = cudaMemcpy(lambda_inv2 + d * p, rl + slot * p, run * p * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && tau_inv2)
      e = cudaMemcpy(tau_inv2 + d, rt + slot, run * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return HS_ECUDA;
    d += run;
  }
  h->drained[chain] = first + count - 1;
  return count;
}

int64_t hs_probit_draws_async(hs_probit* h, int chain, double* beta, double* lambda_inv2, double* tau_inv2,
                              int64_t max_draws) {
  if (!h || max_draws < 0 || chain < 0 || chain >= h->K) return HS_EINVAL;
  DeviceGuard dg(h->device);
  if (!dg.ok) return HS_ECUDA;
  cudaError_t e = cudaSuccess;
  if (!h->s_dl) {
    e = cudaStreamCreateWithFlags(&h->s_dl, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_mark, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_dl, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e);
  }
  // the copies follow everything enqueued on the sweep stream so far
  e = cudaEventRecord(h->ev_mark, h->s0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_dl, h->ev_mark, 0);
  if (e != cudaSuccess) return cuda_status(e);
  const int64_t newest = h->k_host / h->thin;
  int64_t first = h->drained[chain] + 1;
  if (newest - first + 1 > h->ring_size) first = newest - h->ring_size + 1;
  int64_t count = newest >= first ? newest - first + 1 : 0;
  if (count > max_draws) count = max_draws;
  const size_t p = (size_t)h->p;
  const double* rb = h->ring_beta + (size_t)chain * h->ring_size * p;
  const double* rl = h->ring_lam + (size_t)chain * h->ring_size * p;
  const double* rt = h->ring_tau + (size_t)chain * h->ring_size;
  for (int64_t d = 0; d < count && e == cudaSuccess;) {
    const int64_t slot = (first + d - 1) % h->ring_size;
    int64_t run = h->ring_size - slot;
    if (run > count - d) run = count - d;
    if (beta)
      e = cudaMemcpyAsync(beta + d * p, rb + slot * p, run * p * sizeof(double), cudaMemcpyDeviceToHost, h->s_dl);
    if (e == cudaSuccess && lambda_inv2)
      e = cudaMemcpyAsync(lambda_inv2 + d * p, rl + slot * p, run * p * sizeof(double), cudaMemcpyDeviceToHost,
                          h->s_dl);
    if (e == cudaSuccess && tau_inv2)
      e = cudaMemcpyAsync(tau_inv2 + d, rt + slot, run * sizeof(double), cudaMemcpyDeviceToHost, h->s_dl);
    d += run;
  }
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_dl, h->s_dl);
  if (e != cudaSuccess) return cuda_status(e);
  if (count > 0) h->dl_oldest = h->dl_oldest < 0 ? first : std::min(h->dl_oldest, first);
  h->drained[chain] = first + count - 1;
  return count;
}

int hs_probit_draws_wait(hs_probit* h) {
  if (!h) return HS_EINVAL;
  if (!h->ev_dl) return HS_OK;
  DeviceGuard dg(h->device);
  if (!dg.ok) return HS_ECUDA;
  if (cudaEventSynchronize(h->ev_dl) != cudaSuccess) return HS_ECUDA;
  h->dl_oldest = -1;
  return HS_OK;
}

int64_t hs_probit_draws(hs_probit* h, double* beta, double* lambda_inv2, double* tau_inv2, int64_t max_draws) {
  return hs_probit_draws_chain(h, 0, beta, lambda_inv2, tau_inv2, max_draws);
}

int hs_probit_num_chains(const hs_probit* h) { return h ? h->K : HS_EINVAL; }

int hs_probit_get_state_chain(const hs_probit* hc, int chain, hs_probit_state_view* out) {
  hs_probit* h = const_cast<hs_probit*>(hc);
  if (!h || !out || chain < 0 || chain >= h->K) return HS_EINVAL;
  DeviceGuard dg(h->device);
  if (!dg.ok) return HS_ECUDA;
  if (cudaStreamSynchronize(h->s0) != cudaSuccess) return HS_ECUDA;
  const size_t pd = (size_t)h->p * sizeof(double), off = (size_t)chain * h->p;
  cudaError_t e = cudaSuccess;
  if (out->beta) e = cudaMemcpy(out->beta, h->beta + off, pd, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && out->lambda_inv2)
    e = cudaMemcpy(out->lambda_inv2, h->lam + off, pd, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && out->nu_inv) e = cudaMemcpy(out->nu_inv, h->nu + off, pd, cudaMemcpyDeviceToHost);
  double sc[2] = {0, 0};
  int64_t k = 0;
  if (e == cudaSuccess) e = cudaMemcpy(sc, h->scal + 2 * chain, sizeof(sc), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&k, h->k_dev, sizeof(k), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return HS_ECUDA;
  out->tau_inv2 = sc[0];
  out->xi_inv = sc[1];
  out->k = k;
  return HS_OK;
}

int hs_probit_get_state(const hs_probit* h, hs_probit_state_view* out) { return hs_probit_get_state_chain(h, 0, out); }

int hs_probit_set_state_chain(hs_probit* h, int chain, const hs_probit_state_view* in) {
  if (!h || !in || !in->beta || !in->lambda_inv2 || !in->nu_inv || in->k < 0 || !std::isfinite(in->tau_inv2) ||
      !std::isfinite(in->xi_inv) || in->k >= (int64_t)0xFFFFFFFF || chain < 0 || chain >= h->K)
    return HS_EINVAL;
  DeviceGuard dg(h->device);
  if (!dg.ok) return HS_ECUDA;
  if (cudaStreamSynchronize(h->s0) != cudaSuccess) return HS_ECUDA;
  if (cudaStreamSynchronize(h->s1) != cudaSuccess) return HS_ECUDA;
  const size_t pd = (size_t)h->p * sizeof(double), off = (size_t)chain * h->p;
  const double sc[2] = {in->tau_inv2, in->xi_inv};
  const int64_t k = in->k;
  const size_t bc_bytes = (size_t)h->ld * (h->x_dtype == HS_X_F64 ? 8 : 4);
  cudaError_t e = cudaMemcpy(h->beta + off, in->beta, pd, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->lam + off, in->lambda_inv2, pd, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->nu + off, in->nu_inv, pd, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->scal + 2 * chain, sc, sizeof(sc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->k_dev, &k, sizeof(k), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(h->err, 0, sizeof(int));
  if (e == cudaSuccess)
    e = hs::beta_c_launch(h->beta + off, h->colscale, h->p, h->ld,
                          static_cast<unsigned char*>(h->beta_c) + (size_t)chain * bc_bytes,
                          h->x_dtype == HS_X_F64 ? 1 : 0, h->s0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s0);
  if (e != cudaSuccess) return HS_ECUDA;
  h->sticky = HS_OK;
  h->k_host = k;
  for (auto& d : h->drained) d = k / h->thin;
  return HS_OK;
}

int hs_probit_set_state(hs_probit* h, const hs_probit_state_view* in) { return hs_probit_set_state_chain(h, 0, in); }

int hs_probit_debug_z_chain(hs_probit* h, int chain, double* z_out) {
  if (!h || !z_out || chain < 0 || chain >= h->K) return HS_EINVAL;
  if (!h->cfg.debug) return HS_EUNSUPPORTED;
  DeviceGuard dg(h->device);
  if (cudaStreamSynchronize(h->s0) != cudaSuccess) return HS_ECUDA;
  return cuda_status(cudaMemcpy(z_out, h->z + (size_t)chain * h->N, (size_t)h->N * sizeof(double),
                                cudaMemcpyDeviceToHost));
}

int hs_probit_debug_z(hs_probit* h, double* z_out) { return hs_probit_debug_z_chain(h, 0, z_out); }

int hs_probit_debug_xtz_chain(hs_probit* h, int chain, double* xtz_out) {
  if (!h || !xtz_out || chain < 0 || chain >= h->K) return HS_EINVAL;
  if (!h->cfg.debug) return HS_EUNSUPPORTED;
  DeviceGuard dg(h->device);
  if (cudaStreamSynchronize(h->s0) != cudaSuccess) return HS_ECUDA;
  return cuda_status(cudaMemcpy(xtz_out, h->xtz + (size_t)chain * h->p, (size_t)h->p * sizeof(double),
                                cudaMemcpyDeviceToHost));
}

int hs_probit_debug_xtz(hs_probit* h, double* xtz_out) { return hs_probit_debug_xtz_chain(h, 0, xtz_out); }

int hs_probit_gram(hs_probit* h, double* G_out) {
  if (!h || !G_out) return HS_EINVAL;
  DeviceGuard dg(h->device);
  if (cudaStreamSynchronize(h->s0) != cudaSuccess) return HS_ECUDA;
  return cuda_status(
      cudaMemcpy(G_out, h->G, (size_t)h->p * h->p * sizeof(double), cudaMemcpyDeviceToHost));
}

int hs_probit_info(const hs_probit* h, int64_t* N, int64_t* p, void** stream) {
  if (!h) return HS_EINVAL;
  if (N) *N = h->N;
  if (p) *p = h->p;
  if (stream) *stream = (void*)h->s0;
  return HS_OK;
}

int hs_probit_sweep(hs_probit* h, int64_t n_iter) {
  try {
    return sweep_impl(h, n_iter);
  } catch (...) {
    return HS_ENOMEM;
  }
}

int hs_probit_set_profiling(hs_probit* h, int on) {
  if (!h) return HS_EINVAL;
  h->profiling = on ? 1 : 0;
  for (int i = 0; i < kProfGroups; ++i) {
    if (on) {
      h->prof_ms[i] = 0;
      h->prof_n[i] = 0;
    }
  }
  return HS_OK;
}

int hs_probit_kernel_time(hs_probit* h, int which, double* total_ms, int64_t* launches) {
  if (!h || which < 0 || which >= kProfGroups) return HS_EINVAL;
  if (total_ms) *total_ms = h->prof_ms[which];
  if (launches) *launches = h->prof_n[which];
  return HS_OK;
}

int64_t hs_probit_launches_per_sweep(const hs_probit* h) {
  if (!h) return HS_EINVAL;
  return h->launches;
}

int64_t hs_chol_task_list(int32_t T, int32_t workers, int32_t inverse, int32_t* codes, int64_t max_codes) {
  if (T < 1 || T > 256 || workers < 1 || (inverse != 0 && inverse != 1) || max_codes < 0 ||
      (max_codes > 0 && !codes))
    return HS_EINVAL;
  try {
    const std::vector<int> list = hs::chol_task_codes(T, workers, inverse != 0);
    const int64_t n = (int64_t)list.size();
    for (int64_t t = 0; t < n && t < max_codes; ++t) codes[t] = list[(size_t)t];
    return n;
  } catch (...) {
    return HS_ENOMEM;
  }
}

int hs_probit_debug_factor(hs_probit* h, int chain, double* L_out) {
  if (!h || !L_out || chain < 0 || chain >= h->K) return HS_EINVAL;
  if (h->cfg.chol_arith != HS_CHOL_DF32) return HS_EUNSUPPORTED;
  DeviceGuard dg(h->device);
  if (cudaStreamSynchronize(h->s0) != cudaSuccess || cudaStreamSynchronize(h->s1) != cudaSuccess) return HS_ECUDA;
  const size_t P2 = (size_t)h->P * h->P;
  std::vector<float> pairs(2 * P2);
  if (cudaMemcpy(pairs.data(), h->A + chain * P2, P2 * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return HS_ECUDA;
  for (size_t e = 0; e < P2; ++e) L_out[e] = (double)pairs[2 * e] + (double)pairs[2 * e + 1];
  return HS_OK;
}

int hs_probit_get_launch_shape(const hs_probit* h, hs_launch_shape* out) {
  if (!h || !out) return HS_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->xk_chains = h->xk ? h->xk_kc : 0;
  out->xk_stages = h->xk ? h->xk_stages : 0;
  out->xk_ctas_per_sm = h->xk ? h->xk_per_sm : 0;
  out->overlap = (h->K == 1 || h->chol_grid == 0 || h->beside) ? 1 : 2;
  out->xstream_ctas = h->xk ? h->kgrid : h->grid;
  out->chol_ctas = h->chol_grid;
  out->trail_ctas = h->tensor_sched ? h->trail_grid : 0;
  return HS_OK;
}

int hs_probit_set_launch_shape(hs_probit* h, const hs_launch_shape* in) {
  if (!h || !in) return HS_EINVAL;
  for (int r : in->reserved)
    if (r != 0) return HS_EINVAL;
  const int kc = in->xk_chains ? in->xk_chains : h->xk_kc;
  const int st = h->xk_split ? hs::xstream_k_split_stages(kc) : in->xk_stages ? in->xk_stages : h->xk_stages;
  const int pm = in->xk_ctas_per_sm ? in->xk_ctas_per_sm : h->xk_per_sm;
  const int xs = in->xstream_ctas ? in->xstream_ctas : (h->xk ? h->kgrid : h->grid);
  const int cg = in->chol_ctas ? in->chol_ctas : h->chol_grid;
  const int tg = in->trail_ctas ? in->trail_ctas : h->trail_grid;
  if (in->xk_chains < 0 || in->xk_stages < 0 || in->xstream_ctas < 0 || in->chol_ctas < 0 || in->trail_ctas < 0 ||
      in->xk_ctas_per_sm < 0 || in->overlap < 0 || in->overlap > 2)
    return HS_EINVAL;
  if ((in->xk_chains || in->xk_stages || in->xk_ctas_per_sm) && !h->xk) return HS_EUNSUPPORTED;
  if (h->xk && kc < h->K) return HS_EINVAL;
  if (h->xk && h->xk_split &&
      (!hs::xstream_k_split_supported(h->p, kc) || pm != 1 || (in->xk_stages && in->xk_stages != st)))
    return HS_EINVAL;  // the split form has one tile shape per width
  if (h->xk && !h->xk_split && !hs::xstream_k_supported(h->p, kc, st, pm)) return HS_EINVAL;
  // the partial sums were sized for the starting grid at 32 chain columns
  const int64_t xs_max = h->xk ? std::min<int64_t>(hs::xstream_k_tiles(h->N), (int64_t)h->kgrid_max * 32 / kc)
                               : h->grid_max;
  if (xs < 1 || xs > xs_max) return HS_EINVAL;
  if (in->chol_ctas && (h->chol_grid == 0 || cg < h->K + 1 || cg > h->chol_max)) return HS_EINVAL;
  if (in->trail_ctas && (!h->tensor_sched || tg < 1 || tg > h->trail_max)) return HS_EINVAL;
  DeviceGuard dg(h->device);
  if (!dg.ok) return HS_ECUDA;
  if (cudaStreamSynchronize(h->s0) != cudaSuccess || cudaStreamSynchronize(h->s1) != cudaSuccess) return HS_ECUDA;
  if (h->xk && !h->xk_split && hs::xstream_k_prepare(kc, st, pm) != cudaSuccess) return HS_ECUDA;
  h->xk_kc = kc;
  h->xk_stages = st;
  h->xk_per_sm = pm;
  if (in->overlap) h->beside = in->overlap == 1;
  if (h->xk) h->kgrid = xs;
  else h->grid = xs;
  h->trail_grid = tg;
  if (cg != h->chol_grid) {
    // the task lists are ordered for the worker count; their lengths do not change
    h->chol_grid = cg;
    if (h->chol_order) {
      const std::vector<int> order = single_task_list(h);
      if ((int)order.size() != h->chol_ntasks) return HS_EINVAL;
      if (cudaMemcpy(h->chol_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        return HS_ECUDA;
    }
    if (h->blk_order) {
      const std::vector<int> all = block_task_lists(h);
      if (!all.empty() &&
          cudaMemcpy(h->blk_order, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        return HS_ECUDA;
    }
  }
  // a captured sweep holds the old shapes (a batch holding this problem recaptures on the epoch)
  ++h->shape_epoch;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->gexec = nullptr;
  h->graph = nullptr;
  h->graph_ready = false;
  return HS_OK;
}

int hs_probit_debug_error_word(const hs_probit* h, int* word) {
  if (!h || !word) return HS_EINVAL;
  *word = h->last_err_word;
  return HS_OK;
}

int64_t hs_chol_block_task_list(int32_t T, int32_t k0, int32_t k1, int32_t workers, int32_t* codes,
                                int64_t max_codes) {
  if (T < 1 || T > 256 || k0 < 0 || k1 <= k0 || k1 > T || workers < 1 || max_codes < 0 || (max_codes > 0 && !codes))
    return HS_EINVAL;
  try {
    const std::vector<int> list = hs::chol_block_task_codes(T, k0, k1, workers);
    const int64_t n = (int64_t)list.size();
    for (int64_t t = 0; t < n && t < max_codes; ++t) codes[t] = list[(size_t)t];
    return n;
  } catch (...) {
    return HS_ENOMEM;
  }
}

int hs_probit_debug_wait_timeout(hs_probit* h, int64_t max_spins) {
  if (!h || max_spins < 0) return HS_EINVAL;
  DeviceGuard dg(h->device);
  if (!dg.ok) return HS_ECUDA;
  int bits = 0;
  cudaError_t e = cudaMemsetAsync(h->hook_flag, 0, sizeof(int), h->s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->hook_err, 0, sizeof(int), h->s0);
  if (e == cudaSuccess) e = hs::wait_timeout_launch(h->hook_flag, max_spins, h->hook_err, h->s0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_err, h->hook_err, sizeof(int), cudaMemcpyDeviceToHost, h->s0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s0);
  if (e != cudaSuccess) return HS_ECUDA;
  bits = *h->h_err;
  return (bits & hs::kErrTimeout) ? HS_ETIMEOUT : HS_OK;
}

void hs_probit_free(hs_probit* h) {
  if (!h || h->batch_member) return;  // a batch's problems are released with the batch
  DeviceGuard dg(h->device);
  destroy(h);
}

}  // extern "C"

// ---- many problems in one launch (Sect. 4) ------------------------------------
struct hs_probit_batch {
  std::vector<hs_probit*> probs;
  int device = 0;
  int num_sms = 1;
  cudaStream_t root = nullptr;
  bool own_root = false;
  cudaEvent_t ev_start = nullptr;
  std::vector<cudaEvent_t> ev_done;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<double> wx, wc;  // each problem's X bytes and factorization work (K P^3)
  double wx_sum = 0, wc_sum = 0;
  std::vector<hs_tune_trial> trials;
  uint64_t shape_epochs = 0;  // sum of the problems' shape epochs when the graph was captured
};

namespace {

void batch_drop_graph(hs_probit_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
}

// One graph for a sweep of every problem: the root stream forks to each
// problem's streams and joins them again, so the problems are independent
// branches.
cudaError_t batch_build_graph(hs_probit_batch* b) {
  batch_drop_graph(b);
  b->shape_epochs = 0;
  for (hs_probit* h : b->probs) b->shape_epochs += h->shape_epoch;
  cudaError_t e = cudaStreamBeginCapture(b->root, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t e2 = cudaEventRecord(b->ev_start, b->root);
  for (size_t m = 0; m < b->probs.size() && e2 == cudaSuccess; ++m) {
    hs_probit* h = b->probs[m];
    e2 = cudaStreamWaitEvent(h->s0, b->ev_start, 0);
    if (e2 == cudaSuccess) e2 = enqueue_sweep(h);
    if (e2 == cudaSuccess) e2 = cudaEventRecord(b->ev_done[m], h->s0);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(b->root, b->ev_done[m], 0);
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->root, &g);
  if (e2 != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return e2 != cudaSuccess ? e2 : e;
  }
  e = cudaGraphInstantiate(&b->gexec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return e;
  }
  b->graph = g;
  return cudaSuccess;
}

// After the root stream is idle: each problem's error word and sweep count.
int batch_check(hs_probit_batch* b) {
  if (cudaStreamSynchronize(b->root) != cudaSuccess) return HS_ECUDA;
  int first = HS_OK;
  for (hs_probit* h : b->probs) {
    const int st = sync_and_check(h);
    if (st != HS_OK) {
      h->sticky = st;
      if (first == HS_OK) first = st;
    }
  }
  return first;
}

// Launch shapes of every problem: X-stream CTAs in proportion to the
// problem's share of the X bytes (oversubscription factor f, times the CTAs
// per SM of the X-stream tile), trailing-update CTAs to its share of the
// factorization work (f), factorization blocks to the same share (factor fc:
// those blocks mostly wait on their diagonal chains, so they want a factor of
// their own); the tensor-core X-stream tile (kc chain columns, stages, CTAs
// per SM; kc = 0: the handle's starting tile); overlap as the launch-shape
// field (1 beside, 2 after).
int batch_apply_shapes(hs_probit_batch* b, double f, double fc, int kc, int stages, int per_sm, int overlap) {
  for (size_t m = 0; m < b->probs.size(); ++m) {
    hs_probit* h = b->probs[m];
    const double sx = b->wx[m] / b->wx_sum, sc = b->wc[m] / b->wc_sum;
    auto share = [](double v, int lo, int64_t hi) {
      const long r = std::lround(v);
      return (int)std::max<long>(lo, std::min<long>((long)hi, r));
    };
    hs_launch_shape ls{};
    int c = 0, st = 0, pm = 1;
    if (h->xk) {
      c = hs::xstream_k_default_kc(h->K);
      st = h->xk_split ? hs::xstream_k_split_stages(c) : hs::kXkDefaultStages;
      if (kc > 0 && !h->xk_split) {
        const int c2 = kc >= h->K ? kc : 32, pm2 = c2 == 16 ? per_sm : 1;
        if (hs::xstream_k_supported(h->p, c2, stages, pm2)) {
          c = c2;
          st = stages;
          pm = pm2;
        }
      }
      ls.xk_chains = c;
      ls.xk_stages = st;
      ls.xk_ctas_per_sm = pm;
    }
    const int64_t xs_hi = h->xk ? std::min<int64_t>(hs::xstream_k_tiles(h->N), (int64_t)h->kgrid_max * 32 / c)
                                : h->grid_max;
    ls.xstream_ctas = share(f * pm * b->num_sms * sx, 1, xs_hi);
    if (h->chol_grid > 0) ls.chol_ctas = share(fc * h->chol_max * sc, h->K + 1, h->chol_max);
    if (h->tensor_sched) ls.trail_ctas = share(f * b->num_sms * sc, 1, h->trail_max);
    ls.overlap = overlap;
    const int r = hs_probit_set_launch_shape(h, &ls);
    if (r != HS_OK) return r;
  }
  return HS_OK;
}

// Time `sweeps` graph launches (after one untimed launch); ms per sweep.
int batch_time(hs_probit_batch* b, int sweeps, double* ms) {
  cudaError_t e = batch_build_graph(b);
  if (e != cudaSuccess) return cuda_status(e);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->gexec, b->root);
  if (e == cudaSuccess) e = cudaEventRecord(t0, b->root);
  for (int i = 0; i < sweeps && e == cudaSuccess; ++i) e = cudaGraphLaunch(b->gexec, b->root);
  if (e == cudaSuccess) e = cudaEventRecord(t1, b->root);
  int st = e == cudaSuccess ? batch_check(b) : cuda_status(e);
  float t = 0.f;
  if (st == HS_OK && cudaEventElapsedTime(&t, t0, t1) != cudaSuccess) st = HS_ECUDA;
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  *ms = (double)t / sweeps;
  return st;
}

void batch_destroy(hs_probit_batch* b) {
  if (b->root) cudaStreamSynchronize(b->root);
  batch_drop_graph(b);
  for (hs_probit* h : b->probs) {
    DeviceGuard dg(h->device);
    destroy(h);
  }
  for (cudaEvent_t ev : b->ev_done)
    if (ev) cudaEventDestroy(ev);
  if (b->ev_start) cudaEventDestroy(b->ev_start);
  if (b->own_root && b->root) cudaStreamDestroy(b->root);
  delete b;
}

hs_probit_batch* batch_init_impl(const hs_probit_config* cfg, int32_t n, const hs_problem* problems, uint64_t seed) {
  if (!cfg || n < 1 || !problems) {
    fail(HS_EINVAL);
    return nullptr;
  }
  for (int32_t m = 0; m < n; ++m)
    if (!problems[m].X || !problems[m].y || problems[m].N < 2 || problems[m].p < 1) {
      fail(HS_EINVAL);
      return nullptr;
    }
  DeviceGuard dg(cfg->device);
  if (!dg.ok) {
    fail(HS_ECUDA);
    return nullptr;
  }
  hs_probit_batch* b = new hs_probit_batch();
  b->device = cfg->device;
  auto bail = [&](int st) -> hs_probit_batch* {
    batch_destroy(b);
    fail(st);
    return nullptr;
  };
  if (cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, cfg->device) != cudaSuccess)
    return bail(HS_ECUDA);
  cudaError_t e = cudaSuccess;
  if (cfg->stream) {
    b->root = static_cast<cudaStream_t>(cfg->stream);
  } else {
    e = cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking);
    b->own_root = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming);
  b->ev_done.assign((size_t)n, nullptr);
  for (int32_t m = 0; m < n && e == cudaSuccess; ++m) e = cudaEventCreateWithFlags(&b->ev_done[m], cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(cuda_status(e));
  const int64_t eb = cfg->x_dtype == HS_X_F64 ? 8 : cfg->x_dtype == HS_X_F32 ? 4 : cfg->x_dtype == HS_X_BF16 ? 2 : 1;
  for (int32_t m = 0; m < n; ++m) {
    hs_probit_config c = *cfg;
    c.problem = cfg->problem + (uint32_t)m;
    c.x_scales = problems[m].x_scales;
    c.stream = nullptr;
    c.use_graph = 0;
    hs_probit* h = init_ex_impl(&c, problems[m].X, problems[m].y, problems[m].N, problems[m].p, seed);
    if (!h) return bail(g_last_error != HS_OK ? g_last_error : HS_ECUDA);
    h->batch_member = true;
    b->probs.push_back(h);
    b->wx.push_back((double)problems[m].N * (double)problems[m].p * (double)eb);
    b->wc.push_back((double)h->K * (double)h->P * (double)h->P * (double)h->P);
    b->wx_sum += b->wx.back();
    b->wc_sum += b->wc.back();
  }
  // the starting shapes: every problem's kernels sized to its share of the GPU
  const int st = batch_apply_shapes(b, 1.0, 1.0, 0, 0, 1, 2);
  if (st != HS_OK) return bail(st);
  g_last_error = HS_OK;
  return b;
}

}  // namespace

extern "C" {

hs_probit_batch* hs_probit_batch_init(const hs_probit_config* cfg, int32_t n, const hs_problem* problems,
                                      uint64_t seed) {
  try {
    return batch_init_impl(cfg, n, problems, seed);
  } catch (...) {
    fail(HS_ENOMEM);
    return nullptr;
  }
}

int32_t hs_probit_batch_size(const hs_probit_batch* b) { return b ? (int32_t)b->probs.size() : HS_EINVAL; }

hs_probit* hs_probit_batch_problem(hs_probit_batch* b, int32_t m) {
  if (!b || m < 0 || m >= (int32_t)b->probs.size()) return nullptr;
  return b->probs[(size_t)m];
}

int hs_probit_batch_sweep(hs_probit_batch* b, int64_t n_iter) {
  if (!b || n_iter < 0) return HS_EINVAL;
  for (hs_probit* h : b->probs)
    if (h->sticky != HS_OK) return HS_ESTATE;
  if (n_iter == 0) return HS_OK;
  DeviceGuard dg(b->device);
  if (!dg.ok) return HS_ECUDA;
  try {
    // a problem's own work (a sweep, a state change) is ordered before the batch's
    for (hs_probit* h : b->probs) {
      if (cudaStreamSynchronize(h->s0) != cudaSuccess || cudaStreamSynchronize(h->s1) != cudaSuccess)
        return HS_ECUDA;
    }
    uint64_t epochs = 0;
    for (hs_probit* h : b->probs) epochs += h->shape_epoch;
    if (!b->gexec || epochs != b->shape_epochs) {
      const cudaError_t e = batch_build_graph(b);
      if (e != cudaSuccess) return cuda_status(e);
    }
    cudaError_t e = cudaSuccess;
    for (hs_probit* h : b->probs)
      if (e == cudaSuccess) e = guard_ring(h, n_iter, b->root);
    for (int64_t i = 0; i < n_iter && e == cudaSuccess; ++i) e = cudaGraphLaunch(b->gexec, b->root);
    if (e != cudaSuccess) {
      cudaStreamSynchronize(b->root);
      return cuda_status(e);
    }
    return batch_check(b);
  } catch (...) {
    return HS_ENOMEM;
  }
}

int hs_probit_batch_tune(hs_probit_batch* b, int32_t sweeps, double* best_ms) {
  if (!b || sweeps < 1) return HS_EINVAL;
  for (hs_probit* h : b->probs)
    if (h->sticky != HS_OK) return HS_ESTATE;
  DeviceGuard dg(b->device);
  if (!dg.ok) return HS_ECUDA;
  try {
    // save every chain's state
    struct Saved {
      std::vector<double> beta, lam, nu;
      double tau, xi;
      int64_t k;
    };
    std::vector<std::vector<Saved>> saved(b->probs.size());
    for (size_t m = 0; m < b->probs.size(); ++m) {
      hs_probit* h = b->probs[m];
      saved[m].resize((size_t)h->K);
      for (int c = 0; c < h->K; ++c) {
        Saved& sv = saved[m][(size_t)c];
        sv.beta.resize((size_t)h->p);
        sv.lam.resize((size_t)h->p);
        sv.nu.resize((size_t)h->p);
        hs_probit_state_view v{sv.beta.data(), sv.lam.data(), sv.nu.data(), 0.0, 0.0, 0};
        const int st = hs_probit_get_state_chain(h, c, &v);
        if (st != HS_OK) return st;
        sv.tau = v.tau_inv2;
        sv.xi = v.xi_inv;
        sv.k = v.k;
      }
    }
    b->trials.clear();
    int status = HS_OK;
    auto trial = [&](double f, double fc, int kc, int stages, int per_sm, int overlap) -> double {
      double ms = -1.0;
      if (status != HS_OK) return ms;
      status = batch_apply_shapes(b, f, fc, kc, stages, per_sm, overlap);
      if (status == HS_OK) status = batch_time(b, sweeps, &ms);
      if (status != HS_OK) return -1.0;
      hs_tune_trial t{};
      t.ms_per_sweep = ms;
      t.oversub = f;
      t.chol_oversub = fc;
      t.xk_chains = kc;
      t.xk_stages = stages;
      t.xk_ctas_per_sm = kc > 0 ? per_sm : 0;
      t.overlap = overlap;
      b->trials.push_back(t);
      return ms;
    };
    // oversubscription of the proportional shares, then the factorization's
    // own factor, then the X-stream tiles, each at the best so far
    const double fs[] = {0.5, 1.0, 2.0, 4.0};
    double best = -1.0, best_f = 1.0, best_fc = 1.0;
    for (double f : fs) {
      const double ms = trial(f, f, 0, 0, 1, 2);
      if (ms >= 0 && (best < 0 || ms < best)) {
        best = ms;
        best_f = best_fc = f;
      }
    }
    const double fcs[] = {0.125, 0.25, 0.5, 2.0};
    const double f0 = best_f;
    for (double r : fcs) {
      const double ms = trial(f0, f0 * r, 0, 0, 1, 2);
      if (ms >= 0 && (best < 0 || ms < best)) {
        best = ms;
        best_fc = f0 * r;
      }
    }
    int best_kc = 0, best_st = 0, best_pm = 1, best_ov = 2;
    bool any_xk = false, any_multi = false;
    for (hs_probit* h : b->probs) {
      any_xk = any_xk || h->xk;
      any_multi = any_multi || (h->K > 1 && h->chol_grid > 0);
    }
    if (any_xk) {
      const int shapes[][3] = {{16, 4, 1}, {16, 6, 1}, {16, 8, 1}, {16, 4, 2}, {32, 8, 1}};
      for (const auto& sh : shapes) {
        const double ms = trial(best_f, best_fc, sh[0], sh[1], sh[2], 2);
        if (ms >= 0 && (best < 0 || ms < best)) {
          best = ms;
          best_kc = sh[0];
          best_st = sh[1];
          best_pm = sh[2];
        }
      }
    }
    if (any_multi) {
      // the K chains' factorization beside the X-stream instead of after it
      const double ms = trial(best_f, best_fc, best_kc, best_st, best_pm, 1);
      if (ms >= 0 && (best < 0 || ms < best)) {
        best = ms;
        best_ov = 1;
      }
    }
    if (status == HS_OK) status = batch_apply_shapes(b, best_f, best_fc, best_kc, best_st, best_pm, best_ov);
    if (status == HS_OK) {
      const cudaError_t e = batch_build_graph(b);
      if (e != cudaSuccess) status = cuda_status(e);
    }
    // put every chain back where it was
    for (size_t m = 0; m < b->probs.size(); ++m) {
      hs_probit* h = b->probs[m];
      if (h->sticky != HS_OK) continue;
      for (int c = 0; c < h->K; ++c) {
        Saved& sv = saved[m][(size_t)c];
        hs_probit_state_view v{sv.beta.data(), sv.lam.data(), sv.nu.data(), sv.tau, sv.xi, sv.k};
        const int st = hs_probit_set_state_chain(h, c, &v);
        if (st != HS_OK && status == HS_OK) status = st;
      }
    }
    if (best_ms) *best_ms = best;
    return status;
  } catch (...) {
    return HS_ENOMEM;
  }
}

int32_t hs_probit_batch_tune_trials(const hs_probit_batch* b, hs_tune_trial* out, int32_t max) {
  if (!b || max < 0 || (max > 0 && !out)) return HS_EINVAL;
  const int32_t n = (int32_t)b->trials.size();
  for (int32_t i = 0; i < n && i < max; ++i) out[i] = b->trials[(size_t)i];
  return n;
}

void hs_probit_batch_free(hs_probit_batch* b) {
  if (!b) return;
  DeviceGuard dg(b->device);
  batch_destroy(b);
}

}  // extern "C"

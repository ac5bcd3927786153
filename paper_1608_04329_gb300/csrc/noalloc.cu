// The X-stream pass of a sweep without any device allocation.
//
// Who needs this: callers that must not call cudaMalloc while they run.
// cudaMalloc can synchronize the whole device and takes memory outside any
// pool the caller manages, so a runtime that plans all of its device memory
// up front (a serving process multiplexing many samplers on one GPU, or a
// latency-critical loop that treats a device-wide synchronization as a
// fault) cannot create an hs_probit handle mid-run, because the handle
// allocates its own work buffers.  This entry point runs the same X-stream
// kernel as hs_probit_sweep on buffers the caller already owns; the only
// scratch it needs (the per-CTA partial sums of X^T z, the device error word
// and the sweep number) lives in one fixed array in this file, loaded with
// the library, so no call allocates anything.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "hs_internal.h"
#include "hs_probit.h"

namespace hs {
namespace {

// Scratch layout: [0, 256) header {int err; int pad; int64_t sweeps_done},
// then the partial sums (grid x ld values of the compute type).
constexpr size_t kHeaderBytes = 256;
constexpr size_t kPartialBytesMax = (size_t)4 << 20;  // 4 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kHeaderBytes + kPartialBytesMax];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
int g_num_sms[kMaxDevices] = {0};

__global__ void noalloc_header_kernel(int* err, int64_t* sweeps_done, int64_t value) {
  *err = 0;
  *sweeps_done = value;
}

// Device address of the scratch array on the current device (set up once
// per device, with that device current).  The address is kept for the life
// of the process; after cudaDeviceReset it would be stale, so a caller that
// resets a device must not use this entry point on it again.
int scratch_for_device(int dev, unsigned char** ptr, int* num_sms) {
  if (dev < 0 || dev >= kMaxDevices) return HS_EINVAL;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return HS_ECUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
      (void)cudaGetLastError();
      return HS_ECUDA;
    }
    g_num_sms[dev] = sms;
    g_scratch_ptr[dev] = p;
  }
  *ptr = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  *num_sms = g_num_sms[dev];
  return HS_OK;
}

int elem_bytes(int x_dtype) {
  switch (x_dtype) {
    case HS_X_F64: return 8;
    case HS_X_F32: return 4;
    case HS_X_BF16: return 2;
    case HS_X_FP8E4M3: return 1;
  }
  return 0;
}

}  // namespace
}  // namespace hs

extern "C" int hs_probit_xstream_noalloc(int x_dtype, const void* X, int64_t ld, const uint8_t* y, int64_t N,
                                         int64_t p, const void* beta_c, const float* x_scales, uint64_t seed,
                                         uint32_t chain, uint32_t problem, int64_t sweep, double* xtz, double* z,
                                         void* stream) {
  using namespace hs;
  const int eb = elem_bytes(x_dtype);
  // Every check below is on the host and comes before any CUDA call.  The
  // bulk copies read rows of X from 16-byte boundaries, so X must start on
  // one; beta_c, xtz and z are read or written as whole doubles (floats for
  // beta_c of the narrow types).  (ld * eb) / 16 > 2048: more 16-byte slices
  // per row than the kernel takes.
  const uintptr_t bc_align = x_dtype == HS_X_F64 ? 8 : 4;
  if (eb == 0 || !X || !y || !beta_c || !xtz || N < 1 || p < 1 || p > 8192 || ld < p || sweep < 1 ||
      sweep > (int64_t)0xFFFFFFFF || N > (int64_t)0xFFFFFFFF || chain >= (1u << 24) || (ld * eb) % 16 != 0 ||
      (x_dtype == HS_X_FP8E4M3) != (x_scales != nullptr) || ld > 16384 || (ld * eb) / 16 > 2048 ||
      (reinterpret_cast<uintptr_t>(X) & 15u) != 0 || (reinterpret_cast<uintptr_t>(beta_c) & (bc_align - 1)) != 0 ||
      (reinterpret_cast<uintptr_t>(xtz) & 7u) != 0 || (reinterpret_cast<uintptr_t>(z) & 7u) != 0 ||
      (x_scales && (reinterpret_cast<uintptr_t>(x_scales) & 3u) != 0))
    return HS_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HS_ECUDA;
  unsigned char* scratch = nullptr;
  int sms = 0;
  int st = scratch_for_device(dev, &scratch, &sms);
  if (st != HS_OK) return st;
  const int grid = xstream_grid(x_dtype, (int)p, (int)ld, N, sms);
  const size_t part_bytes = (size_t)grid * (size_t)ld * (size_t)partial_elem_bytes(x_dtype);
  if (part_bytes > kPartialBytesMax) return HS_EINVAL;  // beyond the fixed scratch
  int* err = reinterpret_cast<int*>(scratch);
  int64_t* sweeps_done = reinterpret_cast<int64_t*>(scratch + 8);
  void* partials = scratch + kHeaderBytes;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  cudaError_t e = xstream_prepare();
  if (e == cudaSuccess) {
    noalloc_header_kernel<<<1, 1, 0, s>>>(err, sweeps_done, sweep - 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    XStreamArgs a{};
    a.X = X;
    a.y = y;
    a.N = N;
    a.ld = (int)ld;
    a.p = (int)p;
    a.beta_c = beta_c;
    a.partials = partials;
    a.z_out = z;
    a.k_dev = sweeps_done;
    a.rng = RngKey{(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32), chain, problem};
    a.err = err;
    e = xstream_launch(x_dtype, a, grid, s);
  }
  if (e == cudaSuccess) e = reduce_partials_launch(x_dtype, partials, grid, (int)ld, (int)p, x_scales, xtz, s);
  int h_err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return HS_ECUDA;
  }
  if (h_err & kErrNonFinite) return HS_ENONFINITE;
  if (h_err & kErrTimeout) return HS_ETIMEOUT;
  return h_err ? HS_ECUDA : HS_OK;
}

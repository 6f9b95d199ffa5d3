// randutv_small_svd_noalloc: the small-block Jacobi SVD without any device
// allocation.
//
// randutv_small_svd obtains its scratch (the Jacobi iterate, the rotation
// accumulator, the ordering arrays and the barrier words) from
// cudaMallocAsync on every call.  Some callers cannot allow that: code that
// runs while its host framework owns all device memory through its own
// allocator, code on a latency-critical path where an allocation may
// synchronise or fail under memory pressure, and code embedded in a plugin
// that is not permitted to call the CUDA allocator at all.  This variant
// takes its scratch from one fixed array in device global memory that the
// library declares at file scope; the caller still passes M, Us, d and Vs.
//
// Limits and sharing: p <= kNoAllocMaxP.  The array (about 4 MB) exists on
// every GPU that loads the library until the process exits.  All calls on a
// device share it and it keeps the last call's contents, so two calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race on it; serialise them.  The first call on each device looks up the
// device address of the array (cudaGetSymbolAddress, with that device
// current) and caches it; make that first call before any stream capture.
#include <cstdio>
#include <mutex>
#include "common.cuh"
#include "internal.h"

namespace rutv {
namespace {

constexpr int kNoAllocMaxP = 256;
constexpr int kMaxDevices = 64;
// jacobi_work_elems(256) doubles, then 8 doubles of barrier/error words
constexpr int64_t kNoAllocElems = jacobi_work_elems_for(kNoAllocMaxP) + 8;

static __device__ __align__(256) double g_svd_scratch[kNoAllocElems];

std::mutex g_mu;
double* g_dev_ptr[kMaxDevices] = {};

// Device address of g_svd_scratch on the current device (looked up once).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_svd_scratch);
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_dev_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace rutv

extern "C" int randutv_small_svd_noalloc(int64_t p, const double* M, int64_t ldm, double* Us, double* d,
                                         double* Vs, int max_sweeps) {
  using namespace rutv;
  if (p < 1) return -1;
  if (!M) return -2;
  if (ldm < p) return -3;
  if (!Us) return -4;
  if (!d) return -5;
  if (!Vs) return -6;
  if (max_sweeps < 1) return -7;
  if (p > kNoAllocMaxP) {
    set_last_error("randutv_small_svd_noalloc: p exceeds the 256 x 256 limit of its static scratch");
    return RANDUTV_EUNSUPPORTED;
  }
  const int pi = static_cast<int>(p);
  double* base = nullptr;
  char msg[192];
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "randutv_small_svd_noalloc: cudaGetSymbolAddress of the scratch array: %s",
             cudaGetErrorString(e));
    set_last_error(msg);
    return RANDUTV_ECUDA;
  }
  cudaStream_t s = current_stream();
  double* work = base;
  unsigned* flags = reinterpret_cast<unsigned*>(base + jacobi_work_elems(pi));
  unsigned herr[4] = {0, 0, 0, 0};
  // The barrier count/generation and the error word must start at zero.
  e = cudaMemsetAsync(flags, 0, 4 * sizeof(unsigned), s);
  if (e == cudaSuccess) e = jacobi_svd(s, pi, M, ldm, Us, d, Vs, max_sweeps, work, flags);
  if (e == cudaSuccess) e = cudaMemcpyAsync(herr, flags, sizeof(herr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    // no work this call queued may still be writing the shared scratch once it returns
    cudaStreamSynchronize(s);
    snprintf(msg, sizeof(msg), "randutv_small_svd_noalloc: %s", cudaGetErrorString(e));
    set_last_error(msg);
    return RANDUTV_ECUDA;
  }
  if (herr[2] & kDevErrTimeout) return RANDUTV_ETIMEOUT;
  if (herr[2] & kDevErrNoConv) return RANDUTV_ENOCONV;
  return RANDUTV_OK;
}

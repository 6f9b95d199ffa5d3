// Self-test of the bounded device waits: a wait that nothing will end runs
// out after a short limit, the kernel records the timeout in an error word
// and returns, and the host reports RANDUTV_ETIMEOUT with the context still
// usable.  The paper has no counterpart; this checks the failure path that
// every grid barrier and mbarrier wait of the library relies on, without
// faulting or hanging the GPU: the wait targets an mbarrier no thread arrives
// at, or a grid barrier sized for two CTAs in a launch of one.
#include <cstdio>
#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace rutv {
namespace {

// Barrier count, generation slot and error word of the test (zeroed by the
// kernel before it waits; one launch at a time per device).
__device__ unsigned g_selftest_words[4];

__global__ void wait_selftest_kernel(int kind, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  unsigned* words = g_selftest_words;
  int* err = reinterpret_cast<int*>(words + 2);
  if (kind == 0) {
    // an mbarrier expecting one arrival that never comes
    if (threadIdx.x == 0) {
      mbar_init(&bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0, global_ns(), limit_ns)) atomicOr(err, kDevErrTimeout);
    __syncthreads();
  } else {
    // a grid barrier for two CTAs in a grid of one
    GridBarrier gb{words, words + 1, err};
    grid_barrier(gb, 2, limit_ns);
  }
}

__global__ void selftest_clear_kernel() {
  if (threadIdx.x < 4) g_selftest_words[threadIdx.x] = 0;
}

}  // namespace
}  // namespace rutv

extern "C" int randutv_selftest_wait(int kind, double seconds) {
  using namespace rutv;
  if (kind != 0 && kind != 1) return -1;
  if (!(seconds > 0.0) || seconds > 2.0) return -2;
  const unsigned long long limit = static_cast<unsigned long long>(seconds * 1e9);
  cudaStream_t s = nullptr;
  selftest_clear_kernel<<<1, 32, 0, s>>>();
  note_launch();
  wait_selftest_kernel<<<1, 64, 0, s>>>(kind, limit);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  unsigned words[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(words, g_selftest_words, sizeof(words));
  if (e != cudaSuccess) {
    char msg[160];
    snprintf(msg, sizeof(msg), "randutv_selftest_wait: %s", cudaGetErrorString(e));
    set_last_error(msg);
    cudaGetLastError();
    return RANDUTV_ECUDA;
  }
  if (static_cast<int>(words[2]) & kDevErrTimeout) {
    set_last_error(kind == 0 ? "self-test: mbarrier wait timed out" : "self-test: grid barrier timed out");
    return RANDUTV_ETIMEOUT;
  }
  return RANDUTV_OK;
}

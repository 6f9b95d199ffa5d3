// Shared device utilities of the randUTV engine (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/randutv.h"

namespace rutv {

constexpr int kNumSMs = 152;

// Device-side error word values (written by kernels, read by the host).
constexpr int kDevErrTimeout = 1;   // a grid barrier wait ran out
constexpr int kDevErrNoConv  = 2;   // Jacobi hit its sweep cap
constexpr int kDevErrNaN     = 4;   // non-finite value met

// Barrier state for kernels launched cooperatively (all CTAs co-resident).
struct GridBarrier {
  unsigned* count;  // arrivals since the launch (zeroed before it)
  unsigned* gen;    // unused (kept for the slot layout)
  int* err;         // device error word (kDevErr* bits)
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier with a bounded wait.  One monotonic arrival counter
// (zeroed before the launch): a CTA adds 1 with acquire-release semantics and
// waits until the counter reaches the next multiple of the grid size, so the
// last arriver does a single atomic and nobody resets anything.  Returns false
// (in every thread of the CTA) when the wait ran out or another CTA reported
// an error; the caller must then return without touching shared state.  The
// wait gives up after limit_ns of wall time (2 s by default) and sets
// kDevErrTimeout.
__device__ __forceinline__ bool grid_barrier(const GridBarrier& g, unsigned nblocks,
                                             unsigned long long limit_ns = 2000000000ull) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(g.count) : "memory");
    const unsigned target = (old / nblocks + 1) * nblocks;
    if (old + 1 != target) {
      const unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (static_cast<int>(ld_acquire_u32(g.count) - target) < 0) {
        if (++spins > 1024) __nanosleep(32);
        if ((spins & 255u) == 0 && global_ns() - t0 > limit_ns) {
          atomicOr(g.err, kDevErrTimeout);
          ok = 0;
          break;
        }
      }
    }
    if (ok && (*(volatile int*)g.err & kDevErrTimeout)) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__host__ __device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }
__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace rutv

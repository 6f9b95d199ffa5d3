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
  unsigned* count;  // arrivals in the current generation
  unsigned* gen;    // generation number
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

// Grid-wide barrier with a bounded wait.  Returns false (in every thread of
// the CTA) when the wait ran out or another CTA reported an error; the caller
// must then return without touching shared state.  The wait gives up after
// ~2 s of wall time and sets kDevErrTimeout.
__device__ __forceinline__ bool grid_barrier(const GridBarrier& g, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned my_gen = ld_acquire_u32(g.gen);
    __threadfence();
    unsigned prev = atomicAdd(g.count, 1u);
    if (prev == nblocks - 1) {
      atomicExch(g.count, 0u);
      __threadfence();
      atomicAdd(g.gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (ld_acquire_u32(g.gen) == my_gen) {
        if (++spins > 1024) __nanosleep(32);
        if ((spins & 255u) == 0 && global_ns() - t0 > 2000000000ull) {
          atomicOr(g.err, kDevErrTimeout);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
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

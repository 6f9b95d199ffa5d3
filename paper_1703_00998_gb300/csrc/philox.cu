// Gaussian matrices G of the randomized steps (Fig. 4, randn) from the
// counter-based generator Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11,
// Section 4.2), written from its published definition.
#include "common.cuh"
#include "internal.h"
#include "philox.cuh"

namespace rutv {

// Open-interval uniform from the top 52 bits of (hi:lo): exact in FP64.
__device__ __forceinline__ double uniform52(uint32_t lo, uint32_t hi) {
  uint64_t w = (static_cast<uint64_t>(hi) << 32) | lo;
  return (static_cast<double>(w >> 12) + 0.5) * 0x1p-52;
}

__global__ void gaussian_kernel(uint32_t k0, uint32_t k1, uint32_t step, int64_t k, int64_t b,
                                double* __restrict__ G, int64_t ldg) {
  const int64_t npairs = (k + 1) / 2;
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= npairs * b) return;
  const int64_t p = t % npairs, c = t / npairs;
  U4 w = philox4x32_10(U4{static_cast<uint32_t>(p), static_cast<uint32_t>(c), step, 0u}, k0, k1);
  const double u1 = uniform52(w.x0, w.x1), u2 = uniform52(w.x2, w.x3);
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  double* col = G + c * ldg;
  col[2 * p] = r * cs;
  if (2 * p + 1 < k) col[2 * p + 1] = r * sn;
}

__global__ void philox_words_kernel(uint32_t k0, uint32_t k1, uint32_t step, int64_t k, int64_t b,
                                    uint32_t* __restrict__ W) {
  const int64_t npairs = (k + 1) / 2;
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= npairs * b) return;
  const int64_t p = t % npairs, c = t / npairs;
  U4 w = philox4x32_10(U4{static_cast<uint32_t>(p), static_cast<uint32_t>(c), step, 0u}, k0, k1);
  uint32_t* o = W + 4 * t;
  o[0] = w.x0; o[1] = w.x1; o[2] = w.x2; o[3] = w.x3;
}

cudaError_t launch_gaussian(cudaStream_t s, uint64_t seed, int64_t step, int64_t k, int64_t b,
                            double* G, int64_t ldg) {
  const int64_t total = (k + 1) / 2 * b;
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (total + threads - 1) / threads;
  const ProfToken tok = prof_begin(s, kProfGauss);
  gaussian_kernel<<<static_cast<unsigned>(blocks), threads, 0, s>>>(
      static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32), static_cast<uint32_t>(step),
      k, b, G, ldg);
  note_launch();
  prof_end(s, tok, 0.0, 8.0 * k * b);
  return cudaGetLastError();
}

cudaError_t launch_philox_words(cudaStream_t s, uint64_t seed, int64_t step, int64_t k, int64_t b,
                                uint32_t* W) {
  const int64_t total = (k + 1) / 2 * b;
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (total + threads - 1) / threads;
  philox_words_kernel<<<static_cast<unsigned>(blocks), threads, 0, s>>>(
      static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32), static_cast<uint32_t>(step),
      k, b, W);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rutv

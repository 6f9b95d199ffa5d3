// FP32 GEMM for the mixed-precision form: C = alpha op(A) op(B) + beta C,
// column-major, FP32 operands and accumulation on the FFMA pipe (74 TFLOP/s
// measured, 62x the FP64 rate).  Same products as the FP64 form (sketch,
// block-reflector applications, small rotations); T, U and V are stored in
// FP32 there.  Thin products are split along K like the FP64 GEMM; the
// partial sums of a split are added in FP64 before the single rounding to
// FP32, which keeps the long reductions (K = k ~ n) near one FP32 rounding.
#include "common.cuh"
#include "internal.h"

namespace rutv {

namespace {
constexpr int SBM = 128, SBN = 128, SBK = 8, SNT = 256;
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(SNT, 2)
sgemm_kernel(int64_t M, int64_t N, int64_t K, float alpha, const float* __restrict__ A, int64_t lda,
             const float* __restrict__ B, int64_t ldb, float beta, float* __restrict__ C, int64_t ldc,
             float* __restrict__ part, int64_t kchunk) {
  __shared__ __align__(16) float As[2][SBK][SBM];
  __shared__ __align__(16) float Bs[2][SBK][SBN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;   // 16 x 16 threads, 8 x 8 outputs each
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * SBM;
  const int64_t n0 = static_cast<int64_t>(blockIdx.y) * SBN;
  const int64_t kbeg = static_cast<int64_t>(blockIdx.z) * kchunk;
  const int64_t kend = min(K, kbeg + kchunk);

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  // each thread loads 4 elements of the A tile (128 x 8) and 4 of B (8 x 128)
  float ra[4], rb[4];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int i, kk;
      if (!TA) { i = tid % 128; kk = tid / 128 + 2 * r; } else { kk = tid % 8; i = tid / 8 + 32 * r; }
      const int64_t gi = m0 + i, gk = k0 + kk;
      float v = 0.f;
      if (gi < M && gk < kend) v = TA ? A[gk + gi * lda] : A[gi + gk * lda];
      ra[r] = v;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int j, kk;
      if (!TB) { kk = tid % 8; j = tid / 8 + 32 * r; } else { j = tid % 128; kk = tid / 128 + 2 * r; }
      const int64_t gj = n0 + j, gk = k0 + kk;
      float v = 0.f;
      if (gj < N && gk < kend) v = TB ? B[gj + gk * ldb] : B[gk + gj * ldb];
      rb[r] = v;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (!TA) As[buf][tid / 128 + 2 * r][tid % 128] = ra[r]; else As[buf][tid % 8][tid / 8 + 32 * r] = ra[r];
      if (!TB) Bs[buf][tid % 8][tid / 8 + 32 * r] = rb[r]; else Bs[buf][tid / 128 + 2 * r][tid % 128] = rb[r];
    }
  };

  int buf = 0;
  if (kbeg < kend) {
    load(kbeg);
    store(0);
  }
  __syncthreads();
  for (int64_t k0 = kbeg; k0 < kend; k0 += SBK) {
    const bool more = k0 + SBK < kend;
    if (more) load(k0 + SBK);
#pragma unroll
    for (int kk = 0; kk < SBK; ++kk) {
      // rows tx*4 + {0..3} and 64 + tx*4 + {0..3}; columns likewise with ty
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][tx * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + tx * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][ty * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + ty * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }

#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int64_t gj = n0 + (j < 4 ? ty * 4 + j : 64 + ty * 4 + (j - 4));
    if (gj >= N) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t gi = m0 + (i < 4 ? tx * 4 + i : 64 + tx * 4 + (i - 4));
      if (gi >= M) continue;
      if (part) {
        part[static_cast<int64_t>(blockIdx.z) * M * N + gi + gj * M] = acc[i][j];
      } else {
        float* c = C + gi + gj * ldc;
        *c = (beta == 0.f) ? alpha * acc[i][j] : fmaf(alpha, acc[i][j], beta * *c);
      }
    }
  }
}

// Sum the split-K partials in FP64, round once.
__global__ void sgemm_reduce_kernel(int64_t M, int64_t N, int splits, float alpha, const float* __restrict__ part,
                                    float beta, float* __restrict__ C, int64_t ldc) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= M * N) return;
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += static_cast<double>(part[z * M * N + t]);
  float* c = C + t % M + (t / M) * ldc;
  const double v = static_cast<double>(alpha) * s;
  *c = (beta == 0.f) ? static_cast<float>(v) : static_cast<float>(fma(static_cast<double>(beta), *c, v));
}

__global__ void sscale_kernel(int64_t M, int64_t N, float beta, float* __restrict__ C, int64_t ldc) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= M * N) return;
  float* c = C + t % M + (t / M) * ldc;
  *c = (beta == 0.f) ? 0.f : beta * *c;
}

namespace {
struct SPlan { int splits; int64_t kchunk; };

// Split K when the output has too few 128 x 128 tiles to fill 152 SMs x 2;
// among nearly equal plans prefer chunks of at most 1024 (shorter FP32
// accumulations).
SPlan plan_sgemm(int64_t M, int64_t N, int64_t K, int64_t work_elems) {
  const int64_t tiles = ((M + SBM - 1) / SBM) * ((N + SBN - 1) / SBN);
  SPlan best{1, ((K + SBK - 1) / SBK) * SBK};
  double best_t = 1e300;
  const double fma_per_s = 128.0 * 1.9e9;   // one SM's FFMA rate
  for (int s = 1; s <= 64; ++s) {
    int64_t kc = (K + s - 1) / s;
    kc = ((kc + SBK - 1) / SBK) * SBK;
    if (s > 1 && kc < 128) break;
    const int se = static_cast<int>((K + kc - 1) / kc);
    if (se > 1 && se * M * N > work_elems) break;
    const int64_t units = tiles * se;
    const int64_t per_sm = (units + 2 * kNumSMs - 1) / (2 * kNumSMs);
    double t = per_sm * 2.0 * static_cast<double>(SBM * SBN) * kc / fma_per_s;
    if (se > 1) t += 4e-6 + (se + 2.0) * M * N * 4.0 / 5.0e12;
    if (kc > 1024) t *= 1.02;   // prefer shorter FP32 accumulations when nearly free
    if (t < best_t * 0.999) { best_t = t; best = SPlan{se, kc}; }
  }
  return best;
}
}  // namespace

cudaError_t gemm_f32_reduce(cudaStream_t s, int64_t m, int64_t n, int splits, float alpha, const float* part,
                            float beta, float* C, int64_t ldc) {
  const int64_t tot = m * n;
  sgemm_reduce_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, s>>>(m, n, splits, alpha, part, beta, C,
                                                                               ldc);
  note_launch();
  return cudaGetLastError();
}

int64_t gemm_f32_work_elems(int64_t m, int64_t n, int64_t k) {
  SPlan p = plan_sgemm(m, n, k, INT64_MAX / 4);
  return p.splits > 1 ? p.splits * m * n : 0;
}

cudaError_t gemm_f32(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, float alpha,
                     const float* A, int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                     float* work, int64_t work_elems) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (k <= 0 || alpha == 0.f) {
    if (beta == 1.f) return cudaSuccess;
    const int64_t tot = m * n;
    sscale_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, s>>>(m, n, beta, C, ldc);
    note_launch();
    return cudaGetLastError();
  }
  SPlan p = plan_sgemm(m, n, k, work ? work_elems : 0);
  const ProfToken tok = prof_begin(s, kProfGemm32);
  dim3 grid(static_cast<unsigned>((m + SBM - 1) / SBM), static_cast<unsigned>((n + SBN - 1) / SBN),
            static_cast<unsigned>(p.splits));
  float* part = p.splits > 1 ? work : nullptr;
#define RUTV_SGEMM_LAUNCH(TA_, TB_) \
  sgemm_kernel<TA_, TB_><<<grid, SNT, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, part, p.kchunk)
  if (!ta && !tb) RUTV_SGEMM_LAUNCH(false, false);
  else if (ta && !tb) RUTV_SGEMM_LAUNCH(true, false);
  else if (!ta && tb) RUTV_SGEMM_LAUNCH(false, true);
  else RUTV_SGEMM_LAUNCH(true, true);
#undef RUTV_SGEMM_LAUNCH
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && p.splits > 1) {
    const int64_t tot = m * n;
    sgemm_reduce_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, s>>>(m, n, p.splits, alpha, part,
                                                                                 beta, C, ldc);
    note_launch();
    e = cudaGetLastError();
  }
  prof_end(s, tok, 2.0 * m * n * k, 4.0 * (m * k + k * n + m * n * (beta != 0.f ? 2.0 : 1.0)));
  return e;
}

}  // namespace rutv

extern "C" int randutv_sgemm(char transa, char transb, int64_t m, int64_t n, int64_t k, float alpha, const float* A,
                             int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc) {
  using namespace rutv;
  const bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
  if (!ta && transa != 'N' && transa != 'n') return -1;
  if (!tb && transb != 'N' && transb != 'n') return -2;
  if (m < 0) return -3;
  if (n < 0) return -4;
  if (k < 0) return -5;
  if (lda < (ta ? (k > 1 ? k : 1) : (m > 1 ? m : 1))) return -8;
  if (ldb < (tb ? (n > 1 ? n : 1) : (k > 1 ? k : 1))) return -10;
  if (ldc < (m > 1 ? m : 1)) return -13;
  cudaStream_t s = current_stream();
  const int64_t we = gemm_f32_work_elems(m, n, k);
  float* ws = nullptr;
  cudaError_t e = cudaSuccess;
  if (we > 0) e = cudaMallocAsync(&ws, we * sizeof(float), s);
  if (e == cudaSuccess) e = gemm_f32(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, we);
  if (ws) cudaFreeAsync(ws, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return RANDUTV_ECUDA;
  }
  return RANDUTV_OK;
}

// FP64 GEMM on the DFMA pipe: C = alpha op(A) op(B) + beta C, column-major.
//
// Every O(n^3) flop of randUTV is a product of the trailing matrix with a thin
// b-column matrix (Section 1.1 (iii), Section 5.4): the sketch X^T G, X Y and
// the block-reflector applications C V, W S, W V^T.  On GB300 FP64 runs at
// about 4 flop/clk/SM on the CUDA cores (the FP64 mma.sync path measures
// slower), so these products are bound by DFMA issue, not by HBM: a 64 x 64
// register-blocked tile re-reads each operand element 64 times from shared
// memory, far above what the 2-DFMA/clk/SM pipe needs (small products use
// a 32 x 32 tile so that they still spread over many SMs).  What matters is
// keeping every SM's DFMA pipe busy, so thin products are split along K until
// the work divides evenly over the 152 SMs (partials reduced by a second,
// memory-bound kernel).
#include <cmath>
#include "common.cuh"
#include "internal.h"

namespace rutv {

constexpr int BK = 16, NT = 256;

// Tile (16 TM) x (16 TM) per CTA, TM x TM outputs per thread: TM = 4 for the
// large products, TM = 2 for small ones (p x p products of the small SVD),
// which gives four times as many CTAs.
template <bool TA, bool TB, int TM>
__global__ void __launch_bounds__(NT, 2)
dgemm_kernel(int64_t M, int64_t N, int64_t K, double alpha, const double* __restrict__ A, int64_t lda,
             const double* __restrict__ B, int64_t ldb, double beta, double* __restrict__ C, int64_t ldc,
             double* __restrict__ part, int64_t kchunk) {
  constexpr int BM = 16 * TM, BN = 16 * TM;
  constexpr int LA = BM * BK / NT;   // elements of A (and of B) each thread loads per tile
  __shared__ __align__(16) double As[BK][BM];
  __shared__ __align__(16) double Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * BM;
  const int64_t n0 = static_cast<int64_t>(blockIdx.y) * BN;
  const int64_t kbeg = static_cast<int64_t>(blockIdx.z) * kchunk;
  const int64_t kend = min(K, kbeg + kchunk);

  double acc[TM][TM];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) acc[i][j] = 0.0;

  // A tile BM x BK: untransposed, consecutive threads walk the BM rows;
  // transposed, they walk the BK entries of one row of op(A).  B likewise.
  double ra[LA], rb[LA];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + r * NT;
      int i, kk;
      if (!TA) { i = e % BM; kk = e / BM; } else { kk = e % BK; i = e / BK; }
      const int64_t gi = m0 + i, gk = k0 + kk;
      double v = 0.0;
      if (gi < M && gk < kend) v = TA ? A[gk + gi * lda] : A[gi + gk * lda];
      ra[r] = v;
    }
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + r * NT;
      int j, kk;
      if (!TB) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
      const int64_t gj = n0 + j, gk = k0 + kk;
      double v = 0.0;
      if (gj < N && gk < kend) v = TB ? B[gj + gk * ldb] : B[gk + gj * ldb];
      rb[r] = v;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + r * NT;
      if (!TA) As[e / BM][e % BM] = ra[r]; else As[e % BK][e / BK] = ra[r];
      if (!TB) Bs[e % BK][e / BK] = rb[r]; else Bs[e / BN][e % BN] = rb[r];
    }
  };

  if (kbeg < kend) load(kbeg);
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    store();
    __syncthreads();
    if (k0 + BK < kend) load(k0 + BK);  // prefetch the next tile into registers
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[TM], b[TM];
#pragma unroll
      for (int h = 0; h < TM; h += 2) {
        const double2 av = *reinterpret_cast<const double2*>(&As[kk][tx * TM + h]);
        const double2 bv = *reinterpret_cast<const double2*>(&Bs[kk][ty * TM + h]);
        a[h] = av.x; a[h + 1] = av.y;
        b[h] = bv.x; b[h + 1] = bv.y;
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int j = 0; j < TM; ++j) {
    const int64_t gj = n0 + ty * TM + j;
    if (gj >= N) continue;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t gi = m0 + tx * TM + i;
      if (gi >= M) continue;
      if (part) {
        part[static_cast<int64_t>(blockIdx.z) * M * N + gi + gj * M] = acc[i][j];
      } else {
        double* c = C + gi + gj * ldc;
        *c = (beta == 0.0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *c);
      }
    }
  }
}

__global__ void splitk_reduce_kernel(int64_t M, int64_t N, int splits, double alpha,
                                     const double* __restrict__ part, double beta, double* __restrict__ C,
                                     int64_t ldc) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= M * N) return;
  const int64_t i = t % M, j = t / M;
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += part[z * M * N + t];
  double* c = C + i + j * ldc;
  *c = (beta == 0.0) ? alpha * s : fma(alpha, s, beta * *c);
}

__global__ void scale_kernel(int64_t M, int64_t N, double beta, double* __restrict__ C, int64_t ldc) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= M * N) return;
  double* c = C + t % M + (t / M) * ldc;
  *c = (beta == 0.0) ? 0.0 : beta * *c;
}

namespace {

struct Plan { int splits; int64_t kchunk; int tm; };

// Choose the tile (64 or 32 square) and the K split: minimise the modelled
// time of the busiest SM (units of tile x kchunk handed out evenly over the
// SMs, FP64-bound; the 32 tile issues about 15 % more per flop) plus the
// memory-bound reduction of the partial sums.
Plan plan_gemm(int64_t M, int64_t N, int64_t K, int64_t work_elems) {
  Plan best{1, ((K + BK - 1) / BK) * BK, 4};
  double best_t = 1e300;
  const double fma_per_s = 2.0 * 1.9e9;   // one SM's DFMA rate
  for (int tm = 4; tm >= 2; tm -= 2) {
    const int bm = 16 * tm;
    const int64_t tiles = ((M + bm - 1) / bm) * ((N + bm - 1) / bm);
    const double eff = (tm == 4) ? 1.0 : 1.15;
    for (int s = 1; s <= 64; ++s) {
      int64_t kc = (K + s - 1) / s;
      kc = ((kc + BK - 1) / BK) * BK;
      if (s > 1 && kc < 64) break;
      const int se = static_cast<int>((K + kc - 1) / kc);
      if (se > 1 && se * M * N > work_elems) break;
      const int64_t units = tiles * se;
      const int64_t per_sm = (units + kNumSMs - 1) / kNumSMs;
      double t = eff * per_sm * static_cast<double>(bm * bm) * kc / fma_per_s + 2e-6;
      if (se > 1) t += 4e-6 + (se + 2.0) * M * N * 8.0 / 5.0e12;
      if (t < best_t * 0.999) { best_t = t; best = Plan{se, kc, tm}; }
    }
  }
  return best;
}

}  // namespace

int64_t gemm_f64_work_elems(int64_t m, int64_t n, int64_t k) {
  Plan p = plan_gemm(m, n, k, INT64_MAX / 4);
  return p.splits > 1 ? p.splits * m * n : 0;
}

cudaError_t gemm_f64(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k,
                     double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                     double beta, double* C, int64_t ldc, double* work, int64_t work_elems) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (k <= 0 || alpha == 0.0) {
    if (beta == 1.0) return cudaSuccess;
    const int64_t tot = m * n;
    scale_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, s>>>(m, n, beta, C, ldc);
    note_launch();
    return cudaGetLastError();
  }
  Plan p = plan_gemm(m, n, k, work ? work_elems : 0);
  const ProfToken tok = prof_begin(s, kProfGemm);
  const int bm = 16 * p.tm;
  dim3 grid(static_cast<unsigned>((m + bm - 1) / bm), static_cast<unsigned>((n + bm - 1) / bm),
            static_cast<unsigned>(p.splits));
  double* part = p.splits > 1 ? work : nullptr;
#define RUTV_GEMM_LAUNCH(TA_, TB_, TM_)                                                              \
  dgemm_kernel<TA_, TB_, TM_><<<grid, NT, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, part, \
                                                 p.kchunk)
  if (p.tm == 4) {
    if (!ta && !tb) RUTV_GEMM_LAUNCH(false, false, 4);
    else if (ta && !tb) RUTV_GEMM_LAUNCH(true, false, 4);
    else if (!ta && tb) RUTV_GEMM_LAUNCH(false, true, 4);
    else RUTV_GEMM_LAUNCH(true, true, 4);
  } else {
    if (!ta && !tb) RUTV_GEMM_LAUNCH(false, false, 2);
    else if (ta && !tb) RUTV_GEMM_LAUNCH(true, false, 2);
    else if (!ta && tb) RUTV_GEMM_LAUNCH(false, true, 2);
    else RUTV_GEMM_LAUNCH(true, true, 2);
  }
#undef RUTV_GEMM_LAUNCH
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && p.splits > 1) {
    const int64_t tot = m * n;
    splitk_reduce_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, s>>>(
        m, n, p.splits, alpha, part, beta, C, ldc);
    note_launch();
    e = cudaGetLastError();
  }
  // algorithmic work: 2 m n k flops; one read of A, B (and C if beta != 0), one write of C
  prof_end(s, tok, 2.0 * m * n * k,
           8.0 * (m * k + k * n + m * n * (beta != 0.0 ? 2.0 : 1.0)));
  return e;
}

}  // namespace rutv

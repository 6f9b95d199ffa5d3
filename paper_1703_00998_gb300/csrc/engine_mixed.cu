// The mixed-precision form of the randUTV step loop (Fig. 4): the same
// method with T, U and V stored in FP32 and every O(n^3) product (sketch,
// block-reflector applications, small rotations) on the FP32 pipe, while
// each panel is up-cast to FP64 for its Householder QR, its compact-WY
// factor and the small SVD (Section 2.4, Remark 1).  The FP64 reflectors,
// S, Us and Vs are rounded once to FP32 for their applications.
//
// Error budget: errors of the sketch only change which subspace a step
// captures (U and V remain products of exactly orthogonal FP64-built
// transforms rounded once), so they do not enter the residual; the
// applications and the FP32 storage do, at the level of FP32 rounding.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include "common.cuh"
#include "internal.h"

namespace rutv {
namespace {

__global__ void f32_to_f64_kernel(int64_t m, int64_t n, const float* __restrict__ A, int64_t lda,
                                  double* __restrict__ B, int64_t ldb) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= m * n) return;
  const int64_t i = t % m, j = t / m;
  B[i + j * ldb] = static_cast<double>(A[i + j * lda]);
}

__global__ void f64_to_f32_kernel(int64_t m, int64_t n, const double* __restrict__ A, int64_t lda,
                                  float* __restrict__ B, int64_t ldb) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= m * n) return;
  const int64_t i = t % m, j = t / m;
  B[i + j * ldb] = static_cast<float>(A[i + j * lda]);
}

__global__ void f32_transpose_to_f64_kernel(int64_t m, int64_t n, const float* __restrict__ A, int64_t lda,
                                            double* __restrict__ B, int64_t ldb) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= m * n) return;
  const int64_t i = t % m, j = t / m;
  B[j + i * ldb] = static_cast<double>(A[i + j * lda]);
}

__global__ void f32_fill_kernel(int64_t m, int64_t n, float* X, int64_t ldx, float v) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= m * n) return;
  X[t % m + (t / m) * ldx] = v;
}

__global__ void f32_identity_kernel(int64_t n, float* X, int64_t ldx) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= n * n) return;
  const int64_t i = t % n, j = t / n;
  X[i + j * ldx] = (i == j) ? 1.f : 0.f;
}

__global__ void f32_set_diag_kernel(int64_t p, const double* d, float* X, int64_t ldx) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t < p) X[t + t * ldx] = static_cast<float>(d[t]);
}

__global__ void f32_sumsq_kernel(int64_t m, int64_t n, const float* X, int64_t ldx, double* part) {
  __shared__ double red[8];
  double s = 0.0;
  const int64_t tot = m * n;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < tot;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double v = X[t % m + (t / m) * ldx];
    s = fma(v, v, s);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x) / 32; ++w) a += red[w];
    part[blockIdx.x] = a;
  }
}

__global__ void sum_kernel(int nparts, const double* part, double* out) {
  __shared__ double red[8];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x) / 32; ++w) a += red[w];
    *out = a;
  }
}

inline unsigned blocks_for(int64_t n) { return static_cast<unsigned>((n + 255) / 256); }

cudaError_t up(cudaStream_t s, int64_t m, int64_t n, const float* A, int64_t lda, double* B, int64_t ldb) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  f32_to_f64_kernel<<<blocks_for(m * n), 256, 0, s>>>(m, n, A, lda, B, ldb);
  note_launch();
  return cudaGetLastError();
}

cudaError_t down(cudaStream_t s, int64_t m, int64_t n, const double* A, int64_t lda, float* B, int64_t ldb) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  f64_to_f32_kernel<<<blocks_for(m * n), 256, 0, s>>>(m, n, A, lda, B, ldb);
  note_launch();
  return cudaGetLastError();
}

cudaError_t fill32(cudaStream_t s, int64_t m, int64_t n, float* X, int64_t ldx) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  f32_fill_kernel<<<blocks_for(m * n), 256, 0, s>>>(m, n, X, ldx, 0.f);
  note_launch();
  return cudaGetLastError();
}

cudaError_t copy32(cudaStream_t s, int64_t m, int64_t n, const float* A, int64_t lda, float* B, int64_t ldb) {
  if (m <= 0 || n <= 0 || A == B) return cudaSuccess;
  return cudaMemcpy2DAsync(B, ldb * sizeof(float), A, lda * sizeof(float), m * sizeof(float), n,
                           cudaMemcpyDeviceToDevice, s);
}

constexpr int kSumBlocks = 2 * kNumSMs;

cudaError_t sumsq32(cudaStream_t s, int64_t m, int64_t n, const float* X, int64_t ldx, double* part, double* out) {
  f32_sumsq_kernel<<<kSumBlocks, 256, 0, s>>>(m, n, X, ldx, part);
  sum_kernel<<<1, 256, 0, s>>>(kSumBlocks, part, out);
  note_launch(2);
  return cudaGetLastError();
}

// Depth of the ring of per-step reflectors and small factors that the U/V
// stream reads while the T chain goes on with the next steps.
constexpr int kRing = 3;

// Workspace of the mixed form.
struct MWork {
  // FP32
  float *G, *Y, *Z, *Vv, *Vu, *S, *Us, *Vs, *W1, *W2, *tmp, *gws;
  float *Vvr[kRing], *Vur[kRing], *Svr[kRing], *Sur[kRing], *Usr[kRing], *Vsr[kRing];
  float *W1u, *W2u, *tmpu, *gwsu;
  float *tmps, *gwss;   // the SVD lane's rotation buffer and GEMM partials
  // FP64
  double *G64, *Y64, *Z64, *P64, *Vv64, *Vu64, *tau, *R, *Rt, *gram, *S64, *Us64, *Vs64, *d, *part, *jws, *gws64,
      *red, *scal;
  void* oz = nullptr;   // workspace of the sliced sketch products (gemm_oz_sketch), or null
  size_t ozb = 0;
  void* ozX = nullptr;  // the slices of X^T, shared by a step's X^T G and X^T Z (or null)
  size_t ozXb = 0;
  int64_t gws_elems, gws64_elems;
  unsigned* flags;
  void* base;
};

size_t al(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

unsigned* slot_of(unsigned* flags, int i) { return flags + 4 * i; }

__global__ void f64_transpose_kernel(int64_t m, int64_t n, const double* A, int64_t lda, double* B, int64_t ldb) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= m * n) return;
  B[t / m + (t % m) * ldb] = A[t % m + (t / m) * lda];
}

cudaError_t transpose_f64(cudaStream_t s, int64_t m, int64_t n, const double* A, int64_t lda, double* B,
                          int64_t ldb) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  f64_transpose_kernel<<<static_cast<unsigned>((m * n + 255) / 256), 256, 0, s>>>(m, n, A, lda, B, ldb);
  note_launch();
  return cudaGetLastError();
}

cudaError_t mwork_alloc(cudaStream_t s, int64_t m, int64_t n, int b, MWork* w) {
  const int64_t mx = std::max(m, n), bb = static_cast<int64_t>(b) * b;
  w->gws_elems = std::max<int64_t>(24 * mx * b, 64 * bb);
  w->gws64_elems = std::max<int64_t>(64 * bb, 4 * mx * b);
  struct I32 { float** p; int64_t n; };
  struct I64 { double** p; int64_t n; };
  I32 f[] = {{&w->G, m * b}, {&w->Y, n * b}, {&w->Z, m * b}, {&w->Vv, mx * b}, {&w->Vu, mx * b}, {&w->S, bb},
             {&w->Us, bb}, {&w->Vs, bb}, {&w->W1, mx * b}, {&w->W2, mx * b}, {&w->tmp, mx * b},
             {&w->gws, w->gws_elems},
             {&w->Vvr[0], mx * b}, {&w->Vvr[1], mx * b}, {&w->Vvr[2], mx * b},
             {&w->Vur[0], mx * b}, {&w->Vur[1], mx * b}, {&w->Vur[2], mx * b},
             {&w->Svr[0], bb}, {&w->Svr[1], bb}, {&w->Svr[2], bb}, {&w->Sur[0], bb}, {&w->Sur[1], bb},
             {&w->Sur[2], bb}, {&w->Usr[0], bb}, {&w->Usr[1], bb}, {&w->Usr[2], bb}, {&w->Vsr[0], bb},
             {&w->Vsr[1], bb}, {&w->Vsr[2], bb},
             {&w->W1u, mx * b}, {&w->W2u, mx * b}, {&w->tmpu, mx * b}, {&w->gwsu, w->gws_elems},
             {&w->tmps, mx * b}, {&w->gwss, w->gws_elems}};
  static_assert(kRing == 3, "ring buffers listed above");
  I64 d[] = {{&w->G64, m * b}, {&w->Y64, mx * b}, {&w->Z64, mx * b}, {&w->P64, mx * b}, {&w->Vv64, mx * b}, {&w->Vu64, mx * b},
             {&w->tau, b}, {&w->R, bb}, {&w->Rt, bb}, {&w->gram, bb}, {&w->S64, bb}, {&w->Us64, bb},
             {&w->Vs64, bb}, {&w->d, b}, {&w->part, panel_qr_part_elems(mx, b)}, {&w->jws, jacobi_work_elems(b)},
             {&w->gws64, w->gws64_elems}, {&w->red, kSumBlocks}, {&w->scal, 8}};
  size_t total = al(4 * kFlagSlots * sizeof(unsigned));
  for (auto& x : f) total += al(static_cast<size_t>(x.n) * sizeof(float));
  for (auto& x : d) total += al(static_cast<size_t>(x.n) * sizeof(double));
  cudaError_t e = cudaMallocAsync(&w->base, total, s);
  if (e != cudaSuccess) return e;
  char* p = static_cast<char*>(w->base);
  for (auto& x : d) { *x.p = reinterpret_cast<double*>(p); p += al(static_cast<size_t>(x.n) * sizeof(double)); }
  for (auto& x : f) { *x.p = reinterpret_cast<float*>(p); p += al(static_cast<size_t>(x.n) * sizeof(float)); }
  w->flags = reinterpret_cast<unsigned*>(p);
  return cudaMemsetAsync(w->flags, 0, 4 * kFlagSlots * sizeof(unsigned), s);
}

// Where each FP32 product runs.  The sketch products (kSketch) only decide
// which subspace a step captures, so with tensor_cores = 1 they run on the
// tcgen05 tensor cores (3xTF32, FP32 accumulation in tensor memory).  The
// products of the block-reflector applications and rotations (kUpdate)
// enter the backward error directly and stay on the FP32 CUDA cores (round
// to nearest, split sums in FP64): the tensor-core accumulator does not
// round to nearest, and putting even the inner-dimension-b updates on it
// measured a residual of 3e-6 at n = 8000 (1e-6 is the target), and slower.
enum GemmKind { kSketch = 0, kUpdate = 1 };

struct Mg {
  bool tc;
  bool split;   // sketch on the tensor cores as 3xTF32 (else one TF32 product)
  int* err;
  float* gws;
  int64_t ge;
  cudaError_t run(cudaStream_t s, GemmKind kind, bool ta, bool tb, int64_t m, int64_t n, int64_t k, float alpha,
                  const float* A, int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                  int64_t ldc) const {
    if (kind == kSketch && tc && gemm_tc_supported(A, lda, B, ldb, m, n, k))
      return gemm_tc(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, gws, ge, err, split);
    return gemm_f32(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, gws, ge);
  }
};

// C (rows x cols) <- C (I - Vx S Vx^T), Vx cols x w, all FP32.
cudaError_t wy_right32(cudaStream_t s, const Mg& g, int64_t rows, int64_t cols, float* C, int64_t ldc,
                       const float* Vx, const float* S, int w, float* W1, float* W2) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  cudaError_t e;
  if ((e = g.run(s, kUpdate, false, false, rows, w, cols, 1.f, C, ldc, Vx, cols, 0.f, W1, rows))) return e;
  if ((e = g.run(s, kUpdate, false, false, rows, w, w, 1.f, W1, rows, S, w, 0.f, W2, rows))) return e;
  return g.run(s, kUpdate, false, true, rows, cols, w, -1.f, W2, rows, Vx, cols, 1.f, C, ldc);
}

// C (rows x cols) <- (I - Vx S Vx^T)^T C, Vx rows x w.
cudaError_t wy_left_t32(cudaStream_t s, const Mg& g, int64_t rows, int64_t cols, float* C, int64_t ldc,
                        const float* Vx, const float* S, int w, float* W1, float* W2) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  cudaError_t e;
  if ((e = g.run(s, kUpdate, true, false, w, cols, rows, 1.f, Vx, rows, C, ldc, 0.f, W1, w))) return e;
  if ((e = g.run(s, kUpdate, true, false, w, cols, w, 1.f, S, w, W1, w, 0.f, W2, w))) return e;
  return g.run(s, kUpdate, false, false, rows, cols, w, -1.f, Vx, rows, W2, w, 1.f, C, ldc);
}

cudaError_t rot_right32(cudaStream_t s, const Mg& g, int64_t rows, int w, float* X, int64_t ldx, const float* Q,
                        float* tmp) {
  if (rows <= 0 || w <= 0) return cudaSuccess;
  cudaError_t e = g.run(s, kUpdate, false, false, rows, w, w, 1.f, X, ldx, Q, w, 0.f, tmp, rows);
  if (e) return e;
  return copy32(s, rows, w, tmp, rows, X, ldx);
}

cudaError_t rot_left_t32(cudaStream_t s, const Mg& g, int w, int64_t cols, float* X, int64_t ldx, const float* Q,
                         float* tmp) {
  if (cols <= 0 || w <= 0) return cudaSuccess;
  cudaError_t e = g.run(s, kUpdate, true, false, w, cols, w, 1.f, Q, w, X, ldx, 0.f, tmp, w);
  if (e) return e;
  return copy32(s, w, cols, tmp, w, X, ldx);
}

// Householder QR of an FP64 panel P64 (k x w) with its compact-WY factor; the
// FP32 copies Vx32 (k x w) and S32 (w x w) are what the applications use.
cudaError_t panel_wy(cudaStream_t s, int64_t k, int w, double* P64, double* tau, double* V64, double* R,
                     double* gram, double* S64, float* V32, float* S32, MWork& mw, unsigned* bar) {
  cudaError_t e;
  if ((e = panel_qr(s, k, w, P64, k, tau, V64, R, mw.part, bar))) return e;
  if ((e = gemm_f64(s, true, false, w, w, k, 1.0, V64, k, V64, k, 0.0, gram, w, mw.gws64, mw.gws64_elems))) return e;
  if ((e = tfactor_from_gram(s, w, gram, tau, S64))) return e;
  if ((e = down(s, k, w, V64, k, V32, k))) return e;
  return down(s, w, w, S64, w, S32, w);
}

}  // namespace
}  // namespace rutv

using namespace rutv;

namespace {
int mstatus(cudaError_t e, const char* where) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  set_last_error(buf);
  return RANDUTV_ECUDA;
}
}  // namespace

#define RUTV_MCK(call)                                           \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) { st = mstatus(e_, #call); goto done; } \
  } while (0)

extern "C" int randutv_factor_mixed(int64_t m, int64_t n, const float* A, int64_t lda, int b, int q, double tol,
                                    float* U, int64_t ldu, float* T, int64_t ldt, float* V, int64_t ldv,
                                    int64_t* k_reached, const randutv_opts* opts_in) {
  randutv_opts opts;
  if (opts_in) opts = *opts_in; else randutv_opts_default(&opts);
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (!A) return -3;
  if (lda < m) return -4;
  if (b < 1) return -5;
  if (q < 0) return -6;
  if (!(tol >= 0.0) || std::isinf(tol)) return -7;
  if (opts.form_uv && !U) return -8;
  if (opts.form_uv && ldu < m) return -9;
  if (!T) return -10;
  if (ldt < m || (static_cast<const void*>(T) == static_cast<const void*>(A) && ldt != lda)) return -11;
  if (opts.form_uv && !V) return -12;
  if (opts.form_uv && ldv < n) return -13;
  if (!k_reached) return -14;
  if (opts.p != 0 || opts.max_sweeps < 1 ||
      (opts.sketch_prec != RANDUTV_SKETCH_OZAKI && opts.sketch_prec != RANDUTV_SKETCH_3XTF32 &&
       opts.sketch_prec != RANDUTV_SKETCH_TF32))
    return -15;

  const int64_t mn = std::min(m, n);
  if (b > mn) b = static_cast<int>(mn);
  if (b > 256) { set_last_error("block size above 256"); return RANDUTV_EUNSUPPORTED; }
  const bool uv = opts.form_uv != 0;
  cudaStream_t s = current_stream();
  MWork w{};
  Lanes L;
  Mg gT{}, gU{};
  int st = RANDUTV_OK;
  double h_norm2 = 0.0, normA = 0.0;
  int64_t g_off = 0;
  *k_reached = mn;
  const int64_t nsteps = std::min((m + b - 1) / b, (n + b - 1) / b);
  {
    cudaError_t e = mwork_alloc(s, m, n, b, &w);
    if (e == cudaSuccess && opts.sketch_prec == RANDUTV_SKETCH_OZAKI) {
      if (!gemm_oz_supported()) {
        set_last_error("sliced sketch: cuTensorMapEncodeTiled is not available");
        if (w.base) cudaFreeAsync(w.base, s);
        cudaStreamSynchronize(s);
        return RANDUTV_EUNSUPPORTED;
      }
      const int64_t mx = std::max(m, n);
      w.ozb = gemm_oz_sketch_work_bytes(mx, b, mx);   // bounds every sketch product of the factorization
      w.ozXb = gemm_oz_keep_bytes(mx, b, mx, true);
      e = cudaMallocAsync(&w.oz, w.ozb, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(w.oz, 0, gemm_oz_head_bytes(), s);
      if (e == cudaSuccess && q > 0) e = cudaMallocAsync(&w.ozX, w.ozXb, s);
    }
    if (e != cudaSuccess) {
      if (w.ozX) cudaFreeAsync(w.ozX, s);
      if (w.oz) cudaFreeAsync(w.oz, s);
      if (w.base) cudaFreeAsync(w.base, s);
      cudaStreamSynchronize(s);
      cudaGetLastError();
      set_last_error("workspace allocation failed");
      return e == cudaErrorMemoryAllocation ? RANDUTV_ENOMEM : RANDUTV_ECUDA;
    }
  }
  {
    const bool tcl = opts.tensor_cores != 0;
    const bool split = opts.sketch_prec != RANDUTV_SKETCH_TF32;
    int* tc_err = reinterpret_cast<int*>(slot_of(w.flags, 3) + 2);
    gT = Mg{tcl, split, tc_err, w.gws, w.gws_elems};
    gU = Mg{tcl, split, tc_err, w.gwsu, w.gws_elems};
  }
  RUTV_MCK(L.open(s, opts.overlap != 0));
  {
    cudaStream_t sT = L.t, sU = L.uv, sS = L.sv;
    const Mg gS{false, false, gT.err, w.gwss, w.gws_elems};   // SVD lane: the rotations (CUDA cores)
    int prev_sl = -1;   // ring slot of the previous randomized step (its rotations of T run on the SVD lane)
    RUTV_MCK(copy32(sT, m, n, A, lda, T, ldt));
    if (uv) {
      f32_identity_kernel<<<blocks_for(m * m), 256, 0, sU>>>(m, U, ldu);
      f32_identity_kernel<<<blocks_for(n * n), 256, 0, sU>>>(n, V, ldv);
      note_launch(2);
      RUTV_MCK(cudaGetLastError());
    }
    RUTV_MCK(sumsq32(sT, m, n, T, ldt, w.red, w.scal));
    RUTV_MCK(cudaMemcpyAsync(&h_norm2, w.scal, sizeof(double), cudaMemcpyDeviceToHost, sT));
    RUTV_MCK(cudaStreamSynchronize(sT));
    if (!std::isfinite(h_norm2)) { st = RANDUTV_ENAN; goto done; }
    normA = std::sqrt(h_norm2);

    for (int64_t i = 1; i <= nsteps; ++i) {
      const int64_t r0 = b * (i - 1);
      const int64_t r1 = std::min<int64_t>(r0 + b, m), c1 = std::min<int64_t>(r0 + b, n);
      const int64_t kr = m - r0, kc = n - r0;
      const int sl = static_cast<int>((i - 1) % kRing);
      float* X = T + r0 + r0 * ldt;
      if (tol > 0.0) {
        double t2 = 0.0;
        RUTV_MCK(sumsq32(sT, kr, kc, X, ldt, w.red, w.scal));
        RUTV_MCK(cudaMemcpyAsync(&t2, w.scal, sizeof(double), cudaMemcpyDeviceToHost, sT));
        RUTV_MCK(cudaStreamSynchronize(sT));
        if (!std::isfinite(t2)) { st = RANDUTV_ENAN; goto done; }
        if (std::sqrt(t2) <= tol * normA) { *k_reached = r0; break; }
      }
      // the ring slot of this step is free once the U/V stream finished step i - kRing
      if (i > kRing) RUTV_MCK(cudaStreamWaitEvent(sT, L.done[sl], 0));
      float *Vv = w.Vvr[sl], *Vu = w.Vur[sl], *Sv = w.Svr[sl], *Su = w.Sur[sl], *Us = w.Usr[sl], *Vs = w.Vsr[sl];
      if (r1 < m && c1 < n) {
        // sketch on the FP32 pipe; G from the same Philox stream (or the injected one) rounded to FP32
        if (opts.g_inject) {
          RUTV_MCK(down(sT, kr, b, opts.g_inject + g_off, kr, w.G, kr));
          if (opts.g_capture)
            RUTV_MCK(cudaMemcpyAsync(opts.g_capture + g_off, opts.g_inject + g_off, kr * b * sizeof(double),
                                     cudaMemcpyDeviceToDevice, sT));
        } else {
          RUTV_MCK(launch_gaussian(sT, opts.seed, i, kr, b, w.G64, kr));
          RUTV_MCK(down(sT, kr, b, w.G64, kr, w.G, kr));
          if (opts.g_capture)
            RUTV_MCK(cudaMemcpyAsync(opts.g_capture + g_off, w.G64, kr * b * sizeof(double),
                                     cudaMemcpyDeviceToDevice, sT));
        }
        if (w.oz) {
          // sliced sketch: the FP32 trailing block exactly, G / Y / Z to 35 bits, FP64 results
          const double* G64 = opts.g_inject ? opts.g_inject + g_off : w.G64;
          int* oz_err = reinterpret_cast<int*>(slot_of(w.flags, 3) + 2);
          // X^T is sliced once for X^T G and every X^T Z of the step (X does not change in between)
          OzKeep kx{w.ozX, w.ozXb, false};
          OzKeep* kxp = w.ozX ? &kx : nullptr;
          RUTV_MCK(gemm_oz_sketch(sT, true, false, kc, b, kr, X, ldt, G64, kr, w.Y64, kc, w.oz, w.ozb, oz_err, kxp));
          for (int j = 0; j < q; ++j) {
            RUTV_MCK(gemm_oz_sketch(sT, false, false, kr, b, kc, X, ldt, w.Y64, kc, w.Z64, kr, w.oz, w.ozb, oz_err));
            RUTV_MCK(gemm_oz_sketch(sT, true, false, kc, b, kr, X, ldt, w.Z64, kr, w.Y64, kc, w.oz, w.ozb, oz_err,
                                    kxp));
          }
        } else {
          RUTV_MCK(gT.run(sT, kSketch, true, false, kc, b, kr, 1.f, X, ldt, w.G, kr, 0.f, w.Y, kc));
          for (int j = 0; j < q; ++j) {
            RUTV_MCK(gT.run(sT, kSketch, false, false, kr, b, kc, 1.f, X, ldt, w.Y, kc, 0.f, w.Z, kr));
            RUTV_MCK(gT.run(sT, kSketch, true, false, kc, b, kr, 1.f, X, ldt, w.Z, kr, 0.f, w.Y, kc));
          }
          RUTV_MCK(up(sT, kc, b, w.Y, kc, w.Y64, kc));
        }
        g_off += kr * b;
        // QR(Y) in FP64
        RUTV_MCK(panel_wy(sT, kc, b, w.Y64, w.tau, w.Vv64, w.Rt, w.gram, w.S64, Vv, Sv, w, slot_of(w.flags, 0)));
        RUTV_MCK(cudaEventRecord(L.v[sl], sT));
        // rows I2 of the previous step are rotated on the SVD lane: wait for it
        if (prev_sl >= 0) RUTV_MCK(cudaStreamWaitEvent(sT, L.g[prev_sl], 0));
        RUTV_MCK(wy_right32(sT, gT, m, kc, T + r0 * ldt, ldt, Vv, Sv, b, w.W1, w.W2));
        if (uv) {
          RUTV_MCK(cudaStreamWaitEvent(sU, L.v[sl], 0));
          RUTV_MCK(wy_right32(sU, gU, n, kc, V + r0 * ldv, ldv, Vv, Sv, b, w.W1u, w.W2u));
        }
        // QR of the panel in FP64
        RUTV_MCK(up(sT, kr, b, X, ldt, w.P64, kr));
        RUTV_MCK(panel_wy(sT, kr, b, w.P64, w.tau, w.Vu64, w.R, w.gram, w.S64, Vu, Su, w, slot_of(w.flags, 1)));
        if (uv) {
          RUTV_MCK(cudaEventRecord(L.u[sl], sT));
          RUTV_MCK(cudaStreamWaitEvent(sU, L.u[sl], 0));
          RUTV_MCK(wy_right32(sU, gU, m, kr, U + r0 * ldu, ldu, Vu, Su, b, w.W1u, w.W2u));
        }
        RUTV_MCK(wy_left_t32(sT, gT, kr, kc - b, T + r0 + c1 * ldt, ldt, Vu, Su, b, w.W1, w.W2));
        RUTV_MCK(fill32(sT, kr, b, X, ldt));
        RUTV_MCK(cudaEventRecord(L.e[sl], sT));
        // small SVD in FP64 and the rotations of T on the SVD lane (they touch
        // rows I2 and columns J2 only; the next step's sketch reads neither)
        RUTV_MCK(cudaStreamWaitEvent(sS, L.e[sl], 0));
        RUTV_MCK(jacobi_svd(sS, b, w.R, b, w.Us64, w.d, w.Vs64, opts.max_sweeps, w.jws, slot_of(w.flags, 2)));
        f32_set_diag_kernel<<<(b + 127) / 128, 128, 0, sS>>>(b, w.d, X, ldt);
        note_launch();
        RUTV_MCK(cudaGetLastError());
        RUTV_MCK(down(sS, b, b, w.Us64, b, Us, b));
        RUTV_MCK(down(sS, b, b, w.Vs64, b, Vs, b));
        RUTV_MCK(cudaEventRecord(L.s[sl], sS));
        if (uv) {
          RUTV_MCK(cudaStreamWaitEvent(sU, L.s[sl], 0));
          RUTV_MCK(rot_right32(sU, gU, m, b, U + r0 * ldu, ldu, Us, w.tmpu));
          RUTV_MCK(rot_right32(sU, gU, n, b, V + r0 * ldv, ldv, Vs, w.tmpu));
        }
        RUTV_MCK(rot_left_t32(sS, gS, b, kc - b, T + r0 + c1 * ldt, ldt, Us, w.tmps));
        RUTV_MCK(rot_right32(sS, gS, r0, b, T + r0 * ldt, ldt, Vs, w.tmps));
        RUTV_MCK(cudaEventRecord(L.g[sl], sS));
        prev_sl = sl;
      } else {
        // last block: QR first (tall or square) or QR of the rows (wide), then the FP64 SVD
        if (prev_sl >= 0) RUTV_MCK(cudaStreamWaitEvent(sT, L.g[prev_sl], 0));
        int p;
        if (kr >= kc) {
          p = static_cast<int>(kc);
          RUTV_MCK(up(sT, kr, kc, X, ldt, w.P64, kr));
          RUTV_MCK(panel_wy(sT, kr, p, w.P64, w.tau, w.Vu64, w.R, w.gram, w.S64, Vu, Su, w, slot_of(w.flags, 1)));
          if (uv) {
            RUTV_MCK(cudaEventRecord(L.u[sl], sT));
            RUTV_MCK(cudaStreamWaitEvent(sU, L.u[sl], 0));
            RUTV_MCK(wy_right32(sU, gU, m, kr, U + r0 * ldu, ldu, Vu, Su, p, w.W1u, w.W2u));
          }
        } else {
          p = static_cast<int>(kr);
          f32_transpose_to_f64_kernel<<<blocks_for(kr * kc), 256, 0, sT>>>(kr, kc, X, ldt, w.P64, kc);
          note_launch();
          RUTV_MCK(cudaGetLastError());
          RUTV_MCK(panel_wy(sT, kc, p, w.P64, w.tau, w.Vv64, w.Rt, w.gram, w.S64, Vv, Sv, w, slot_of(w.flags, 0)));
          RUTV_MCK(wy_right32(sT, gT, m, kc, T + r0 * ldt, ldt, Vv, Sv, p, w.W1, w.W2));
          if (uv) {
            RUTV_MCK(cudaEventRecord(L.v[sl], sT));
            RUTV_MCK(cudaStreamWaitEvent(sU, L.v[sl], 0));
            RUTV_MCK(wy_right32(sU, gU, n, kc, V + r0 * ldv, ldv, Vv, Sv, p, w.W1u, w.W2u));
          }
          RUTV_MCK(transpose_f64(sT, p, p, w.Rt, p, w.R, p));
        }
        RUTV_MCK(jacobi_svd(sT, p, w.R, p, w.Us64, w.d, w.Vs64, opts.max_sweeps, w.jws, slot_of(w.flags, 2)));
        RUTV_MCK(fill32(sT, kr, kc, X, ldt));
        f32_set_diag_kernel<<<(p + 127) / 128, 128, 0, sT>>>(p, w.d, X, ldt);
        note_launch();
        RUTV_MCK(cudaGetLastError());
        RUTV_MCK(down(sT, p, p, w.Us64, p, Us, p));
        RUTV_MCK(down(sT, p, p, w.Vs64, p, Vs, p));
        if (uv) {
          RUTV_MCK(cudaEventRecord(L.s[sl], sT));
          RUTV_MCK(cudaStreamWaitEvent(sU, L.s[sl], 0));
          RUTV_MCK(rot_right32(sU, gU, m, p, U + r0 * ldu, ldu, Us, w.tmpu));
          RUTV_MCK(rot_right32(sU, gU, n, p, V + r0 * ldv, ldv, Vs, w.tmpu));
        }
        RUTV_MCK(rot_right32(sT, gT, r0, p, T + r0 * ldt, ldt, Vs, w.tmp));
      }
      if (uv) RUTV_MCK(cudaEventRecord(L.done[sl], sU));
    }
  }
  RUTV_MCK(L.join(s));
  RUTV_MCK(cudaStreamSynchronize(s));
  {
    unsigned h[4 * kFlagSlots];
    RUTV_MCK(cudaMemcpy(h, w.flags, sizeof(h), cudaMemcpyDeviceToHost));
    unsigned err = 0;
    for (int k = 0; k < kFlagSlots; ++k) err |= h[4 * k + 2];
    if (err & kDevErrTimeout) { set_last_error("device grid barrier timed out"); st = RANDUTV_ETIMEOUT; }
    else if (err & kDevErrNoConv) st = RANDUTV_ENOCONV;
  }
  if (prof_enabled()) prof_flush();
done:
  L.join(s);
  if (w.oz) cudaFreeAsync(w.oz, s);
  if (w.ozX) cudaFreeAsync(w.ozX, s);
  if (w.base) {
    cudaFreeAsync(w.base, s);
    cudaStreamSynchronize(s);
  }
  L.close();
  return st;
}

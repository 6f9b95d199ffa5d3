// The randUTV step loop (Fig. 4, Section 5.2) and the C ABI of include/randutv.h.
//
// The host walks the steps and queues kernels on one stream; T, U, V and
// every intermediate stay in device memory for the whole factorization, and
// each transform is applied as soon as it is formed (Section 5.2, first
// modification).  There is no host synchronisation inside the loop unless a
// tolerance asks for the trailing norm.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include "common.cuh"
#include "internal.h"

namespace rutv {

static cudaStream_t g_stream = nullptr;
cudaStream_t current_stream() { return g_stream; }

static thread_local char g_detail[256] = "";

void set_last_error(const char* msg) { snprintf(g_detail, sizeof(g_detail), "%s", msg); }

static int cuda_status(cudaError_t e, const char* where) {
  snprintf(g_detail, sizeof(g_detail), "%s: %s", where, cudaGetErrorString(e));
  return RANDUTV_ECUDA;
}

#define RUTV_CK(call)                                            \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) { st = cuda_status(e_, #call); goto done; } \
  } while (0)

// ---------------------------------------------------------------- utilities
__global__ void set_identity_kernel(int64_t n, double* X, int64_t ldx) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= n * n) return;
  const int64_t i = t % n, j = t / n;
  X[i + j * ldx] = (i == j) ? 1.0 : 0.0;
}

cudaError_t set_identity(cudaStream_t s, int64_t n, double* X, int64_t ldx) {
  if (n <= 0) return cudaSuccess;
  set_identity_kernel<<<static_cast<unsigned>((n * n + 255) / 256), 256, 0, s>>>(n, X, ldx);
  note_launch();
  return cudaGetLastError();
}

cudaError_t copy_matrix(cudaStream_t s, int64_t m, int64_t n, const double* A, int64_t lda, double* B,
                        int64_t ldb) {
  if (m <= 0 || n <= 0 || A == B) return cudaSuccess;
  return cudaMemcpy2DAsync(B, ldb * sizeof(double), A, lda * sizeof(double), m * sizeof(double), n,
                           cudaMemcpyDeviceToDevice, s);
}

__global__ void fill_kernel(int64_t m, int64_t n, double* X, int64_t ldx, double v) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= m * n) return;
  X[t % m + (t / m) * ldx] = v;
}

static cudaError_t fill(cudaStream_t s, int64_t m, int64_t n, double* X, int64_t ldx, double v) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  fill_kernel<<<static_cast<unsigned>((m * n + 255) / 256), 256, 0, s>>>(m, n, X, ldx, v);
  note_launch();
  return cudaGetLastError();
}

__global__ void set_diag_kernel(int64_t p, const double* d, double* X, int64_t ldx) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t < p) X[t + t * ldx] = d[t];
}

__global__ void transpose_kernel(int64_t m, int64_t n, const double* A, int64_t lda, double* B, int64_t ldb) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= m * n) return;
  const int64_t i = t % m, j = t / m;
  B[j + i * ldb] = A[i + j * lda];
}

static cudaError_t transpose(cudaStream_t s, int64_t m, int64_t n, const double* A, int64_t lda, double* B,
                             int64_t ldb) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  transpose_kernel<<<static_cast<unsigned>((m * n + 255) / 256), 256, 0, s>>>(m, n, A, lda, B, ldb);
  note_launch();
  return cudaGetLastError();
}

// Sum of squares of an m x n strided matrix: block partials, then one block.
__global__ void sumsq_partial_kernel(int64_t m, int64_t n, const double* X, int64_t ldx, double* part) {
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

__global__ void sumsq_final_kernel(int nparts, const double* part, double* out) {
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

constexpr int kSumsqBlocks = 2 * kNumSMs;

static cudaError_t sumsq(cudaStream_t s, int64_t m, int64_t n, const double* X, int64_t ldx, double* part,
                         double* out) {
  sumsq_partial_kernel<<<kSumsqBlocks, 256, 0, s>>>(m, n, X, ldx, part);
  note_launch();
  sumsq_final_kernel<<<1, 256, 0, s>>>(kSumsqBlocks, part, out);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------- block reflectors
// Where an FP64 product runs: the Ozaki-scheme tensor-core GEMM (gemm_oz.cu)
// when enabled and the product is large enough for its tiles, else the
// DFMA GEMM.  Each lane has its own split-K partials and slice workspace.
struct G64 {
  bool oz;
  void* ow;
  size_t owb;
  int* err;
  double* gws;
  int64_t ge;
  cudaError_t run(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                  int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                  OzKeep* keep = nullptr) const {
    if (oz && m >= 64 && n >= 32 && k >= 32 && gemm_oz_work_bytes(m, n, k) <= owb) {
      if (keep && keep->base && gemm_oz_keep_bytes(m, n, k, false) <= keep->bytes)
        return gemm_oz_keep(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ow, owb, err, keep);
      return gemm_oz(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ow, owb, err);
    }
    return gemm_f64(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, gws, ge);
  }
};
// C (rows x cols) <- C (I - Vx S Vx^T), Vx cols x w.
static cudaError_t wy_right(cudaStream_t s, int64_t rows, int64_t cols, double* C, int64_t ldc,
                            const double* Vx, const double* S, int w, double* W1, double* W2,
                            const G64& g) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  cudaError_t e;
  if ((e = g.run(s, false, false, rows, w, cols, 1.0, C, ldc, Vx, cols, 0.0, W1, rows))) return e;
  if ((e = g.run(s, false, false, rows, w, w, 1.0, W1, rows, S, w, 0.0, W2, rows))) return e;
  return g.run(s, false, true, rows, cols, w, -1.0, W2, rows, Vx, cols, 1.0, C, ldc);
}

// C (rows x cols) <- (I - Vx S Vx^T)^T C, Vx rows x w.
static cudaError_t wy_left_t(cudaStream_t s, int64_t rows, int64_t cols, double* C, int64_t ldc,
                             const double* Vx, const double* S, int w, double* W1, double* W2,
                             const G64& g) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  cudaError_t e;
  if ((e = g.run(s, true, false, w, cols, rows, 1.0, Vx, rows, C, ldc, 0.0, W1, w))) return e;
  if ((e = g.run(s, true, false, w, cols, w, 1.0, S, w, W1, w, 0.0, W2, w))) return e;
  return g.run(s, false, false, rows, cols, w, -1.0, Vx, rows, W2, w, 1.0, C, ldc);
}

// X (rows x w) <- X Q with Q w x w (through tmp).
static cudaError_t rot_right(cudaStream_t s, int64_t rows, int w, double* X, int64_t ldx, const double* Q,
                             double* tmp, const G64& g) {
  if (rows <= 0 || w <= 0) return cudaSuccess;
  cudaError_t e;
  if ((e = g.run(s, false, false, rows, w, w, 1.0, X, ldx, Q, w, 0.0, tmp, rows))) return e;
  return copy_matrix(s, rows, w, tmp, rows, X, ldx);
}

// X (w x cols) <- Q^T X with Q w x w (through tmp).
static cudaError_t rot_left_t(cudaStream_t s, int w, int64_t cols, double* X, int64_t ldx, const double* Q,
                              double* tmp, const G64& g) {
  if (cols <= 0 || w <= 0) return cudaSuccess;
  cudaError_t e;
  if ((e = g.run(s, true, false, w, cols, w, 1.0, Q, w, X, ldx, 0.0, tmp, w))) return e;
  return copy_matrix(s, w, cols, tmp, w, X, ldx);
}

// ------------------------------------------------------------- workspace
// The reflectors and small-SVD factors of a step live in a ring of
// Lanes::kSlots slots, so the U/V lane can still be applying step i's while
// the T lane forms step i+1's; W1u/W2u/tmpu/gwsu are the U/V lane's scratch.
struct Work {
  static constexpr int kR = Lanes::kSlots;
  double *G, *Y, *Z, *tau, *R, *Rt, *gram, *W1, *W2, *d, *tmp;
  double *Vvr[kR], *Vur[kR], *Svr[kR], *Sur[kR], *Usr[kR], *Vsr[kR];
  double *W1u, *W2u, *tmpu, *gwsu;
  double *tmps, *gwss;   // the SVD lane's rotation buffer and GEMM partials
  // over-sampling (p > 0): the Householder QR of the (b+p)-wide sketch, the
  // SVD of its R, the basis Z of the b dominant left singular vectors
  double *Vq, *Rq, *Sq, *Usq, *Vsq, *dq, *Eb, *jws2;
  double *gws, *part, *jws, *red, *scal;
  int64_t gws_elems;
  unsigned* flags;
  void* base;
  size_t bytes;
  void *ozT, *ozU, *ozS;   // Ozaki GEMM workspaces of the T, U/V and SVD lanes (or null)
  size_t ozb, ozbS;
  void* ozX;               // the slices of X^T, shared by a step's products X^T G and X^T Z (or null)
  size_t ozXb;
};

// Largest Ozaki workspace any product of the factorization needs: the
// first step's shapes bound every later one.
static size_t oz_budget(int64_t m, int64_t n, int b) {
  const int64_t mx = std::max(m, n);
  const int64_t sh[][3] = {{mx, b, mx}, {b, mx, mx}, {mx, mx, b}, {mx, b, b}, {b, mx, b}};
  size_t w = 0;
  for (auto& x : sh) w = std::max(w, gemm_oz_work_bytes(x[0], x[1], x[2]));
  return w;
}

static size_t align_up(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

static int64_t gemm_budget(int64_t mx, int b) {
  return std::max<int64_t>(24 * mx * b, 64ll * b * b);
}

static cudaError_t work_alloc(cudaStream_t s, int64_t m, int64_t n, int b, int pov, bool uv, Work* w) {
  const int64_t mx = std::max(m, n);
  const int64_t bb = static_cast<int64_t>(b) * b;
  const int64_t wv = b + pov;                  // sketch width
  const int64_t ww = wv * wv;
  const int64_t ov = pov > 0 ? 1 : 0;          // over-sampling buffers only when p > 0
  const int64_t ux = uv ? 1 : 0;   // the U/V lane's scratch only when U and V are formed
  struct Item { double** p; int64_t n; };
  w->gws_elems = gemm_budget(mx, static_cast<int>(wv));
  Item items[] = {
      {&w->G, m * wv}, {&w->Y, n * wv}, {&w->Z, m * wv},
      {&w->tau, wv}, {&w->R, bb}, {&w->Rt, bb}, {&w->gram, ww}, {&w->W1, mx * b},
      {&w->Vq, ov * mx * wv}, {&w->Rq, ov * ww}, {&w->Sq, ov * ww}, {&w->Usq, ov * ww}, {&w->Vsq, ov * ww},
      {&w->dq, ov * wv}, {&w->Eb, ov * mx * b}, {&w->jws2, ov * jacobi_work_elems(static_cast<int>(wv))},
      {&w->W2, mx * b}, {&w->d, b}, {&w->tmp, mx * b},
      {&w->Vvr[0], mx * b}, {&w->Vvr[1], mx * b}, {&w->Vvr[2], mx * b},
      {&w->Vur[0], mx * b}, {&w->Vur[1], mx * b}, {&w->Vur[2], mx * b},
      {&w->Svr[0], bb}, {&w->Svr[1], bb}, {&w->Svr[2], bb}, {&w->Sur[0], bb}, {&w->Sur[1], bb}, {&w->Sur[2], bb},
      {&w->Usr[0], bb}, {&w->Usr[1], bb}, {&w->Usr[2], bb}, {&w->Vsr[0], bb}, {&w->Vsr[1], bb}, {&w->Vsr[2], bb},
      {&w->W1u, ux * mx * b}, {&w->W2u, ux * mx * b}, {&w->tmpu, ux * mx * b}, {&w->gwsu, ux * w->gws_elems},
      {&w->tmps, mx * b}, {&w->gwss, w->gws_elems},
      {&w->gws, w->gws_elems}, {&w->part, panel_qr_part_elems(mx, static_cast<int>(wv))},
      {&w->jws, jacobi_work_elems(b)},
      {&w->red, kSumsqBlocks}, {&w->scal, 8},
  };
  static_assert(Work::kR == 3, "ring buffers listed above");
  size_t total = 0;
  for (auto& it : items) total += align_up(static_cast<size_t>(it.n) * sizeof(double));
  total += align_up(4 * kFlagSlots * sizeof(unsigned));
  cudaError_t e = cudaMallocAsync(&w->base, total, s);
  if (e != cudaSuccess) return e;
  w->bytes = total;
  char* p = static_cast<char*>(w->base);
  for (auto& it : items) {
    *it.p = reinterpret_cast<double*>(p);
    p += align_up(static_cast<size_t>(it.n) * sizeof(double));
  }
  w->flags = reinterpret_cast<unsigned*>(p);
  return cudaMemsetAsync(w->flags, 0, 4 * kFlagSlots * sizeof(unsigned), s);
}

static unsigned* slot(Work& w, int i) { return w.flags + 4 * i; }

// Read the error words of every barrier slot (after a stream sync).
static int device_status(Work& w) {
  unsigned h[4 * kFlagSlots];
  if (cudaMemcpy(h, w.flags, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return RANDUTV_ECUDA;
  unsigned err = 0;
  for (int i = 0; i < kFlagSlots; ++i) err |= h[4 * i + 2];
  if (err & kDevErrTimeout) { snprintf(g_detail, sizeof(g_detail), "device grid barrier timed out"); return RANDUTV_ETIMEOUT; }
  if (err & kDevErrNaN) return RANDUTV_ENAN;
  if (err & kDevErrNoConv) return RANDUTV_ENOCONV;
  return RANDUTV_OK;
}

}  // namespace rutv

using namespace rutv;

// ================================================================== C ABI
extern "C" {

void randutv_opts_default(randutv_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = RANDUTV_FP64;
  o->form_uv = 1;
  o->max_sweeps = 30;
  o->p = 0;
  o->seed = 998;
  o->g_inject = nullptr;
  o->overlap = 1;
  o->tensor_cores = 1;
  o->fp64_emulation = 1;
  o->sketch_prec = RANDUTV_SKETCH_OZAKI;
  o->g_capture = nullptr;
}

int randutv_set_stream(void* s) {
  g_stream = static_cast<cudaStream_t>(s);
  return RANDUTV_OK;
}

const char* randutv_strerror(int st) {
  if (st < 0) return "invalid argument (the code is minus its 1-based position)";
  switch (st) {
    case RANDUTV_OK: return "success";
    case RANDUTV_ENOMEM: return "device allocation failed";
    case RANDUTV_ENOCONV: return "small SVD did not converge within max_sweeps";
    case RANDUTV_ENAN: return "non-finite value in the input or the trailing block";
    case RANDUTV_EUNSUPPORTED: return "valid arguments outside what this library supports";
    case RANDUTV_ECUDA: return "a CUDA runtime call failed";
    case RANDUTV_ETIMEOUT: return "a device-side grid barrier gave up waiting";
    default: return "unknown status";
  }
}

const char* randutv_last_error(void) { return g_detail; }

void randutv_free(void* p) {
  if (p) cudaFree(p);
}

int randutv_factor_ex(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q, double tol,
                      double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv,
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
  if (ldt < m || (T == A && ldt != lda)) return -11;
  if (opts.form_uv && !V) return -12;
  if (opts.form_uv && ldv < n) return -13;
  if (!k_reached) return -14;
  if (opts.precision != RANDUTV_FP64 || opts.p < 0 || opts.max_sweeps < 1 ||
      opts.sketch_prec != RANDUTV_SKETCH_OZAKI)
    return -15;

  const int64_t mn = std::min(m, n);
  if (b > mn) b = static_cast<int>(mn);
  if (b > 256) { snprintf(g_detail, sizeof(g_detail), "block size above 256"); return RANDUTV_EUNSUPPORTED; }
  const int pov = opts.p;   // over-sampling
  if (b + pov > 256) {
    snprintf(g_detail, sizeof(g_detail), "block size plus over-sampling above 256");
    return RANDUTV_EUNSUPPORTED;
  }
  const bool uv = opts.form_uv != 0;
  cudaStream_t s = g_stream;
  Work w{};
  Lanes L;
  int st = RANDUTV_OK;
  double h_norm2 = 0.0, normA = 0.0;
  int64_t g_off = 0;
  *k_reached = mn;
  const int64_t nsteps = std::min((m + b - 1) / b, (n + b - 1) / b);

  {
    cudaError_t e = work_alloc(s, m, n, b, pov, uv, &w);
    if (e == cudaSuccess && opts.fp64_emulation && gemm_oz_supported()) {
      w.ozb = oz_budget(m, n, b + pov);
      const int64_t mx = std::max(m, n);
      w.ozbS = std::max(gemm_oz_work_bytes(b, mx, b), gemm_oz_work_bytes(mx, b, b));   // the rotations
      w.ozXb = gemm_oz_keep_bytes(mx, b + pov, mx, false);   // X^T (n_k x m_k) of the first step bounds all
      e = cudaMallocAsync(&w.ozT, w.ozb, s);
      if (e == cudaSuccess && uv) e = cudaMallocAsync(&w.ozU, w.ozb, s);
      if (e == cudaSuccess) e = cudaMallocAsync(&w.ozS, w.ozbS, s);
      if (e == cudaSuccess && q > 0) e = cudaMallocAsync(&w.ozX, w.ozXb, s);
      for (void* oz : {w.ozT, w.ozU, w.ozS})
        if (e == cudaSuccess && oz) e = cudaMemsetAsync(oz, 0, gemm_oz_head_bytes(), s);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      snprintf(g_detail, sizeof(g_detail), "workspace: %s", cudaGetErrorString(e));
      if (w.ozT) cudaFreeAsync(w.ozT, s);
      if (w.ozU) cudaFreeAsync(w.ozU, s);
      if (w.ozS) cudaFreeAsync(w.ozS, s);
      if (w.ozX) cudaFreeAsync(w.ozX, s);
      if (w.base) cudaFreeAsync(w.base, s);
      cudaStreamSynchronize(s);
      return e == cudaErrorMemoryAllocation ? RANDUTV_ENOMEM : RANDUTV_ECUDA;
    }
  }
  // Two lanes (Section 5.2's transforms applied as soon as formed, split by
  // what they touch): the T lane (high priority) carries the serial chain
  // sketch -> QR(Y) -> T right apply -> panel QR -> T left apply -> small
  // SVD -> T rotations; the U/V lane (low priority) applies each step's
  // reflectors and rotations to V and U as soon as the T lane has formed
  // them, filling the SMs that the latency-bound panel QR and Jacobi SVD
  // leave idle.  No step of the T lane reads U or V, so only the ring slots
  // order the lanes.  overlap = 0 puts both on the caller's stream.
  RUTV_CK(L.open(s, opts.overlap != 0));
  {
    cudaStream_t sT = L.t, sU = L.uv, sS = L.sv;
    const int64_t ge = w.gws_elems;
    int* oz_err = reinterpret_cast<int*>(slot(w, 3) + 2);
    const G64 gT{w.ozT != nullptr, w.ozT, w.ozb, oz_err, w.gws, ge};
    const G64 gU{w.ozU != nullptr, w.ozU, w.ozb, oz_err, w.gwsu, ge};
    const G64 gS{w.ozS != nullptr, w.ozS, w.ozbS, oz_err, w.gwss, ge};
    int prev_sl = -1;   // ring slot of the previous randomized step (its rotations of T run on the SVD lane)
    RUTV_CK(copy_matrix(sT, m, n, A, lda, T, ldt));
    if (uv) {
      RUTV_CK(set_identity(sU, m, U, ldu));
      RUTV_CK(set_identity(sU, n, V, ldv));
    }
    RUTV_CK(sumsq(sT, m, n, T, ldt, w.red, w.scal));
    RUTV_CK(cudaMemcpyAsync(&h_norm2, w.scal, sizeof(double), cudaMemcpyDeviceToHost, sT));
    RUTV_CK(cudaStreamSynchronize(sT));
    if (!std::isfinite(h_norm2)) { st = RANDUTV_ENAN; goto done; }
    normA = std::sqrt(h_norm2);

    for (int64_t i = 1; i <= nsteps; ++i) {
      const int64_t r0 = b * (i - 1);
      const int64_t r1 = std::min<int64_t>(r0 + b, m), c1 = std::min<int64_t>(r0 + b, n);
      const int64_t kr = m - r0, kc = n - r0;
      const int sl = static_cast<int>((i - 1) % Work::kR);
      double* X = T + r0 + r0 * ldt;
      if (tol > 0.0) {
        double t2 = 0.0;
        RUTV_CK(sumsq(sT, kr, kc, X, ldt, w.red, w.scal));
        RUTV_CK(cudaMemcpyAsync(&t2, w.scal, sizeof(double), cudaMemcpyDeviceToHost, sT));
        RUTV_CK(cudaStreamSynchronize(sT));
        if (!std::isfinite(t2)) { st = RANDUTV_ENAN; goto done; }
        if (std::sqrt(t2) <= tol * normA) { *k_reached = r0; break; }
      }
      // this step's ring slot is free once the U/V lane has finished step i - kR
      if (i > Work::kR) RUTV_CK(cudaStreamWaitEvent(sT, L.done[sl], 0));
      double *Vv = w.Vvr[sl], *Vu = w.Vur[sl], *Sv = w.Svr[sl], *Su = w.Sur[sl], *Us = w.Usr[sl], *Vs = w.Vsr[sl];
      if (r1 < m && c1 < n) {
        // ---- randomized step: sketch, QR(Y) -> VV, QR(panel) -> UU, small SVD
        // G has b + p columns (over-sampling); a step whose trailing block has
        // fewer than b + p columns uses the first kc of them
        const int wv = static_cast<int>(std::min<int64_t>(b + pov, kc));
        const double* G = w.G;
        if (opts.g_inject) {
          G = opts.g_inject + g_off;
        } else {
          RUTV_CK(launch_gaussian(sT, opts.seed, i, kr, b + pov, w.G, kr));
        }
        if (opts.g_capture)
          RUTV_CK(cudaMemcpyAsync(opts.g_capture + g_off, G, kr * (b + pov) * sizeof(double),
                                  cudaMemcpyDeviceToDevice, sT));
        g_off += kr * (b + pov);
        // X^T is sliced once for X^T G and every X^T Z of the step (X does not change in between)
        OzKeep kx{w.ozX, w.ozXb, false};
        RUTV_CK(gT.run(sT, true, false, kc, wv, kr, 1.0, X, ldt, G, kr, 0.0, w.Y, kc, &kx));
        for (int j = 0; j < q; ++j) {
          RUTV_CK(gT.run(sT, false, false, kr, wv, kc, 1.0, X, ldt, w.Y, kc, 0.0, w.Z, kr));
          RUTV_CK(gT.run(sT, true, false, kc, wv, kr, 1.0, X, ldt, w.Z, kr, 0.0, w.Y, kc, &kx));
        }
        double* Ysk = w.Y;   // the n_k x b matrix whose Householder QR gives VV
        if (pov > 0) {
          // Z = Q_Y Us(:, 1:b): Householder QR Y = Q_Y R_Y, SVD R_Y = Us Ds Vs^T
          // (its own Jacobi scratch and barrier slot: the SVD lane may be
          // running the previous step's), then Z = E - Vq (Sq (Vq^T E)) with
          // E = [Us(:, 1:b); 0]
          RUTV_CK(panel_qr(sT, kc, wv, w.Y, kc, w.tau, w.Vq, w.Rq, w.part, slot(w, 0)));
          RUTV_CK(gemm_f64(sT, true, false, wv, wv, kc, 1.0, w.Vq, kc, w.Vq, kc, 0.0, w.gram, wv, w.gws, ge));
          RUTV_CK(tfactor_from_gram(sT, wv, w.gram, w.tau, w.Sq));
          RUTV_CK(jacobi_svd(sT, wv, w.Rq, wv, w.Usq, w.dq, w.Vsq, opts.max_sweeps, w.jws2, slot(w, 4)));
          RUTV_CK(fill(sT, kc, b, w.Eb, kc, 0.0));
          RUTV_CK(copy_matrix(sT, wv, b, w.Usq, wv, w.Eb, kc));
          RUTV_CK(gemm_f64(sT, true, false, wv, b, wv, 1.0, w.Vq, kc, w.Usq, wv, 0.0, w.W1, wv, w.gws, ge));
          RUTV_CK(gemm_f64(sT, false, false, wv, b, wv, 1.0, w.Sq, wv, w.W1, wv, 0.0, w.W2, wv, w.gws, ge));
          RUTV_CK(gT.run(sT, false, false, kc, b, wv, -1.0, w.Vq, kc, w.W2, wv, 1.0, w.Eb, kc));
          Ysk = w.Eb;
        }
        RUTV_CK(panel_qr(sT, kc, b, Ysk, kc, w.tau, Vv, w.Rt, w.part, slot(w, 0)));
        RUTV_CK(gemm_f64(sT, true, false, b, b, kc, 1.0, Vv, kc, Vv, kc, 0.0, w.gram, b, w.gws, ge));
        RUTV_CK(tfactor_from_gram(sT, b, w.gram, w.tau, Sv));
        RUTV_CK(cudaEventRecord(L.v[sl], sT));
        // rows I2 of the previous step are rotated on the SVD lane: wait for it
        if (prev_sl >= 0) RUTV_CK(cudaStreamWaitEvent(sT, L.g[prev_sl], 0));
        RUTV_CK(wy_right(sT, m, kc, T + r0 * ldt, ldt, Vv, Sv, b, w.W1, w.W2, gT));
        if (uv) {
          RUTV_CK(cudaStreamWaitEvent(sU, L.v[sl], 0));
          RUTV_CK(wy_right(sU, n, kc, V + r0 * ldv, ldv, Vv, Sv, b, w.W1u, w.W2u, gU));
        }

        RUTV_CK(panel_qr(sT, kr, b, X, ldt, w.tau, Vu, w.R, w.part, slot(w, 1)));
        RUTV_CK(gemm_f64(sT, true, false, b, b, kr, 1.0, Vu, kr, Vu, kr, 0.0, w.gram, b, w.gws, ge));
        RUTV_CK(tfactor_from_gram(sT, b, w.gram, w.tau, Su));
        if (uv) {
          RUTV_CK(cudaEventRecord(L.u[sl], sT));
          RUTV_CK(cudaStreamWaitEvent(sU, L.u[sl], 0));
          RUTV_CK(wy_right(sU, m, kr, U + r0 * ldu, ldu, Vu, Su, b, w.W1u, w.W2u, gU));
        }
        RUTV_CK(wy_left_t(sT, kr, kc - b, T + r0 + c1 * ldt, ldt, Vu, Su, b, w.W1, w.W2, gT));
        RUTV_CK(fill(sT, kr, b, X, ldt, 0.0));
        RUTV_CK(cudaEventRecord(L.e[sl], sT));

        // small SVD and the rotations of T on the SVD lane (they touch rows
        // I2 and columns J2 only; the next step's sketch reads neither)
        RUTV_CK(cudaStreamWaitEvent(sS, L.e[sl], 0));
        RUTV_CK(jacobi_svd(sS, b, w.R, b, Us, w.d, Vs, opts.max_sweeps, w.jws, slot(w, 2)));
        set_diag_kernel<<<(b + 127) / 128, 128, 0, sS>>>(b, w.d, X, ldt);
        note_launch();
        RUTV_CK(cudaGetLastError());
        RUTV_CK(cudaEventRecord(L.s[sl], sS));
        if (uv) {
          RUTV_CK(cudaStreamWaitEvent(sU, L.s[sl], 0));
          RUTV_CK(rot_right(sU, m, b, U + r0 * ldu, ldu, Us, w.tmpu, gU));
          RUTV_CK(rot_right(sU, n, b, V + r0 * ldv, ldv, Vs, w.tmpu, gU));
        }
        RUTV_CK(rot_left_t(sS, b, kc - b, T + r0 + c1 * ldt, ldt, Us, w.tmps, gS));
        RUTV_CK(rot_right(sS, r0, b, T + r0 * ldt, ldt, Vs, w.tmps, gS));
        RUTV_CK(cudaEventRecord(L.g[sl], sS));
        prev_sl = sl;
      } else {
        // ---- last block: full SVD, economically through a QR when not square
        if (prev_sl >= 0) RUTV_CK(cudaStreamWaitEvent(sT, L.g[prev_sl], 0));
        int p;
        if (kr >= kc) {
          // QR first, also for a square block: one-sided Jacobi converges in a
          // few sweeps on the rows of a triangular R, far more slowly on a
          // general dense block of high condition number
          p = static_cast<int>(kc);
          RUTV_CK(panel_qr(sT, kr, p, X, ldt, w.tau, Vu, w.R, w.part, slot(w, 1)));
          RUTV_CK(gemm_f64(sT, true, false, p, p, kr, 1.0, Vu, kr, Vu, kr, 0.0, w.gram, p, w.gws, ge));
          RUTV_CK(tfactor_from_gram(sT, p, w.gram, w.tau, Su));
          if (uv) {
            RUTV_CK(cudaEventRecord(L.u[sl], sT));
            RUTV_CK(cudaStreamWaitEvent(sU, L.u[sl], 0));
            RUTV_CK(wy_right(sU, m, kr, U + r0 * ldu, ldu, Vu, Su, p, w.W1u, w.W2u, gU));
          }
        } else {
          p = static_cast<int>(kr);
          RUTV_CK(transpose(sT, kr, kc, X, ldt, w.W1, kc));
          RUTV_CK(panel_qr(sT, kc, p, w.W1, kc, w.tau, Vv, w.Rt, w.part, slot(w, 0)));
          RUTV_CK(gemm_f64(sT, true, false, p, p, kc, 1.0, Vv, kc, Vv, kc, 0.0, w.gram, p, w.gws, ge));
          RUTV_CK(tfactor_from_gram(sT, p, w.gram, w.tau, Sv));
          RUTV_CK(wy_right(sT, m, kc, T + r0 * ldt, ldt, Vv, Sv, p, w.W2, w.tmp, gT));
          if (uv) {
            RUTV_CK(cudaEventRecord(L.v[sl], sT));
            RUTV_CK(cudaStreamWaitEvent(sU, L.v[sl], 0));
            RUTV_CK(wy_right(sU, n, kc, V + r0 * ldv, ldv, Vv, Sv, p, w.W1u, w.W2u, gU));
          }
          RUTV_CK(transpose(sT, p, p, w.Rt, p, w.R, p));
        }
        RUTV_CK(jacobi_svd(sT, p, w.R, p, Us, w.d, Vs, opts.max_sweeps, w.jws, slot(w, 2)));
        RUTV_CK(fill(sT, kr, kc, X, ldt, 0.0));
        set_diag_kernel<<<(p + 127) / 128, 128, 0, sT>>>(p, w.d, X, ldt);
        note_launch();
        RUTV_CK(cudaGetLastError());
        if (uv) {
          RUTV_CK(cudaEventRecord(L.s[sl], sT));
          RUTV_CK(cudaStreamWaitEvent(sU, L.s[sl], 0));
          RUTV_CK(rot_right(sU, m, p, U + r0 * ldu, ldu, Us, w.tmpu, gU));
          RUTV_CK(rot_right(sU, n, p, V + r0 * ldv, ldv, Vs, w.tmpu, gU));
        }
        RUTV_CK(rot_right(sT, r0, p, T + r0 * ldt, ldt, Vs, w.tmp, gT));
      }
      if (uv) RUTV_CK(cudaEventRecord(L.done[sl], sU));
    }
  }
  RUTV_CK(L.join(s));
  RUTV_CK(cudaStreamSynchronize(s));
  st = device_status(w);
  if (prof_enabled()) prof_flush();

done:
  L.join(s);
  if (w.ozT) cudaFreeAsync(w.ozT, s);
  if (w.ozU) cudaFreeAsync(w.ozU, s);
  if (w.ozS) cudaFreeAsync(w.ozS, s);
  if (w.ozX) cudaFreeAsync(w.ozX, s);
  if (w.base) {
    cudaFreeAsync(w.base, s);
    cudaStreamSynchronize(s);
  }
  L.close();
  return st;
}

int randutv_factor(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q, double tol,
                   double** U, double** T, double** V, int64_t* k_reached) {
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (!A) return -3;
  if (lda < m) return -4;
  if (b < 1) return -5;
  if (q < 0) return -6;
  if (!(tol >= 0.0) || std::isinf(tol)) return -7;
  if (!U) return -8;
  if (!T) return -9;
  if (!V) return -10;
  if (!k_reached) return -11;
  *U = *T = *V = nullptr;
  double *u = nullptr, *t = nullptr, *v = nullptr;
  if (cudaMalloc(&u, m * m * sizeof(double)) != cudaSuccess || cudaMalloc(&t, m * n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&v, n * n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(u); cudaFree(t); cudaFree(v);
    return RANDUTV_ENOMEM;
  }
  int st = randutv_factor_ex(m, n, A, lda, b, q, tol, u, m, t, m, v, n, k_reached, nullptr);
  if (st != RANDUTV_OK && st != RANDUTV_ENOCONV) {
    cudaFree(u); cudaFree(t); cudaFree(v);
    return st;
  }
  *U = u; *T = t; *V = v;
  return st;
}

int randutv_factor_host(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q, double tol,
                        double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv,
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
  if (!T || T == A) return -10;
  if (ldt < m) return -11;
  if (opts.form_uv && !V) return -12;
  if (opts.form_uv && ldv < n) return -13;
  if (!k_reached) return -14;
  cudaStream_t s = g_stream;
  const bool uv = opts.form_uv != 0;
  double *dT = nullptr, *dU = nullptr, *dV = nullptr;
  int st = RANDUTV_OK;
  cudaError_t e = cudaMallocAsync(&dT, m * n * sizeof(double), s);
  if (e == cudaSuccess && uv) e = cudaMallocAsync(&dU, m * m * sizeof(double), s);
  if (e == cudaSuccess && uv) e = cudaMallocAsync(&dV, n * n * sizeof(double), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    st = (e == cudaErrorMemoryAllocation) ? RANDUTV_ENOMEM : cuda_status(e, "randutv_factor_host alloc");
    goto done;
  }
  RUTV_CK(cudaMemcpy2DAsync(dT, m * sizeof(double), A, lda * sizeof(double), m * sizeof(double), n,
                            cudaMemcpyHostToDevice, s));
  st = randutv_factor_ex(m, n, dT, m, b, q, tol, dU, m, dT, m, dV, n, k_reached, &opts);
  if (st != RANDUTV_OK && st != RANDUTV_ENOCONV) goto done;
  RUTV_CK(cudaMemcpy2DAsync(T, ldt * sizeof(double), dT, m * sizeof(double), m * sizeof(double), n,
                            cudaMemcpyDeviceToHost, s));
  if (uv) {
    RUTV_CK(cudaMemcpy2DAsync(U, ldu * sizeof(double), dU, m * sizeof(double), m * sizeof(double), m,
                              cudaMemcpyDeviceToHost, s));
    RUTV_CK(cudaMemcpy2DAsync(V, ldv * sizeof(double), dV, n * sizeof(double), n * sizeof(double), n,
                              cudaMemcpyDeviceToHost, s));
  }
  RUTV_CK(cudaStreamSynchronize(s));
done:
  if (dT) cudaFreeAsync(dT, s);
  if (dU) cudaFreeAsync(dU, s);
  if (dV) cudaFreeAsync(dV, s);
  cudaStreamSynchronize(s);
  return st;
}

// ------------------------------------------------------ building blocks
int randutv_gaussian(uint64_t seed, int64_t step, int64_t k, int64_t b, double* G, int64_t ldg) {
  if (step < 1) return -2;
  if (k < 0) return -3;
  if (b < 0) return -4;
  if (!G && k * b > 0) return -5;
  if (ldg < std::max<int64_t>(1, k)) return -6;
  cudaError_t e = launch_gaussian(g_stream, seed, step, k, b, G, ldg);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
  return e == cudaSuccess ? RANDUTV_OK : cuda_status(e, "randutv_gaussian");
}

int randutv_philox_words(uint64_t seed, int64_t step, int64_t k, int64_t b, uint32_t* W) {
  if (step < 1) return -2;
  if (k < 0) return -3;
  if (b < 0) return -4;
  if (!W && k * b > 0) return -5;
  cudaError_t e = launch_philox_words(g_stream, seed, step, k, b, W);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
  return e == cudaSuccess ? RANDUTV_OK : cuda_status(e, "randutv_philox_words");
}

int randutv_dgemm(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                  int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc) {
  const bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
  if (!ta && transa != 'N' && transa != 'n') return -1;
  if (!tb && transb != 'N' && transb != 'n') return -2;
  if (m < 0) return -3;
  if (n < 0) return -4;
  if (k < 0) return -5;
  if (lda < std::max<int64_t>(1, ta ? k : m)) return -8;
  if (ldb < std::max<int64_t>(1, tb ? n : k)) return -10;
  if (ldc < std::max<int64_t>(1, m)) return -13;
  cudaStream_t s = g_stream;
  const int64_t we = gemm_f64_work_elems(m, n, k);
  double* ws = nullptr;
  cudaError_t e = cudaSuccess;
  if (we > 0) e = cudaMallocAsync(&ws, we * sizeof(double), s);
  if (e == cudaSuccess) e = gemm_f64(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, we);
  if (ws) cudaFreeAsync(ws, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  return e == cudaSuccess ? RANDUTV_OK : cuda_status(e, "randutv_dgemm");
}

int randutv_panel_qr(int64_t k, int64_t w, double* P, int64_t ldp, double* tau, double* Vexp, double* S) {
  if (k < 1) return -1;
  if (w < 1 || w > k || w > 256) return -2;
  if (!P) return -3;
  if (ldp < k) return -4;
  if (!tau) return -5;
  if (!Vexp) return -6;
  if (!S) return -7;
  cudaStream_t s = g_stream;
  const int wi = static_cast<int>(w);
  const int64_t part = panel_qr_part_elems(k, wi), gw = gemm_budget(k, wi);
  const int64_t total = part + 2 * w * w + gw + 64;
  double* ws = nullptr;
  cudaError_t e = cudaMallocAsync(&ws, total * sizeof(double), s);
  if (e != cudaSuccess) { cudaGetLastError(); return RANDUTV_ENOMEM; }
  double* R = ws + part;
  double* gram = R + w * w;
  double* gws = gram + w * w;
  unsigned* flags = reinterpret_cast<unsigned*>(gws + gw);
  int st = RANDUTV_OK;
  unsigned herr[4] = {0, 0, 0, 0};
  RUTV_CK(cudaMemsetAsync(flags, 0, 4 * sizeof(unsigned), s));
  RUTV_CK(panel_qr(s, k, wi, P, ldp, tau, Vexp, R, ws, flags));
  RUTV_CK(gemm_f64(s, true, false, w, w, k, 1.0, Vexp, k, Vexp, k, 0.0, gram, w, gws, gw));
  RUTV_CK(tfactor_from_gram(s, wi, gram, tau, S));
  RUTV_CK(cudaMemcpyAsync(herr, flags, sizeof(herr), cudaMemcpyDeviceToHost, s));
  RUTV_CK(cudaStreamSynchronize(s));
  if (herr[2] & kDevErrTimeout) st = RANDUTV_ETIMEOUT;
done:
  cudaFreeAsync(ws, s);
  cudaStreamSynchronize(s);
  return st;
}

int randutv_small_svd(int64_t p, const double* M, int64_t ldm, double* Us, double* d, double* Vs,
                      int max_sweeps) {
  if (p < 1 || p > 256) return -1;
  if (!M) return -2;
  if (ldm < p) return -3;
  if (!Us) return -4;
  if (!d) return -5;
  if (!Vs) return -6;
  if (max_sweeps < 1) return -7;
  cudaStream_t s = g_stream;
  const int pi = static_cast<int>(p);
  const int64_t we = jacobi_work_elems(pi) + 8;
  double* ws = nullptr;
  cudaError_t e = cudaMallocAsync(&ws, we * sizeof(double), s);
  if (e != cudaSuccess) { cudaGetLastError(); return RANDUTV_ENOMEM; }
  unsigned* flags = reinterpret_cast<unsigned*>(ws + jacobi_work_elems(pi));
  int st = RANDUTV_OK;
  unsigned herr[4] = {0, 0, 0, 0};
  RUTV_CK(cudaMemsetAsync(flags, 0, 4 * sizeof(unsigned), s));
  RUTV_CK(jacobi_svd(s, pi, M, ldm, Us, d, Vs, max_sweeps, ws, flags));
  RUTV_CK(cudaMemcpyAsync(herr, flags, sizeof(herr), cudaMemcpyDeviceToHost, s));
  RUTV_CK(cudaStreamSynchronize(s));
  if (herr[2] & kDevErrTimeout) st = RANDUTV_ETIMEOUT;
  else if (herr[2] & kDevErrNoConv) st = RANDUTV_ENOCONV;
done:
  cudaFreeAsync(ws, s);
  cudaStreamSynchronize(s);
  return st;
}

}  // extern "C"

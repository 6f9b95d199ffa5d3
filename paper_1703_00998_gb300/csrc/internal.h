// Host-side interfaces between the engine and its kernels (not exported).
#pragma once
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

namespace rutv {

// One-time setup per device (kernel attributes such as the dynamic shared
// memory limit are per device): per_device_once(o, init) runs init() the
// first time it is called with a given current device and records success;
// thread-safe.  Devices 64 and above run init() on every call.
struct PerDeviceOnce {
  std::mutex mu;
  uint64_t done = 0;   // bit d: device d set up
};
template <class F>
cudaError_t per_device_once(PerDeviceOnce& o, F init) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return init();
  std::lock_guard<std::mutex> lk(o.mu);
  if ((o.done >> dev) & 1ull) return cudaSuccess;
  e = init();
  if (e == cudaSuccess) o.done |= 1ull << dev;
  return e;
}

// Process-wide stream used by every entry point.
cudaStream_t current_stream();
// Set the calling thread's detail message returned by randutv_last_error.
void set_last_error(const char* msg);

// Device scratch for the barrier and error words: {count, gen, err, pad} x slots.
struct DevFlags {
  unsigned* words = nullptr;  // 4 * kFlagSlots unsigned
};
constexpr int kFlagSlots = 8;

// ---- prof.cu ----
enum ProfClass { kProfGemm = 0, kProfPanel = 1, kProfTfactor = 2, kProfJacobi = 3, kProfGauss = 4,
                 kProfOther = 5, kProfGemm32 = 6, kProfGemmTc = 7, kProfGemmOz = 8, kProfGemmOz32 = 9,
                 kProfOzSlice = 10, kProfClasses = 11 };
struct ProfTotals { double ms = 0.0; int64_t launches = 0; double flops = 0.0; double bytes = 0.0; };
struct ProfToken { int idx; };
void note_launch(int n = 1);
unsigned long long launch_count();
bool prof_enabled();
ProfToken prof_begin(cudaStream_t s, int cls);
void prof_end(cudaStream_t s, ProfToken t, double flops, double bytes);
void prof_flush();

// ---- gemm_f64.cu ----
// C = alpha op(A) op(B) + beta C (column-major, FP64 DFMA).  `work` (device,
// `work_elems` doubles) holds split-K partial sums; may be null (no split).
cudaError_t gemm_f64(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k,
                     double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                     double beta, double* C, int64_t ldc, double* work, int64_t work_elems);
// Split-K workspace (doubles) that gemm_f64 may use for an m x n x k product.
int64_t gemm_f64_work_elems(int64_t m, int64_t n, int64_t k);

// ---- gemm_f32.cu ----
// FP32 GEMM of the mixed-precision form (split-K partials summed in FP64).
cudaError_t gemm_f32(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, float alpha,
                     const float* A, int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                     float* work, int64_t work_elems);
int64_t gemm_f32_work_elems(int64_t m, int64_t n, int64_t k);
// Sum split-K FP32 partials (m x n each) in FP64 into C = alpha sum + beta C.
cudaError_t gemm_f32_reduce(cudaStream_t s, int64_t m, int64_t n, int splits, float alpha, const float* part,
                            float beta, float* C, int64_t ldc);

// ---- gemm_tc.cu ----
// D (m x n) = alpha A^T B + beta D on the tensor cores (tcgen05, TF32 inputs,
// FP32 accumulation), A k x m (lda), B k x n (ldb), column-major FP32.  `work`
// holds split-K partials; `err` receives kDevErrTimeout if a wait ran out.
cudaError_t gemm_tc_tn(cudaStream_t s, int64_t m, int64_t n, int64_t k, float alpha, const float* A, int64_t lda,
                       const float* B, int64_t ldb, float beta, float* D, int64_t ldd, float* work, int64_t work_elems,
                       int* err, bool split);
// D (m x n) = alpha op(A) op(B) + beta D on the tensor cores for any of the
// four transpose combinations (K-major or MN-major tiles).
cudaError_t gemm_tc(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, float alpha, const float* A,
                    int64_t lda, const float* B, int64_t ldb, float beta, float* D, int64_t ldd, float* work,
                    int64_t work_elems, int* err, bool split);
// FP64 GEMM from BF16 tensor-core slice products (Ozaki scheme); work holds
// gemm_oz_work_bytes(m, n, k) bytes (slices, scales, chunk partials).
cudaError_t gemm_oz(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                    const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* D, int64_t ldd,
                    void* work, size_t work_bytes, int* err);
size_t gemm_oz_work_bytes(int64_t m, int64_t n, int64_t k);
// A caller-held region for op(A)'s slices (see gemm_oz_keep): products that
// share op(A) slice it once.  ready: the region holds op(A)'s slices.
struct OzKeep {
  void* base = nullptr;
  size_t bytes = 0;
  bool ready = false;
};
// gemm_oz with op(A)'s slices in keep (formed when !keep->ready, reused otherwise:
// the caller vouches that op(A) has not changed); gemm_oz_keep_bytes is the
// region's size for an m x n x k product (sketch: the gemm_oz_sketch form).
cudaError_t gemm_oz_keep(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                         const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* D,
                         int64_t ldd, void* work, size_t work_bytes, int* err, OzKeep* keep);
size_t gemm_oz_keep_bytes(int64_t m, int64_t n, int64_t k, bool sketch);
// D (m x n, FP64) = op(A) op(B) with op(A) FP32 data (split exactly into 4
// slices) and op(B) FP64 data split into 5 slices (35 bits): the sketch
// products of the mixed form, n <= 256 < m.  work: gemm_oz_sketch_work_bytes.
cudaError_t gemm_oz_sketch(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, const float* A,
                           int64_t lda, const double* B, int64_t ldb, double* D, int64_t ldd, void* work,
                           size_t work_bytes, int* err, OzKeep* keep = nullptr);
size_t gemm_oz_sketch_work_bytes(int64_t m, int64_t n, int64_t k);
// Leading bytes of a gemm_oz workspace that must be zero before its first
// use (the split-tile accumulators; every call leaves them zero again).
size_t gemm_oz_head_bytes();
// The FP32 form (4 slices, FP32-accurate): the mixed form's updates.
cudaError_t gemm_oz32(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, float alpha,
                      const float* A, int64_t lda, const float* B, int64_t ldb, float beta, float* D, int64_t ldd,
                      void* work, size_t work_bytes, int* err);
size_t gemm_oz32_work_bytes(int64_t m, int64_t n, int64_t k);
bool gemm_oz_supported();
// Whether gemm_tc can take these operands (TMA alignment rules, driver entry point).
bool gemm_tc_supported(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t m, int64_t n, int64_t k);

// ---- philox.cu ----
cudaError_t launch_gaussian(cudaStream_t s, uint64_t seed, int64_t step, int64_t k, int64_t b,
                            double* G, int64_t ldg);
cudaError_t launch_philox_words(cudaStream_t s, uint64_t seed, int64_t step, int64_t k, int64_t b,
                                uint32_t* W);

// ---- panel_qr.cu ----
// Householder QR of the k x w panel P in place; writes tau (w), Vexp (k x w,
// ld k, explicit unit-lower, zero columns where tau = 0) and R (w x w, ld w,
// upper).  `part` needs panel_qr_part_elems(k, w) doubles.  `bar` points at
// one barrier slot {count, gen, err}.
cudaError_t panel_qr(cudaStream_t s, int64_t k, int w, double* P, int64_t ldp, double* tau,
                     double* Vexp, double* R, double* part, unsigned* bar);
int64_t panel_qr_part_elems(int64_t k, int w);
// S (w x w, ld w) with H_1...H_w = I - Vexp S Vexp^T from the Gram matrix
// Vexp^T Vexp (w x w, ld w, the full symmetric matrix: its lower triangle is
// read) and tau: S = (striu(Gram) + diag(1/tau))^-1.
cudaError_t tfactor_from_gram(cudaStream_t s, int w, const double* gram, const double* tau,
                              double* S);

// ---- jacobi.cu ----
// Scratch of jacobi_svd for a p x p block: W, Q, two p x p temporaries and the
// split-K partials of the p x p products (4 p^2), plus slack.
constexpr int64_t jacobi_work_elems_for(int p) { return 8ll * p * p + 2ll * p + 64; }
// SVD of a p x p matrix M (ld ldm): Us, Vs (p x p, ld p), d (p).  `work`
// needs jacobi_work_elems(p) doubles; `bar` one barrier slot; returns after
// queueing (status through the error word of the slot).
cudaError_t jacobi_svd(cudaStream_t s, int p, const double* M, int64_t ldm, double* Us, double* d,
                       double* Vs, int max_sweeps, double* work, unsigned* bar);
int64_t jacobi_work_elems(int p);

// ---- util kernels (engine.cu) ----
cudaError_t set_identity(cudaStream_t s, int64_t n, double* X, int64_t ldx);
cudaError_t copy_matrix(cudaStream_t s, int64_t m, int64_t n, const double* A, int64_t lda,
                        double* B, int64_t ldb);

// Streams of one factorization, forked from and joined back into the
// caller's stream with events: the T chain (high priority), the U/V
// accumulation (low priority) and the small-SVD lane (high priority: the
// SVD of step i and its rotations of T overlap step i+1's sketch and QR of
// Y, which read only the trailing block).  With overlap off all three are
// the caller's stream.  The per-step events are indexed by ring slot:
// v, u, s (reflectors of Y, of the panel, small factors ready), e (the T
// chain finished step i's left application: R and the trailing block are
// final), g (the SVD lane finished step i's rotations of T), done (the U/V
// stream finished that step's ring slot).
struct Lanes {
  static constexpr int kSlots = 3;
  cudaStream_t t = nullptr, uv = nullptr, sv = nullptr;
  cudaEvent_t v[kSlots] = {}, u[kSlots] = {}, s[kSlots] = {}, e[kSlots] = {}, g[kSlots] = {}, done[kSlots] = {};
  cudaEvent_t fork_ev = nullptr, join_t = nullptr, join_u = nullptr, join_v = nullptr;
  bool own = false;

  cudaError_t open(cudaStream_t caller, bool overlap) {
    cudaError_t err = cudaSuccess;
    cudaEvent_t* sets[] = {v, u, s, e, g, done};
    for (cudaEvent_t* set : sets)
      for (int i = 0; i < kSlots && err == cudaSuccess; ++i) err = cudaEventCreateWithFlags(&set[i], cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&join_t, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&join_u, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&join_v, cudaEventDisableTiming);
    if (err != cudaSuccess) return err;
    if (!overlap) {
      t = uv = sv = caller;
      return cudaSuccess;
    }
    int lo = 0, hi = 0;
    err = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (err == cudaSuccess) err = cudaStreamCreateWithPriority(&t, cudaStreamNonBlocking, hi);
    if (err == cudaSuccess) err = cudaStreamCreateWithPriority(&uv, cudaStreamNonBlocking, lo);
    if (err == cudaSuccess) err = cudaStreamCreateWithPriority(&sv, cudaStreamNonBlocking, hi);
    if (err != cudaSuccess) return err;
    own = true;
    err = cudaEventRecord(fork_ev, caller);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(t, fork_ev, 0);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(uv, fork_ev, 0);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(sv, fork_ev, 0);
    return err;
  }
  // Make the caller's stream wait for everything queued on the lanes.
  cudaError_t join(cudaStream_t caller) {
    if (!own) return cudaSuccess;
    cudaError_t err = cudaEventRecord(join_t, t);
    if (err == cudaSuccess) err = cudaEventRecord(join_u, uv);
    if (err == cudaSuccess) err = cudaEventRecord(join_v, sv);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(caller, join_t, 0);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(caller, join_u, 0);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(caller, join_v, 0);
    return err;
  }
  void close() {
    if (own) {
      cudaStreamDestroy(t);
      cudaStreamDestroy(uv);
      cudaStreamDestroy(sv);
      own = false;
    }
    cudaEvent_t* sets[] = {v, u, s, e, g, done};
    for (cudaEvent_t* set : sets)
      for (int i = 0; i < kSlots; ++i)
        if (set[i]) cudaEventDestroy(set[i]);
    if (fork_ev) cudaEventDestroy(fork_ev);
    if (join_t) cudaEventDestroy(join_t);
    if (join_u) cudaEventDestroy(join_u);
    if (join_v) cudaEventDestroy(join_v);
  }
};

}  // namespace rutv

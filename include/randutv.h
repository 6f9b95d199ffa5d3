/*
 * randutv.h -- C ABI of the GB300 (sm_103a) randUTV engine.
 *
 * randUTV (Martinsson, Quintana-Orti, Heavner, arXiv 1703.00998) factors an
 * m x n matrix A = U T V^T with U (m x m) and V (n x n) orthogonal and T
 * upper triangular (Section 1, eq. defUTVpre), working on b columns per step
 * (Fig. 4, Section 5.2).  Each step draws a Gaussian G, forms the sample
 * Y = (X^T X)^q X^T G of the active block X (Section 4.3), applies the
 * Householder reflector product of QR(Y) from the right, the one of the new
 * b-column panel from the left (Remark 1), and diagonalizes the b x b block
 * with a small SVD rotated into U, T and V (Fig. 4).
 *
 * Conventions for every entry point below:
 *   - matrices are column-major: element (i, j) of X is X[i + j * ldx];
 *   - pointers are DEVICE pointers unless a comment says otherwise, and
 *     the caller keeps ownership of every buffer it passes in;
 *   - work is queued on the stream set by randutv_set_stream (default: the
 *     legacy default stream) and calls return after the result is complete
 *     (they synchronize that stream before returning);
 *   - the return value is a status: 0 success, -i when argument i (1-based)
 *     is invalid (LAPACK info convention, nothing is computed), or one of
 *     the positive RANDUTV_E* codes.  No call aborts the process and no
 *     kernel traps; device-side failures (a bounded wait that ran out, a
 *     non-finite value) are reported through the status.
 */
#ifndef RANDUTV_H
#define RANDUTV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RANDUTV_OK            0
#define RANDUTV_ENOMEM        1  /* device allocation failed                    */
#define RANDUTV_ENOCONV       2  /* small SVD hit max_sweeps (outputs written)  */
#define RANDUTV_ENAN          3  /* non-finite input or trailing norm           */
#define RANDUTV_EUNSUPPORTED  4  /* valid but not supported by this library     */
#define RANDUTV_ECUDA         5  /* a CUDA runtime call failed                  */
#define RANDUTV_ETIMEOUT      6  /* a device grid barrier gave up waiting       */

#define RANDUTV_FP64   0  /* every step in FP64                                */

/* Options of randutv_factor_ex.  Fill with randutv_opts_default first. */
typedef struct randutv_opts {
  int precision;        /* RANDUTV_FP64 (randutv_factor_mixed ignores it)      */
  int form_uv;          /* 1: form U and V (Table 1); 0: T only (Table 4),
                           U and V may then be NULL                            */
  int max_sweeps;       /* cap on cyclic Jacobi sweeps of each small SVD (30)  */
  int p;                /* over-sampling (Remark "Oversampling"): each step
                           sketches b + p columns and takes the b dominant left
                           singular vectors of the sketch (a Householder QR and
                           an SVD of its R); FP64 form: p >= 0 with b + p <=
                           256; the mixed form requires 0.  With g_inject,
                           step i stores (m - b(i-1)) x (b + p) values.       */
  uint64_t seed;        /* Philox4x32-10 key of the Gaussian matrices G        */
  const double* g_inject; /* NULL, or a device buffer holding every randomized
                           step's G, concatenated: step i (1-based, b*i <
                           min(m,n)) stores its (m - b(i-1)) x (b + p) matrix
                           column-major (ld = m - b(i-1)) right after step
                           i-1's.  Used instead of the Philox stream.          */
  int overlap;          /* 1: accumulate U and V on a second, lower-priority
                           stream, overlapped with the serial panel QR and
                           small SVD of the T chain (same results); 0: one
                           stream                                              */
  int tensor_cores;     /* mixed form only: 1 = the sketch products X^T G,
                           X Y and X^T Z on the tcgen05 tensor cores (3xTF32,
                           FP32 accumulation) when the operands meet the TMA
                           alignment rules; 0 = FP32 CUDA cores.  The
                           block-reflector and rotation products always run
                           on the FP32 CUDA cores (round to nearest).        */
  int fp64_emulation;   /* FP64 form only: 1 = the sketch products, block-
                           reflector applications and rotations through the
                           Ozaki-scheme GEMM (randutv_dgemm_oz: BF16 tensor-
                           core slice products, FP64-accurate); 0 = FP64
                           DFMA GEMM.  The Gram matrices of the compact-WY
                           factors and products too small for its tiles
                           always use DFMA.  Needs about 17 n^2 bytes of
                           scratch for each of the T and U/V lanes
                           (n = max(m, n)), and 17 n^2 more when q > 0 for
                           the slices of a step's X^T, which its products
                           X^T G and X^T Z share.                           */
  int sketch_prec;      /* mixed form: how the sketch products (Section 4.3,
                           step 2) are formed; they decide which subspace a
                           step captures, not the backward error, but on
                           slowly decaying spectra FP32-level rounding of the
                           sketch moves |diag T| far more than the FP32
                           backward error does.  RANDUTV_SKETCH_OZAKI
                           (default): tensor-core products of the FP32 trailing
                           block, split exactly into 4 BF16 slices, with the
                           FP64 G / Y / Z split into 5 (35 bits), FP64 results;
                           RANDUTV_SKETCH_3XTF32: hi/lo TF32 split, three
                           products, FP32 accumulation; RANDUTV_SKETCH_TF32:
                           one TF32 product (both with tensor_cores = 1; FP32
                           CUDA cores otherwise).  The FP64 form requires
                           RANDUTV_SKETCH_OZAKI (its sketch is FP64).         */
  double* g_capture;    /* NULL, or a device buffer receiving every randomized
                           step's G (FP64) in the g_inject layout: a run with
                           the Philox stream records the matrices it used, so
                           the same G can be given to another implementation
                           (or back through g_inject).  Size: the sum over
                           randomized steps i of (m - b(i-1)) (b + p).       */
} randutv_opts;

#define RANDUTV_SKETCH_OZAKI  0
#define RANDUTV_SKETCH_3XTF32 1
#define RANDUTV_SKETCH_TF32   2

/* Defaults: FP64, form_uv = 1, max_sweeps = 30, p = 0, seed = 998, no g_inject,
   overlap = 1, tensor_cores = 1, fp64_emulation = 1, sketch_prec =
   RANDUTV_SKETCH_OZAKI, no g_capture. */
void randutv_opts_default(randutv_opts* opts);

/* Stream used by all later calls in this process (a cudaStream_t; NULL =
   legacy default stream).  Always returns RANDUTV_OK. */
int randutv_set_stream(void* cuda_stream);

/* Factor A (m x n, lda >= m, FP64) as A = U T V^T (Fig. 4).  The library
 * allocates T (m x n, ld m), U (m x m, ld m) and V (n x n, ld n) and returns
 * them through *T, *U, *V; release each with randutv_free.  A is not
 * modified.  b >= 1 is the block size (values above min(m,n) give one full
 * SVD), q >= 0 the number of power steps, tol >= 0 the early-stop tolerance:
 * before step i the factorization stops when ||T(I2 u I3, J2 u J3)||_F <=
 * tol * ||A||_F, and *k_reached receives b(i-1) (min(m,n) when it runs to the
 * end; tol = 0 never stops early).  Gaussians from the Philox stream with seed
 * 998.  Argument order for the -i codes: m=1 n=2 A=3 lda=4 b=5 q=6 tol=7 U=8
 * T=9 V=10 k_reached=11. */
int randutv_factor(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q,
                   double tol, double** U, double** T, double** V, int64_t* k_reached);

/* Same with caller-owned outputs: T (ldt >= m), U (ldu >= m), V (ldv >= n).
 * T may equal A (in place, Section 5.2: T overwrites A) when ldt == lda.
 * opts may be NULL (defaults).  Argument order: m=1 n=2 A=3 lda=4 b=5 q=6
 * tol=7 U=8 ldu=9 T=10 ldt=11 V=12 ldv=13 k_reached=14 opts=15. */
int randutv_factor_ex(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q,
                      double tol, double* U, int64_t ldu, double* T, int64_t ldt,
                      double* V, int64_t ldv, int64_t* k_reached, const randutv_opts* opts);

/* Mixed-precision form of randutv_factor_ex (same method and arguments, FP32
 * data): A, T, U, V are FP32 device matrices; the sketch, the
 * block-reflector applications and the small rotations run as FP32 products
 * with FP32 accumulation (split reductions summed in FP64), while every panel
 * is up-cast to FP64 for its Householder QR and compact-WY factor and the
 * b x b SVD is computed in FP64.  opts->g_inject, if given, is the FP64
 * Gaussian stream of randutv_factor_ex (rounded to FP32).  T may equal A
 * when ldt == lda.  Same numbering of invalid arguments. */
int randutv_factor_mixed(int64_t m, int64_t n, const float* A, int64_t lda, int b, int q,
                         double tol, float* U, int64_t ldu, float* T, int64_t ldt,
                         float* V, int64_t ldv, int64_t* k_reached, const randutv_opts* opts);

/* randutv_factor_ex on HOST buffers: A (lda >= m), U (ldu >= m), T (ldt >= m)
 * and V (ldv >= n) are host pointers (page-locked memory gives the fastest
 * copies; A and T must not overlap).  The library allocates device memory,
 * copies A in, factors in place on the device, copies T (and U, V when
 * form_uv) back, and frees the device memory before returning.  Same
 * argument numbering and status codes as randutv_factor_ex. */
int randutv_factor_host(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q,
                        double tol, double* U, int64_t ldu, double* T, int64_t ldt,
                        double* V, int64_t ldv, int64_t* k_reached, const randutv_opts* opts);

/* Release a buffer returned by randutv_factor (NULL is ignored). */
void randutv_free(void* p);

/* Static description of a status code. */
const char* randutv_strerror(int status);

/* Detail of the last RANDUTV_ECUDA / RANDUTV_ETIMEOUT / RANDUTV_EUNSUPPORTED
 * status raised in the calling thread (empty string if none). */
const char* randutv_last_error(void);

/* ---- Diagnostics ---- */

/* Kernel classes of randutv_profile_read. */
#define RANDUTV_PROF_GEMM     0  /* FP64 GEMM (sketch, block-reflector applications, rotations) */
#define RANDUTV_PROF_PANEL    1  /* Householder panel QR                              */
#define RANDUTV_PROF_TFACTOR  2  /* compact-WY factor S                               */
#define RANDUTV_PROF_JACOBI   3  /* small SVD (sweeps + ordering)                     */
#define RANDUTV_PROF_GAUSS    4  /* Philox Gaussian                                   */
#define RANDUTV_PROF_OTHER    5  /* copies, fills, norms                              */
#define RANDUTV_PROF_GEMM32   6  /* FP32 GEMM of the mixed-precision form             */
#define RANDUTV_PROF_GEMMTC   7  /* tensor-core (tcgen05, TF32) GEMM of the sketch    */
#define RANDUTV_PROF_GEMMOZ   8  /* Ozaki-scheme product kernel (tcgen05, BF16 slices) */
#define RANDUTV_PROF_GEMMOZ32 9  /* the FP32 Ozaki form (randutv_sgemm_oz)            */
#define RANDUTV_PROF_OZSLICE 10  /* slicing of the Ozaki products' operands           */

/* Turn per-kernel-class timing on (1) or off (0).  While on, each launch of a
 * class is bracketed by CUDA events on its stream and its algorithmic flops
 * and bytes are recorded; nothing synchronises the host until a read. */
int randutv_profile_enable(int on);
/* Zero the accumulated totals. */
int randutv_profile_reset(void);
/* Totals of class cls since the last reset: summed event time (ms), number
 * of timed launches, algorithmic flops and bytes.  Synchronises pending
 * events.  Any output pointer may be NULL.  Returns -1 for an unknown cls. */
int randutv_profile_read(int cls, double* ms, int64_t* launches, double* flops, double* bytes);
/* Number of kernels this library has launched since it was loaded. */
uint64_t randutv_launch_count(void);
/* Self-test of the bounded device waits (no counterpart in the paper): one
 * tiny launch on the legacy default stream whose wait nothing will end, an
 * mbarrier no thread arrives at (kind 0) or a grid barrier sized for two
 * CTAs in a launch of one (kind 1), with a limit of `seconds` (0 < seconds
 * <= 2; the library's own waits use 2 s).  The kernel records the timeout
 * and returns, so the call returns RANDUTV_ETIMEOUT (the expected result)
 * after about `seconds`, and the CUDA context stays usable.  Returns -1 or
 * -2 for an invalid kind or limit (before any CUDA call), RANDUTV_ECUDA if
 * a CUDA call failed, RANDUTV_OK if the wait was not cut short (a fault of
 * the self-test).  Calls that overlap on a device share its error word. */
int randutv_selftest_wait(int kind, double seconds);
/* Sweeps of the small-SVD Jacobi kernels on the current device since the
 * last reset: FP32 sweeps, FP64 sweeps, and the number of small SVDs (FP64
 * sweep launches).  reset != 0 clears the counters after reading.  Waits for
 * the device's pending work (a synchronous copy).  Any output pointer may be
 * NULL.  Returns RANDUTV_ECUDA if the counters cannot be read. */
int randutv_jacobi_sweeps(int64_t* fp32_sweeps, int64_t* fp64_sweeps, int64_t* svds, int reset);

/* ---- Building blocks of one step, exposed so each kernel can be tested on
 * its own against the CPU oracle.  Same conventions as above. ---- */

/* G (k x b, ld ldg >= k): the Gaussian matrix of global step `step` (1-based)
 * from Philox4x32-10 with key (seed mod 2^32, seed div 2^32) and counter
 * (r div 2, c, step, 0) for row r, column c; Box-Muller of two open-interval
 * uniforms u = (floor(w / 2^12) + 1/2) 2^-52 from words (x0, x1) and (x2, x3):
 * row 2p gets sqrt(-2 ln u1) cos(2 pi u2), row 2p+1 the sine (randn of Fig. 4). */
int randutv_gaussian(uint64_t seed, int64_t step, int64_t k, int64_t b, double* G, int64_t ldg);

/* Raw Philox4x32-10 words of the same counters: W holds ceil(k/2) x b x 4
 * uint32 values, word t of counter (p, c) at W[4 * (p + c * ceil(k/2)) + t]. */
int randutv_philox_words(uint64_t seed, int64_t step, int64_t k, int64_t b, uint32_t* W);

/* C = alpha op(A) op(B) + beta C with op(X) = X ('N') or X^T ('T'); op(A) is
 * m x k, op(B) k x n, C m x n.  beta = 0 never reads C.  The FP64 GEMM every
 * block-reflector application and sketch product of the step runs on. */
int randutv_dgemm(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                  double* C, int64_t ldc);

/* FP32 counterpart of randutv_dgemm (the products of the mixed-precision
 * form): FP32 operands and accumulation, split-K partial sums added in FP64. */
int randutv_sgemm(char transa, char transb, int64_t m, int64_t n, int64_t k, float alpha,
                  const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
                  float* C, int64_t ldc);

/* C = alpha op(A) op(B) + beta C on the tcgen05 tensor cores, FP32
 * column-major operands, FP32 accumulation in tensor memory.  transa 'T':
 * op(A) = A^T with A k x m; 'N': op(A) = A with A m x k.  transb 'N':
 * op(B) = B with B k x n; 'T': op(B) = B^T with B n x k.  C is m x n (ldc).
 * The products of Section 4.3 (sketch) and of the block-reflector
 * applications (eq. WYrepresentation) all take one of these four forms.
 * passes = 1: inputs used as TF32 (10-bit mantissa); passes = 3: each input
 * split into two TF32 parts and three products accumulated (3xTF32,
 * FP32-level products; the accumulator itself does not round to nearest,
 * so the error grows with k).  Requires 16-byte aligned A, B and lda, ldb
 * multiples of 4 (TMA); otherwise RANDUTV_EUNSUPPORTED.  Negative return:
 * the position of the first invalid argument.  Allocates its split-K
 * scratch with cudaMallocAsync on the bound stream and synchronises it. */
int randutv_sgemm_tc(char transa, char transb, int64_t m, int64_t n, int64_t k, float alpha,
                     const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
                     float* C, int64_t ldc, int passes);

/* C = alpha op(A) op(B) + beta C in FP64 (column-major; transa, transb as in
 * randutv_dgemm) from BF16 tensor-core products: the Ozaki scheme, an
 * implementation choice for the products of Fig. 4 with no counterpart in
 * the paper.  Each row of op(A) and column of op(B) is split per K chunk of
 * 128 into a power-of-two scale and 8 slices of 7 bits (56 bits), the 36
 * slice-pair products with slice indices s + t <= 7 are summed exactly in
 * FP32 on the tensor cores and combined exactly in 64-bit integers; the
 * chunks accumulate in a 64-bit fixed-point sum whose unit is set by bounds
 * of the row and column 2-norms (it cannot overflow; the unit is below
 * 2^-60 ||row|| ||column||), two roundings to that unit per chunk, and the
 * result is rounded once to FP64.  Error <= 2 * 128 * 2^-55 * max|op(A)
 * row| * max|op(B) column| per chunk plus one unit per chunk plus the final
 * rounding: the accuracy class of an FP64 GEMM.  k = 0 gives C = beta C.
 * Allocates its scratch (about 16 (m + n) k bytes of slices and 20 MB of
 * split-tile accumulators) with cudaMallocAsync on the bound stream and
 * synchronises it.  Negative return: the position of the first invalid
 * argument. */
int randutv_dgemm_oz(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                     const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                     double* C, int64_t ldc);

/* FP32 counterpart of randutv_dgemm_oz (the mixed form's block-reflector
 * applications and rotations): FP32 operands and result, 4 slices of 7 bits
 * (28 bits) per row / column and K chunk of 128, the 10 slice pairs with
 * s + t <= 3 summed exactly on the tensor cores, one rounding to FP32 per
 * chunk, chunks summed in FP64.  Error per chunk <= 128 * 2^-27 * max|a| *
 * max|b| over the chunk plus FP32 rounding: the accuracy class of an FP32
 * GEMM with round-to-nearest accumulation on operands of even magnitude
 * (the fixed point is relative to each row's chunk maximum).  A building
 * block, not used by the factorization: there it was slower than the FP32
 * CUDA-core GEMM and, on graded operands, less accurate.  Scratch: about
 * 8 (m + n) k bytes plus 4 m n per chunk when k > 128 (cudaMallocAsync,
 * synchronised). */
int randutv_sgemm_oz(char transa, char transb, int64_t m, int64_t n, int64_t k, float alpha,
                     const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
                     float* C, int64_t ldc);

/* Unpivoted Householder QR of the k x w panel P (k >= w >= 1, ldp >= k), in
 * place (eq. unpivQR; LAPACK dlarfg convention: beta = -sign(alpha)||x||,
 * tau = 0 when the part below the diagonal is zero).  On return P holds R on
 * and above the diagonal and the Householder vectors below it; tau (w) the
 * scalars; Vexp (k x w, ld k) the explicit unit-lower vectors (column j zero
 * when tau_j = 0); S (w x w, ld w) the upper triangular factor with
 * H_1 ... H_w = I - Vexp S Vexp^T (eq. WYrepresentation with W = -Vexp S). */
int randutv_panel_qr(int64_t k, int64_t w, double* P, int64_t ldp, double* tau,
                     double* Vexp, double* S);

/* SVD of a p x p block M (1 <= p <= 256, ldm >= p): M = Us diag(d) Vs^T by one-sided cyclic
 * Jacobi in FP64 on the rows of M (fastest for a triangular M such as the R
 * factor of a QR, which is what the factorization passes); d descending and >= 0, the largest-|.| entry of each Vs
 * column positive (lowest index on ties).  Us, Vs are p x p with ld p.
 * Returns RANDUTV_ENOCONV (outputs still written) after max_sweeps sweeps. */
int randutv_small_svd(int64_t p, const double* M, int64_t ldm, double* Us, double* d,
                      double* Vs, int max_sweeps);

/* randutv_small_svd without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that may not allocate
 * device memory themselves or through the library (for example code whose
 * host framework owns all device memory through its own allocator, code on
 * a latency-critical path where an allocation could synchronise or fail,
 * or a plugin that is not allowed to call the CUDA allocator).  Its scratch
 * is one array in device global memory declared by the library (about 4 MB,
 * held on every GPU that loads the library until the process exits), so p is
 * limited to 256; larger p returns RANDUTV_EUNSUPPORTED with a message in
 * randutv_last_error.  The caller passes M, Us, d and Vs exactly as for
 * randutv_small_svd and gets the same results.  All calls on a device share
 * the array and it keeps the last call's contents: calls whose work overlaps
 * on the GPU (other streams or host threads) race on it and must be
 * serialised.  The first call on each device looks up the array's device
 * address (with that device current); make it before any stream capture. */
int randutv_small_svd_noalloc(int64_t p, const double* M, int64_t ldm, double* Us, double* d,
                              double* Vs, int max_sweeps);

/* ---- Batched form: many small FP32 matrices in one launch ----------------
 *
 * Fig. 4 (with the economic final steps of Section 5.2 for m > n and of the
 * Remark on m < n) applied independently to each matrix of a batch, with the
 * early stop of Section 1.1 (ii): before each step, a matrix whose trailing
 * block has ||T(I2 I3, J2 J3)||_F <= tol ||A||_F stops there (k_reached = the
 * number of finished columns; T's trailing block is left as is and
 * A = U T V^T still holds).  Every matrix is m x n with 1 <= m, n <= 512,
 * FP32 in and out, one CTA per matrix at a time in a single persistent
 * kernel that takes matrices from a device queue, largest first.
 *
 * Packed layout (element offsets, see randutv_batched_layout): matrix i is
 * column-major with ld m[i] at offset sum_{j<i} m[j] n[j] of A and T, U_i
 * (m[i] x m[i]) at sum_{j<i} m[j]^2 of U, V_i (n[i] x n[i]) at
 * sum_{j<i} n[j]^2 of V; with g_inject, matrix i's Gaussian stream starts at
 * off_g[i] and holds step s's (m - b(s-1)) x b matrix column-major for every
 * step with b s < min(m, n), in step order.  Drawn in the kernel, G uses
 * Philox4x32-10 with key (seed mod 2^32, seed div 2^32) and counter
 * (row div 2, column, step, i), and FP32 Box-Muller on u1, u2 taken from
 * the top 23 bits of words x1, x3 as (floor(x / 2^9) + 1/2) 2^-23. */
typedef struct randutv_batched_plan randutv_batched_plan;

typedef struct randutv_batched_opts {
  int form_uv;          /* 1: form U and V; 0: T only (U, V may be NULL)       */
  int max_sweeps;       /* Jacobi sweep cap of each small SVD (30)             */
  uint64_t seed;        /* Philox key of the Gaussian matrices                 */
  const float* g_inject;/* NULL, or the device Gaussian streams (layout above) */
  int graph;            /* 1: launch through a CUDA graph the plan captures on
                           first use (re-captured when an argument changes)    */
  int async;            /* 1: return after queueing (no status from the device)*/
} randutv_batched_opts;

void randutv_batched_opts_default(randutv_batched_opts* opts);

/* Plan a batch: count matrices of sizes m[i] x n[i] (HOST arrays).  b is the
 * block size of every matrix (1..32, capped at min(m, n)), or 0 for the
 * per-size-class choice (classes by min(m, n): 1-64, 65-128, ..., 449-512),
 * 32 until randutv_batched_autotune or randutv_batched_set_classes sets it.
 * Allocates the device work table; EUNSUPPORTED when a size exceeds 512.
 * The plan serves one launch at a time. */
int randutv_batched_plan_create(int64_t count, const int32_t* m, const int32_t* n, int b,
                                randutv_batched_plan** plan);
int randutv_batched_plan_destroy(randutv_batched_plan* plan);

/* Host arrays of count entries (any may be NULL): element offsets of each
 * matrix in A/T, U, V and the Gaussian streams, its block size; totals[4]
 * receives the total element counts {A, U, V, G}. */
int randutv_batched_layout(const randutv_batched_plan* plan, int64_t* off_a, int64_t* off_u,
                           int64_t* off_v, int64_t* off_g, int32_t* b, int64_t* totals);

/* Factor every matrix of the plan: A (device, packed, read only) -> T
 * (device, packed; T == A factors in place), U, V (device, packed, written
 * in full), k_reached (device int32, count), info (device int32, count, may
 * be NULL: 0, RANDUTV_ENOCONV when a small SVD hit max_sweeps, RANDUTV_ENAN
 * for a non-finite A, which is then left with k_reached = 0).  q >= 0 power
 * steps, tol >= 0 (0: never stop early).  Returns RANDUTV_ENOCONV /
 * RANDUTV_ENAN when any matrix reported it (unless opts->async). */
int randutv_factor_batched(randutv_batched_plan* plan, const float* A, float* T, float* U, float* V,
                           int q, double tol, int32_t* k_reached, int32_t* info,
                           const randutv_batched_opts* opts);

/* Choose b in {16, 32} per size class by running the whole batch A (device,
 * packed) once with each (into scratch; A is not modified) and comparing
 * the per-matrix device times summed over each class; the plan keeps the
 * choice.  choice (HOST, 8 entries, may be NULL) receives it.  The plan must
 * have been created with b = 0 for the choice to take effect. */
int randutv_batched_autotune(randutv_batched_plan* plan, const float* A, int q, double tol,
                             const randutv_batched_opts* opts, int32_t* choice);

/* The layout a plan with these arguments would hold, computed on the host
 * alone (no device, no plan): count, m, n, b as for
 * randutv_batched_plan_create, b_per_class (8 entries, or NULL for 32
 * everywhere) as for randutv_batched_set_classes; every output (HOST,
 * count entries; totals 4) may be NULL.  order receives the queue order
 * (largest m n min(m, n) first, ties by index). */
int randutv_batched_layout_host(int64_t count, const int32_t* m, const int32_t* n, int b,
                                const int32_t* b_per_class, int64_t* off_a, int64_t* off_u,
                                int64_t* off_v, int64_t* off_g, int32_t* b_out, int32_t* order,
                                int64_t* totals);

/* Set the per-class block sizes (HOST, 8 entries in 1..32) directly. */
int randutv_batched_set_classes(randutv_batched_plan* plan, const int32_t* b_per_class);

/* The k x w Gaussian matrix the batched kernel draws for matrix `index` at
 * step `step` (FP32, column-major, ld ldg): the generator's own output, for
 * checking it against its definition. */
int randutv_batched_gaussian(uint64_t seed, int64_t index, int64_t step, int64_t k, int64_t w,
                             float* G, int64_t ldg);

/* ---- Rank-k approximation and its adjoint (FP64) ---------------------------
 *
 * A_k = U(:, 1:k) T(1:k, :) V^T (eq. Ak_randUTV) for k a multiple of b with
 * k < min(m, n): the first k/b randomized steps of Fig. 4 fix U(:, 1:k) and
 * A_k = U(:, 1:k) U(:, 1:k)^T A.  The Gaussian matrices are those of
 * randutv_factor_ex with the same seed (or opts->g_inject, its first k/b
 * steps), so A_k is a smooth function of A at fixed G.
 *
 * randutv_rank_k writes A_k (m x n, ld ldf, device) and, when state is
 * non-NULL, keeps on the device what the reverse pass needs: A, the final
 * T and U, each step's Gaussian, sketches, reflectors and WY factors (about
 * (q + 4) max(m, n) b doubles per step) and a copy of the injected
 * Gaussians; the reverse pass walks T and U back step by step with the
 * kept reflectors (no per-step copies of T or U);
 * randutv_rank_k_vjp then writes Abar = (dA_k/dA)^T Fbar (m x n, ld ldab)
 * for any number of cotangents Fbar (m x n, ld ldfb); randutv_rank_k_free
 * releases the state.  A state serves one call at a time (its scratch is
 * reused by every randutv_rank_k_vjp).  b <= 32 (EUNSUPPORTED above; also
 * when k >= min(m, n)); opts->p must be 0.  The large products of both
 * passes use the Ozaki-scheme GEMM when opts->fp64_emulation is set (the
 * default; its workspace is part of the state), else FP64 DFMA. */
typedef struct randutv_rank_k_state randutv_rank_k_state;

int randutv_rank_k(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q, int64_t k,
                   double* F, int64_t ldf, const randutv_opts* opts, randutv_rank_k_state** state);
int randutv_rank_k_vjp(randutv_rank_k_state* state, const double* Fbar, int64_t ldfb, double* Abar,
                       int64_t ldab);
int randutv_rank_k_free(randutv_rank_k_state* state);

#ifdef __cplusplus
}
#endif

#endif /* RANDUTV_H */

// Unpivoted Householder QR of a tall k x w panel (eq. unpivQR, Section 2.4)
// and the factor S of its compact WY form (eq. WYrepresentation).
//
// randUTV factors two such panels per step: the sample matrix Y (k_c x b),
// whose reflector product is applied from the right, and the new b-column
// panel T([I2,I3], J2), whose product is applied from the left (Fig. 4).
//
// GB300 design: one cooperative launch over up to 152 CTAs; each CTA keeps
// its slice of rows of the panel in shared memory for the whole
// factorization, so HBM is read and written once.  Column j needs, from all
// rows, ||x(2:)||^2 and x^T P(:, c) for c > j; every CTA publishes its
// partial sums, one grid barrier follows, and every CTA then sums the
// partials in the same fixed order (so all CTAs hold bit-identical beta, tau
// and v^T P) and updates its rows.  The partial sums of column j+1 are formed
// right after the update of column j, so each column costs one barrier.
// Convention: LAPACK dlarfg (beta = -sign(alpha)||x||, tau = (beta-alpha)/beta,
// v = x(2:)/(alpha-beta), tau = 0 when x(2:) = 0).
#include <algorithm>
#include "common.cuh"
#include "internal.h"

namespace rutv {

constexpr int PQ_NT = 256;
constexpr int PQ_WARPS = PQ_NT / 32;
constexpr int kMaxCoopBlocks = kNumSMs;
constexpr size_t kPqSmemBudget = 200 * 1024;

__global__ void __launch_bounds__(PQ_NT, 1)
panel_qr_kernel(int64_t k, int w, double* __restrict__ P, int64_t ldp, double* __restrict__ tau_out,
                double* __restrict__ Vexp, double* __restrict__ R, double* __restrict__ part,
                GridBarrier gb, int rpb) {
  extern __shared__ double sm[];
  const int nb = gridDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r_lo = static_cast<int64_t>(blockIdx.x) * rpb;
  const int nr = static_cast<int>(imax64(0, imin64(k, r_lo + rpb) - r_lo));
  double* slice = sm;                         // rpb x w, column-major, ld rpb
  double* vec = slice + static_cast<size_t>(rpb) * w;  // w: reduced t_c
  double* rowj = vec + w;                     // w: row j of the panel (owner's copy)
  double* taus = rowj + w;                    // w: tau of every column
  __shared__ double s_beta, s_tau, s_scale;
  const int PS = 2 * w;                       // partial record per CTA

  for (int64_t idx = tid; idx < static_cast<int64_t>(nr) * w; idx += PQ_NT) {
    const int i = static_cast<int>(idx % nr), c = static_cast<int>(idx / nr);
    slice[i + static_cast<size_t>(c) * rpb] = P[(r_lo + i) + c * ldp];
  }
  __syncthreads();

  // Partial sums of column j over this CTA's rows below row j:
  //   [c] = sum_{i>j} P(i,j) P(i,c)  (c >= j; c = j gives ||x(2:)||^2)
  //   [w + c] = P(j, c)              (only in the CTA owning row j)
  auto partials = [&](int j) {
    double* out = part + static_cast<size_t>(j & 1) * nb * PS + static_cast<size_t>(blockIdx.x) * PS;
    const int i0 = static_cast<int>(imax64(0, j + 1 - r_lo));
    const double* xj = slice + static_cast<size_t>(j) * rpb;
    for (int c = j + warp; c < w; c += PQ_WARPS) {
      const double* xc = slice + static_cast<size_t>(c) * rpb;
      double s = 0.0;
      for (int i = i0 + lane; i < nr; i += 32) s = fma(xj[i], xc[i], s);
      s = warp_sum(s);
      if (lane == 0) out[c] = s;
    }
    const bool owner = (j >= r_lo && j < r_lo + nr);
    for (int c = j + tid; c < w; c += PQ_NT)
      out[w + c] = owner ? slice[(j - r_lo) + static_cast<size_t>(c) * rpb] : 0.0;
  };

  partials(0);
  for (int j = 0; j < w; ++j) {
    if (!grid_barrier(gb, nb)) return;
    const double* pj = part + static_cast<size_t>(j & 1) * nb * PS;
    const int ob = static_cast<int>(j / rpb);  // CTA owning row j
    for (int c = j + tid; c < w; c += PQ_NT) {
      double s = 0.0;
      for (int b = 0; b < nb; ++b) s += pj[static_cast<size_t>(b) * PS + c];
      vec[c] = s;
      rowj[c] = pj[static_cast<size_t>(ob) * PS + w + c];
    }
    __syncthreads();
    if (tid == 0) {
      const double alpha = rowj[j], xn2 = vec[j];
      double beta = alpha, t = 0.0, sc = 0.0;
      if (xn2 != 0.0) {
        const double nrm = sqrt(fma(alpha, alpha, xn2));
        beta = -copysign(nrm, alpha);
        t = (beta - alpha) / beta;
        sc = 1.0 / (alpha - beta);
      }
      s_beta = beta; s_tau = t; s_scale = sc;
      taus[j] = t;
    }
    __syncthreads();
    const double t = s_tau, sc = s_scale;
    // v^T P(:, c) = P(j, c) + scale * sum_{i>j} P(i,j) P(i,c), stored in vec[c]
    for (int c = j + 1 + tid; c < w; c += PQ_NT) vec[c] = fma(sc, vec[c], rowj[c]);
    __syncthreads();
    const int i0 = static_cast<int>(imax64(0, j + 1 - r_lo));
    double* xj = slice + static_cast<size_t>(j) * rpb;
    if (t != 0.0) {
      const int ncols = w - j - 1;
      const int nrows = nr - i0;
      for (int64_t e = tid; e < static_cast<int64_t>(ncols) * nrows; e += PQ_NT) {
        const int i = i0 + static_cast<int>(e % nrows);
        const int c = j + 1 + static_cast<int>(e / nrows);
        slice[i + static_cast<size_t>(c) * rpb] -= t * (xj[i] * sc) * vec[c];
      }
      if (j >= r_lo && j < r_lo + nr) {
        const int il = static_cast<int>(j - r_lo);
        for (int c = j + 1 + tid; c < w; c += PQ_NT) slice[il + static_cast<size_t>(c) * rpb] -= t * vec[c];
      }
    }
    __syncthreads();
    for (int i = i0 + tid; i < nr; i += PQ_NT) xj[i] *= sc;
    if (j >= r_lo && j < r_lo + nr && tid == 0) xj[j - r_lo] = s_beta;
    __syncthreads();
    if (j + 1 < w) partials(j + 1);
  }

  // Write back: P (R above, vectors below), Vexp (explicit), R, tau.
  for (int64_t idx = tid; idx < static_cast<int64_t>(nr) * w; idx += PQ_NT) {
    const int i = static_cast<int>(idx % nr), c = static_cast<int>(idx / nr);
    const int64_t gi = r_lo + i;
    const double v = slice[i + static_cast<size_t>(c) * rpb];
    P[gi + c * ldp] = v;
    double e;
    if (gi > c) e = v;
    else if (gi == c) e = (taus[c] != 0.0) ? 1.0 : 0.0;
    else e = 0.0;
    Vexp[gi + c * k] = e;
    if (gi < w) R[gi + static_cast<int64_t>(c) * w] = (gi <= c) ? v : 0.0;
  }
  if (blockIdx.x == 0)
    for (int c = tid; c < w; c += PQ_NT) tau_out[c] = taus[c];
}

namespace {
struct PqGeom { int rpb; int nb; size_t smem; };

PqGeom pq_geometry(int64_t k, int w) {
  const int64_t max_rows = static_cast<int64_t>(kPqSmemBudget / sizeof(double) - 3 * w) / w;
  int64_t rpb = std::max<int64_t>(32, (k + kMaxCoopBlocks - 1) / kMaxCoopBlocks);
  rpb = std::min<int64_t>(rpb, std::max<int64_t>(1, max_rows));
  int64_t nb = (k + rpb - 1) / rpb;
  PqGeom g;
  g.rpb = static_cast<int>(rpb);
  g.nb = static_cast<int>(nb);
  g.smem = (static_cast<size_t>(rpb) * w + 3 * static_cast<size_t>(w)) * sizeof(double);
  return g;
}
}  // namespace

int64_t panel_qr_part_elems(int64_t k, int w) {
  PqGeom g = pq_geometry(k, w);
  return 2ll * g.nb * 2 * w;
}

cudaError_t panel_qr(cudaStream_t s, int64_t k, int w, double* P, int64_t ldp, double* tau,
                     double* Vexp, double* R, double* part, unsigned* bar) {
  if (k < w || w < 1) return cudaErrorInvalidValue;
  PqGeom g = pq_geometry(k, w);
  if (g.nb > kMaxCoopBlocks) return cudaErrorInvalidConfiguration;  // panel too tall for this layout
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(panel_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kPqSmemBudget + 4096));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  GridBarrier gb{bar, bar + 1, reinterpret_cast<int*>(bar + 2)};
  void* args[] = {&k, &w, &P, &ldp, &tau, &Vexp, &R, &part, &gb, &g.rpb};
  const ProfToken tok = prof_begin(s, kProfPanel);
  e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(panel_qr_kernel), dim3(g.nb), dim3(PQ_NT), args,
                                  g.smem, s);
  note_launch();
  // Householder QR flops 2 k w^2 - 2 w^3 / 3; bytes: panel read + written, Vexp written
  prof_end(s, tok, 2.0 * k * w * w - 2.0 * w * w * w / 3.0, 8.0 * 3.0 * k * w);
  return e;
}

// S = (striu(Gram) + diag(1/tau))^{-1} column by column:
//   S(c,c) = tau_c,  S(i,c) = -tau_i * sum_{l=i+1..c} Gram(i,l) S(l,c)  (i < c),
// which is the forward accumulation of H_1 ... H_w = I - V S V^T (the
// recurrence of the block reflector, Section 2.4) with every column of S
// solved independently: one warp per column.
constexpr int TF_WARPS = 8;

__global__ void __launch_bounds__(TF_WARPS * 32)
tfactor_kernel(int w, const double* __restrict__ gram, const double* __restrict__ tau, double* __restrict__ S) {
  extern __shared__ double scol[];  // TF_WARPS columns of length w
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x * TF_WARPS + warp;
  if (c >= w) return;
  double* x = scol + static_cast<size_t>(warp) * w;
  for (int i = lane; i < w; i += 32) x[i] = 0.0;
  __syncwarp();
  if (lane == 0) x[c] = tau[c];
  __syncwarp();
  for (int i = c - 1; i >= 0; --i) {
    double s = 0.0;
    for (int l = i + 1 + lane; l <= c; l += 32) s = fma(gram[i + static_cast<int64_t>(l) * w], x[l], s);
    s = warp_sum(s);
    if (lane == 0) x[i] = -tau[i] * s;
    __syncwarp();
  }
  for (int i = lane; i < w; i += 32) S[i + static_cast<int64_t>(c) * w] = x[i];
}

cudaError_t tfactor_from_gram(cudaStream_t s, int w, const double* gram, const double* tau, double* S) {
  const int blocks = (w + TF_WARPS - 1) / TF_WARPS;
  const size_t smem = static_cast<size_t>(TF_WARPS) * w * sizeof(double);
  static int attr_w = 0;
  if (smem > 48 * 1024 && w > attr_w) {
    cudaError_t e = cudaFuncSetAttribute(tfactor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    attr_w = w;
  }
  const ProfToken tok = prof_begin(s, kProfTfactor);
  tfactor_kernel<<<blocks, TF_WARPS * 32, smem, s>>>(w, gram, tau, S);
  note_launch();
  prof_end(s, tok, w * static_cast<double>(w) * w / 3.0, 8.0 * 2.0 * w * w);
  return cudaGetLastError();
}

}  // namespace rutv

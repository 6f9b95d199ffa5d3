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
// rows, ||x(2:)||^2 and x^T P(:, c) for c > j; every CTA adds its partial
// sums into one accumulator vector per column with FP64 atomic reductions in
// L2, one grid barrier follows, and every CTA reads the same sums (so all
// hold identical beta, tau and v^T P) and updates its rows.  The partial sums
// of column j+1 are formed right after the update of column j, so each
// column costs one barrier and one L2 round trip.  (The order of the atomic
// additions is not fixed, so results may differ between runs in the last
// bits.)
// Convention: LAPACK dlarfg (beta = -sign(alpha)||x||, tau = (beta-alpha)/beta,
// v = x(2:)/(alpha-beta), tau = 0 when x(2:) = 0).
#include <algorithm>
#include "common.cuh"
#include "internal.h"

namespace rutv {

constexpr int PQ_NT = 256;
constexpr int PQ_WARPS = PQ_NT / 32;
constexpr int kMaxCoopBlocks = kNumSMs;
// Preferred grid: 136 = 152 - 16, so the panel QR of the next step's Y runs
// beside the previous step's small SVD (one 16-CTA cluster); a panel whose
// rows do not fit 136 CTAs' shared memory takes up to 152.
constexpr int kPreferredCoopBlocks = kNumSMs - 16;
constexpr size_t kPqSmemBudget = 226 * 1024;   // of the 227 KB a CTA may use

__global__ void __launch_bounds__(PQ_NT, 1)
panel_qr_kernel(int64_t k, int w, double* __restrict__ P, int64_t ldp, double* __restrict__ tau_out,
                double* __restrict__ Vexp, double* __restrict__ R, double* __restrict__ part,
                GridBarrier gb, int rpb) {
  extern __shared__ double sm[];
  const int nb = gridDim.x;
  const int tid = threadIdx.x;
  const int64_t r_lo = static_cast<int64_t>(blockIdx.x) * rpb;
  const int nr = static_cast<int>(imax64(0, imin64(k, r_lo + rpb) - r_lo));
  double* slice = sm;                         // rpb x w, column-major, ld rpb
  double* vec = slice + static_cast<size_t>(rpb) * w;  // w: sums, then tau * v^T P(:, c)
  double* rowj = vec + w;                     // w: row j of the panel
  double* taus = rowj + w;                    // w: tau of every column
  __shared__ double s_beta, s_tau, s_scale;
  // part: acc (w x w, zeroed by the host) receives the partial sums of
  // column j at acc[j w + c] through FP64 atomic additions in L2; rowbuf
  // (w x w) row j of the panel at rowbuf[j w + c], stored by the owning CTA.
  double* acc = part;
  double* rowbuf = part + static_cast<size_t>(w) * w;

  for (int64_t idx = tid; idx < static_cast<int64_t>(nr) * w; idx += PQ_NT) {
    const int i = static_cast<int>(idx % nr), c = static_cast<int>(idx / nr);
    slice[i + static_cast<size_t>(c) * rpb] = P[(r_lo + i) + c * ldp];
  }
  __syncthreads();

  // This CTA's contribution to column j's sums over the rows below row j:
  //   acc[j w + c] += sum_{i>j} P(i,j) P(i,c)  (c >= j; c = j gives ||x(2:)||^2)
  // and, from the CTA owning row j, rowbuf[j w + c] = P(j, c).
  auto partials = [&](int j) {
    const int i0 = static_cast<int>(imax64(0, j + 1 - r_lo));
    const double* xj = slice + static_cast<size_t>(j) * rpb;
    if (i0 < nr) {
      for (int c = j + tid; c < w; c += PQ_NT) {
        const double* xc = slice + static_cast<size_t>(c) * rpb;
        double s0 = 0.0, s1 = 0.0;
        int i = i0;
        for (; i + 1 < nr; i += 2) { s0 = fma(xj[i], xc[i], s0); s1 = fma(xj[i + 1], xc[i + 1], s1); }
        if (i < nr) s0 = fma(xj[i], xc[i], s0);
        atomicAdd(acc + static_cast<size_t>(j) * w + c, s0 + s1);
      }
    }
    if (j >= r_lo && j < r_lo + nr)
      for (int c = j + tid; c < w; c += PQ_NT)
        rowbuf[static_cast<size_t>(j) * w + c] = slice[(j - r_lo) + static_cast<size_t>(c) * rpb];
  };

  partials(0);
  for (int j = 0; j < w; ++j) {
    if (!grid_barrier(gb, nb)) return;
    for (int c = j + tid; c < w; c += PQ_NT) {
      vec[c] = __ldcg(acc + static_cast<size_t>(j) * w + c);
      rowj[c] = __ldcg(rowbuf + static_cast<size_t>(j) * w + c);
    }
    __syncthreads();
    if (tid == 0) {
      const double alpha = rowj[j], xn2 = vec[j];
      double beta = alpha, t = 0.0, sc = 0.0;
      if (xn2 != 0.0) {
        const double nrm = sqrt(fma(alpha, alpha, xn2));
        beta = -copysign(nrm, alpha);
        // tau = (beta - alpha) / beta and scale = 1 / (alpha - beta) from one division
        const double r = 1.0 / (beta * (alpha - beta));
        t = (beta - alpha) * ((alpha - beta) * r);
        sc = beta * r;
      }
      s_beta = beta; s_tau = t; s_scale = sc;
      taus[j] = t;
    }
    __syncthreads();
    const double t = s_tau, sc = s_scale;
    // vec[c] <- tau * v^T P(:, c) = tau * (P(j, c) + scale * sum_{i>j} P(i,j) P(i,c))
    for (int c = j + 1 + tid; c < w; c += PQ_NT) vec[c] = t * fma(sc, vec[c], rowj[c]);
    const int i0 = static_cast<int>(imax64(0, j + 1 - r_lo));
    double* xj = slice + static_cast<size_t>(j) * rpb;
    for (int i = i0 + tid; i < nr; i += PQ_NT) xj[i] *= sc;   // x(2:) -> v(2:)
    __syncthreads();
    if (t != 0.0) {
      const int ncols = w - j - 1;
      const int nrows = nr - i0;
      if (nrows > 0)
        for (int64_t e = tid; e < static_cast<int64_t>(ncols) * nrows; e += PQ_NT) {
          const int i = i0 + static_cast<int>(e % nrows);
          const int c = j + 1 + static_cast<int>(e / nrows);
          slice[i + static_cast<size_t>(c) * rpb] = fma(-xj[i], vec[c], slice[i + static_cast<size_t>(c) * rpb]);
        }
      if (j >= r_lo && j < r_lo + nr) {
        const int il = static_cast<int>(j - r_lo);
        for (int c = j + 1 + tid; c < w; c += PQ_NT) slice[il + static_cast<size_t>(c) * rpb] -= vec[c];
      }
    }
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
  int64_t rpb = std::max<int64_t>(32, (k + kPreferredCoopBlocks - 1) / kPreferredCoopBlocks);
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
  (void)k;
  return 2ll * w * w;   // accumulators + rows
}

cudaError_t panel_qr(cudaStream_t s, int64_t k, int w, double* P, int64_t ldp, double* tau,
                     double* Vexp, double* R, double* part, unsigned* bar) {
  if (k < w || w < 1) return cudaErrorInvalidValue;
  PqGeom g = pq_geometry(k, w);
  if (g.nb > kMaxCoopBlocks) return cudaErrorInvalidConfiguration;  // panel too tall for this layout
  static PerDeviceOnce once;
  cudaError_t e = per_device_once(once, [] {
    return cudaFuncSetAttribute(panel_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kPqSmemBudget));
  });
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(part, 0, static_cast<size_t>(w) * w * sizeof(double), s);
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
// solved independently: one warp per column.  Gram = V^T V is symmetric, so
// Gram(i, l) is read as Gram(l, i): consecutive l across the lanes, one
// coalesced segment per step instead of 32 scattered lines.
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
    for (int l = i + 1 + lane; l <= c; l += 32) s = fma(gram[l + static_cast<int64_t>(i) * w], x[l], s);
    s = warp_sum(s);
    if (lane == 0) x[i] = -tau[i] * s;
    __syncwarp();
  }
  for (int i = lane; i < w; i += 32) S[i + static_cast<int64_t>(c) * w] = x[i];
}

cudaError_t tfactor_from_gram(cudaStream_t s, int w, const double* gram, const double* tau, double* S) {
  if (w < 1 || w > 256) return cudaErrorInvalidValue;
  const int blocks = (w + TF_WARPS - 1) / TF_WARPS;
  const size_t smem = static_cast<size_t>(TF_WARPS) * w * sizeof(double);
  // the largest block (w = 256) bounds every launch: one attribute per device
  static PerDeviceOnce once;
  if (smem > 48 * 1024) {
    cudaError_t e = per_device_once(once, [] {
      return cudaFuncSetAttribute(tfactor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(static_cast<size_t>(TF_WARPS) * 256 * sizeof(double)));
    });
    if (e != cudaSuccess) return e;
  }
  const ProfToken tok = prof_begin(s, kProfTfactor);
  tfactor_kernel<<<blocks, TF_WARPS * 32, smem, s>>>(w, gram, tau, S);
  note_launch();
  prof_end(s, tok, w * static_cast<double>(w) * w / 3.0, 8.0 * 2.0 * w * w);
  return cudaGetLastError();
}

}  // namespace rutv

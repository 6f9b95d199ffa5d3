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
// L2, one grid barrier follows, and one thread reads the two sums that
// define the reflector and forms beta, tau and the scale for all (a
// warp-wide FP64 square root and division would cost 32 times as much on
// the slow FP64 pipe).  Per column, after the barrier: column j+1 is
// updated first, then each group of 1-8 threads takes a column c > j+1,
// updates it and, in the same pass over its rows, forms its dot product
// with the new column j+1 (the next column's sums), so a column costs one
// barrier, one L2 round trip and two __syncthreads.  The scaling of x(2:) to v is
// deferred by one column (nobody reads it meanwhile).  (The order of the
// atomic additions is not fixed, so results may differ between runs in the
// last bits.)
// Convention: LAPACK dlarfg (beta = -sign(alpha)||x||, tau = (beta-alpha)/beta,
// v = x(2:)/(alpha-beta), tau = 0 when x(2:) = 0).
#include <algorithm>
#include "common.cuh"
#include "internal.h"

namespace rutv {

constexpr int PQ_NT = 256;
constexpr int kMaxCoopBlocks = kNumSMs;
// Preferred grid: 136 = 152 - 16, so the panel QR of the next step's Y runs
// beside the previous step's small SVD (one 16-CTA cluster); a panel whose
// rows do not fit 136 CTAs' shared memory takes up to 152.
constexpr int kPreferredCoopBlocks = kNumSMs - 16;
constexpr size_t kPqSmemBudget = 226 * 1024;   // of the 227 KB a CTA may use

// Reflector j from its two sums: alpha = P(j, j) and xn2 = ||x(2:)||^2.
// With rho = 1 / ||(alpha, x(2:))|| from one reciprocal square root:
// beta = -sign(alpha) / rho, tau = (beta - alpha) / beta = 1 + |alpha| rho,
// and scale = 1 / (alpha - beta) = sign(alpha) / (|alpha| + ||.||) from one
// reciprocal; no division, fewer instructions on the slow FP64 pipe of the
// one thread that forms it.
struct PqRefl { double beta, tau, scale; };
__device__ __forceinline__ PqRefl pq_reflector(double alpha, double xn2) {
  PqRefl r{alpha, 0.0, 0.0};
  if (xn2 != 0.0) {
    const double nrm2 = fma(alpha, alpha, xn2);
    const double rho = rsqrt(nrm2);
    const double nrm = nrm2 * rho;
    r.beta = -copysign(nrm, alpha);
    r.tau = fma(fabs(alpha), rho, 1.0);
    r.scale = copysign(__drcp_rn(fabs(alpha) + nrm), alpha);
  }
  return r;
}

__global__ void __launch_bounds__(PQ_NT, 1)
panel_qr_kernel(int64_t k, int w, double* __restrict__ P, int64_t ldp, double* __restrict__ tau_out,
                double* __restrict__ Vexp, double* __restrict__ R, double* __restrict__ part,
                GridBarrier gb, int rpb) {
  extern __shared__ double sm[];
  const int nb = gridDim.x;
  const int tid = threadIdx.x;
  const int64_t r_lo = static_cast<int64_t>(blockIdx.x) * rpb;
  const int nr = static_cast<int>(imax64(0, imin64(k, r_lo + rpb) - r_lo));
  double* slice = sm;                                   // rpb x w, column-major, ld rpb
  double* taus = slice + static_cast<size_t>(rpb) * w;  // w: the scale of each column, then its tau
  __shared__ double s_h[5];   // the column's beta, tau, scale, and column j+1's wc, wc * scale
  // part: acc (w x w, zeroed by the host) receives the partial sums of
  // column j at acc[j w + c] through FP64 atomic additions in L2; rowbuf
  // (w x w) row j of the panel at rowbuf[j w + c], stored by the owning CTA.
  double* acc = part;
  double* rowbuf = part + static_cast<size_t>(w) * w;
  auto col = [&](int c) { return slice + static_cast<size_t>(c) * rpb; };
  // local index of global row g in this CTA, or -1
  auto own = [&](int64_t g) { return (g >= r_lo && g < r_lo + nr) ? static_cast<int>(g - r_lo) : -1; };
  // Column groups: G threads (adjacent lanes, G a power of two <= 8) per
  // column, each taking every G-th row; a group's sum is combined by
  // shuffles among its own lanes (groups never straddle a warp and run
  // their loop iterations together).
  auto group_size = [&](int ncols) {
    int g = 1;
    while (g < 8 && 2 * g * ncols <= PQ_NT) g *= 2;
    return g;
  };
  auto group_mask = [&](int G) { return ((1u << G) - 1u) << ((tid & 31) & ~(G - 1)); };

  for (int c = 0; c < w; ++c)
    for (int i = tid; i < nr; i += PQ_NT) col(c)[i] = P[(r_lo + i) + c * ldp];
  __syncthreads();

  // Sums of column 0: acc[c] += sum_{i>0} P(i,0) P(i,c), rowbuf[c] = P(0, c).
  {
    const int G = group_size(w);
    const int grp = tid / G, sub = tid % G;
    const unsigned gm = group_mask(G);
    const int i1 = static_cast<int>(imax64(0, 1 - r_lo));
    const int l0 = own(0);
    const double* x0 = col(0);
    for (int c = grp; c < w; c += PQ_NT / G) {
      const double* xc = col(c);
      double s0 = 0.0;
      for (int i = i1 + sub; i < nr; i += G) s0 = fma(x0[i], xc[i], s0);
      for (int o = G / 2; o > 0; o >>= 1) s0 += __shfl_xor_sync(gm, s0, o, G);
      if (sub == 0) {
        if (i1 < nr) atomicAdd(acc + c, s0);
        if (l0 >= 0) rowbuf[c] = xc[l0];
      }
    }
  }

  for (int j = 0; j < w; ++j) {
    if (!grid_barrier(gb, nb)) return;
    const double* accj = acc + static_cast<size_t>(j) * w;
    const double* rowj = rowbuf + static_cast<size_t>(j) * w;
    // Every sum this thread needs for column j, loaded at once (one L2 round
    // trip): the reflector's two, column j+1's two, and those of the first
    // column of this thread's group in the pass below.
    const int ncols = w - j - 1;
    const int G = group_size(ncols > 0 ? ncols : 1);
    const int grp = tid / G, sub = tid % G;
    // FP64 is the slow pipe here and a warp-wide FP64 instruction costs the
    // same with one lane or 32: thread 0 alone forms the reflector (a square
    // root and a division) and column j+1's coefficients, for all to read.
    double a_c = 0.0, r_c = 0.0;
    if (grp >= 1 && grp < ncols) { a_c = __ldcg(accj + j + 1 + grp); r_c = __ldcg(rowj + j + 1 + grp); }
    if (tid == 0) {
      const double a_jj = __ldcg(accj + j), r_jj = __ldcg(rowj + j);
      double a_n = 0.0, r_n = 0.0;
      if (j + 1 < w) { a_n = __ldcg(accj + j + 1); r_n = __ldcg(rowj + j + 1); }
      const PqRefl hh = pq_reflector(r_jj, a_jj);
      const double wc = hh.tau * fma(hh.scale, a_n, r_n);
      s_h[0] = hh.beta; s_h[1] = hh.tau; s_h[2] = hh.scale; s_h[3] = wc; s_h[4] = wc * hh.scale;
    }
    __syncthreads();
    const PqRefl h{s_h[0], s_h[1], s_h[2]};
    const int lj = own(j);                                        // local row of j (or -1)
    const int i0 = static_cast<int>(imax64(0, j + 1 - r_lo));     // first local row below j
    const double* xj = col(j);                                    // x(2:) of column j, unscaled
    // Column j+1 first (the next reflector's column): for i > j
    // P(i, j+1) -= v_i wc with v_i = scale x_i, wc = tau (P(j, j+1) + scale
    // sum_{i>j} x_i P(i, j+1)), and P(j, j+1) -= wc.  Meanwhile x(2:) of
    // column j-1 becomes v (nobody reads it any more).
    if (j + 1 < w && h.tau != 0.0) {
      const double wc = s_h[3], ws = s_h[4];
      double* xn = col(j + 1);
      for (int i = i0 + tid; i < nr; i += PQ_NT) xn[i] = fma(-xj[i], ws, xn[i]);
      if (lj >= 0 && tid == 0) xn[lj] -= wc;
    }
    if (j > 0) {
      const double sp = taus[j - 1];
      double* xp = col(j - 1);
      for (int i = static_cast<int>(imax64(0, j - r_lo)) + tid; i < nr; i += PQ_NT) xp[i] *= sp;
    }
    if (tid == 0) taus[j] = h.scale;
    __syncthreads();
    // The columns c > j+1: update them, and in the same pass over the rows
    // form the sums of column j+1 over rows > j+1:
    //   acc[(j+1) w + c] += sum_{i>j+1} P(i, j+1) P(i, c)   (c = j+1: ||x(2:)||^2);
    // the owner of row j+1 records that row (after the update) in rowbuf.
    if (j + 1 < w) {
      const unsigned gm = group_mask(G);
      const int i1 = static_cast<int>(imax64(0, j + 2 - r_lo));   // first local row below j+1
      const int ln = own(j + 1);
      const double* xn = col(j + 1);
      double* accn = acc + static_cast<size_t>(j + 1) * w;
      double* rown = rowbuf + static_cast<size_t>(j + 1) * w;
      for (int cc = grp; cc < ncols; cc += PQ_NT / G) {
        const int c = j + 1 + cc;
        double* xc = col(c);
        double s0 = 0.0;
        if (c > j + 1 && h.tau != 0.0) {
          if (cc != grp) { a_c = __ldcg(accj + c); r_c = __ldcg(rowj + c); }   // only when w > PQ_NT
          const double wc = h.tau * fma(h.scale, a_c, r_c);
          const double ws = wc * h.scale;
          if (ln >= 0 && sub == 0) xc[ln] = fma(-xj[ln], ws, xc[ln]);   // row j+1: updated, not summed
          for (int i = i1 + sub; i < nr; i += G) {
            const double v = fma(-xj[i], ws, xc[i]);
            xc[i] = v;
            s0 = fma(xn[i], v, s0);
          }
          if (lj >= 0 && sub == 0) xc[lj] -= wc;
        } else {
          for (int i = i1 + sub; i < nr; i += G) s0 = fma(xn[i], xc[i], s0);
        }
        for (int o = G / 2; o > 0; o >>= 1) s0 += __shfl_xor_sync(gm, s0, o, G);
        if (sub == 0) {
          if (i1 < nr) atomicAdd(accn + c, s0);
          if (ln >= 0) rown[c] = xc[ln];
        }
      }
    }
    if (lj >= 0 && tid == 0) col(j)[lj] = h.beta;
  }
  __syncthreads();
  // the last column's x(2:) becomes v; then the scales in taus[] give way to tau
  {
    const double sp = taus[w - 1];
    double* xp = col(w - 1);
    for (int i = static_cast<int>(imax64(0, w - r_lo)) + tid; i < nr; i += PQ_NT) xp[i] *= sp;
  }
  __syncthreads();
  for (int c = tid; c < w; c += PQ_NT)
    taus[c] = pq_reflector(__ldcg(rowbuf + static_cast<size_t>(c) * w + c), __ldcg(acc + static_cast<size_t>(c) * w + c)).tau;
  __syncthreads();

  // Write back: P (R above, vectors below), Vexp (explicit), R, tau.
  for (int c = 0; c < w; ++c) {
    const double tc = taus[c];
    const double* xc = col(c);
    for (int i = tid; i < nr; i += PQ_NT) {
      const int64_t gi = r_lo + i;
      const double v = xc[i];
      P[gi + c * ldp] = v;
      double e;
      if (gi > c) e = v;
      else if (gi == c) e = (tc != 0.0) ? 1.0 : 0.0;
      else e = 0.0;
      Vexp[gi + c * k] = e;
      if (gi < w) R[gi + static_cast<int64_t>(c) * w] = (gi <= c) ? v : 0.0;
    }
  }
  if (blockIdx.x == 0)
    for (int c = tid; c < w; c += PQ_NT) tau_out[c] = taus[c];
}

namespace {
struct PqGeom { int rpb; int nb; size_t smem; };

PqGeom pq_geometry(int64_t k, int w) {
  const int64_t max_rows = static_cast<int64_t>(kPqSmemBudget / sizeof(double) - w) / w;
  int64_t rpb = std::max<int64_t>(32, (k + kPreferredCoopBlocks - 1) / kPreferredCoopBlocks);
  rpb = std::min<int64_t>(rpb, std::max<int64_t>(1, max_rows));
  int64_t nb = (k + rpb - 1) / rpb;
  PqGeom g;
  g.rpb = static_cast<int>(rpb);
  g.nb = static_cast<int>(nb);
  g.smem = (static_cast<size_t>(rpb) * w + static_cast<size_t>(w)) * sizeof(double);
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
constexpr int TF_STAGED_MAX_W = 128;   // the right-looking form below, up to this width
constexpr int TF_RL_WARPS = 4;         // one warp per SMSP: a warp alone on its FP64 pipe

// Right-looking back-substitution for column c of S, one warp per column
// and one warp per SMSP (FP64 issues at 0.5 lanes per clock per SMSP, so a
// warp-wide FP64 instruction takes 64 cycles and a second warp on the SMSP
// would halve the rate).  With x_c = tau_c, for l = c, c-1, .., 1: every
// lane adds Gram(i, l) x_l into its partial sums acc_i (i < l, lane i mod
// 32, at most 4 per lane), and the owner of i = l-1 forms x_{l-1} = -tau_{l-1}
// acc_{l-1}: a chain of one FMA, one multiply and a shared-memory broadcast
// per step, instead of a 5-step warp reduction in FP64.  The Gram block the
// CTA's columns need (Gram(0:cm, 0:cm), column-major, read down columns) and
// tau are staged in shared memory first.
__global__ void __launch_bounds__(TF_RL_WARPS * 32)
tfactor_rl_kernel(int w, const double* __restrict__ gram, const double* __restrict__ tau, double* __restrict__ S) {
  extern __shared__ double tsm[];
  double* ts = tsm;                                   // tau (w)
  double* xs = ts + w;                                // TF_RL_WARPS columns of x (w each)
  double* gs = xs + static_cast<size_t>(TF_RL_WARPS) * w;   // Gram(0:cm, 0:cm), ld cm
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cm = min(w, (blockIdx.x + 1) * TF_RL_WARPS);
  for (int i = threadIdx.x; i < w; i += TF_RL_WARPS * 32) ts[i] = tau[i];
  for (int l = warp; l < cm; l += TF_RL_WARPS)
    for (int i = lane; i < cm; i += 32) gs[i + l * cm] = gram[i + static_cast<int64_t>(l) * w];
  __syncthreads();
  const int c = blockIdx.x * TF_RL_WARPS + warp;
  if (c >= w) return;
  double* x = xs + static_cast<size_t>(warp) * w;
  double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;   // i = lane + 32 k, k = 0..3
  if (lane == 0) x[c] = ts[c];
  __syncwarp();
  for (int l = c; l >= 1; --l) {
    const double xl = x[l];
    const double* gl = gs + l * cm;
    // rows i < l; the k-th block of 32 rows takes part while 32 k < l
    if (lane < l) acc0 = fma(gl[lane], xl, acc0);
    if (l > 32 && lane + 32 < l) acc1 = fma(gl[lane + 32], xl, acc1);
    if (l > 64 && lane + 64 < l) acc2 = fma(gl[lane + 64], xl, acc2);
    if (l > 96 && lane + 96 < l) acc3 = fma(gl[lane + 96], xl, acc3);
    const int i = l - 1;
    if (lane == (i & 31)) {
      const int k = i >> 5;
      const double a = k == 0 ? acc0 : (k == 1 ? acc1 : (k == 2 ? acc2 : acc3));
      x[i] = -ts[i] * a;
    }
    __syncwarp();
  }
  for (int i = lane; i < w; i += 32) S[i + static_cast<int64_t>(c) * w] = (i <= c) ? x[i] : 0.0;
}

// The same column by column as a left-looking solve (one warp reduction per
// step) for wider blocks: x_i = -tau_i sum_{l=i+1..c} Gram(l, i) x_l, with
// Gram(l, i) read down the lower triangle (coalesced).
__global__ void __launch_bounds__(TF_WARPS * 32)
tfactor_kernel(int w, const double* __restrict__ gram, const double* __restrict__ tau, double* __restrict__ S) {
  extern __shared__ double tsm[];
  double* scol = tsm;                                   // TF_WARPS columns of length w
  double* ts = scol + static_cast<size_t>(TF_WARPS) * w;   // tau (w)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < w; i += TF_WARPS * 32) ts[i] = tau[i];
  __syncthreads();
  const int c = blockIdx.x * TF_WARPS + warp;
  if (c >= w) return;
  double* x = scol + static_cast<size_t>(warp) * w;
  for (int i = lane; i < w; i += 32) x[i] = 0.0;
  __syncwarp();
  if (lane == 0) x[c] = ts[c];
  __syncwarp();
  for (int i = c - 1; i >= 0; --i) {
    double sum = 0.0;
    for (int l = i + 1 + lane; l <= c; l += 32) sum = fma(gram[l + static_cast<int64_t>(i) * w], x[l], sum);
    sum = warp_sum(sum);
    if (lane == 0) x[i] = -ts[i] * sum;
    __syncwarp();
  }
  for (int i = lane; i < w; i += 32) S[i + static_cast<int64_t>(c) * w] = x[i];
}

cudaError_t tfactor_from_gram(cudaStream_t s, int w, const double* gram, const double* tau, double* S) {
  if (w < 1 || w > 256) return cudaErrorInvalidValue;
  static PerDeviceOnce once;
  cudaError_t e = per_device_once(once, [] {
    const size_t s1 = (static_cast<size_t>(TF_STAGED_MAX_W) * (1 + TF_RL_WARPS) +
                       static_cast<size_t>(TF_STAGED_MAX_W) * TF_STAGED_MAX_W) * sizeof(double);
    const size_t s0 = (static_cast<size_t>(TF_WARPS) * 256 + 256) * sizeof(double);
    cudaError_t r = cudaFuncSetAttribute(tfactor_rl_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(s1));
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(tfactor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(s0));
    return r;
  });
  if (e != cudaSuccess) return e;
  const ProfToken tok = prof_begin(s, kProfTfactor);
  if (w <= TF_STAGED_MAX_W) {
    const int blocks = (w + TF_RL_WARPS - 1) / TF_RL_WARPS;
    const size_t smem = (static_cast<size_t>(w) * (1 + TF_RL_WARPS) + static_cast<size_t>(w) * w) * sizeof(double);
    tfactor_rl_kernel<<<blocks, TF_RL_WARPS * 32, smem, s>>>(w, gram, tau, S);
  } else {
    const int blocks = (w + TF_WARPS - 1) / TF_WARPS;
    const size_t smem = (static_cast<size_t>(TF_WARPS) * w + w) * sizeof(double);
    tfactor_kernel<<<blocks, TF_WARPS * 32, smem, s>>>(w, gram, tau, S);
  }
  note_launch();
  prof_end(s, tok, w * static_cast<double>(w) * w / 3.0, 8.0 * 2.0 * w * w);
  return cudaGetLastError();
}

}  // namespace rutv

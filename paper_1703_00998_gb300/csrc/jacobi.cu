// SVD of the small active block (Fig. 4: [Us, Ds, Vs] = svd(R(1:b,1:b)), and
// the full SVD of the last block) by one-sided cyclic Jacobi (Hestenes) in
// FP64.
//
// The rotations act on the columns of W = M^T (the rows of M): pairs i < j
// are rotated until |w_i . w_j| <= tol ||w_i|| ||w_j|| for all of them, the
// rotations accumulate in Q, and then W = M^T Q = N diag(sigma) with unit
// columns N, i.e. M = Q diag(sigma) N^T: Us = Q, Vs = N.  Working on the rows
// matters for the upper triangular R11 of randUTV: its columns are graded
// like its singular values and one-sided Jacobi on them converges several
// times more slowly than on its rows.  The p(p-1)/2 pairs of a sweep are
// ordered as a round-robin tournament: p-1 rounds of p/2 disjoint pairs.
//
// GB300 design: FP64 runs at ~4 flop/clk/SM, so one SM would need tens of
// milliseconds for a 128 x 128 SVD.  One thread-block cluster of 16 CTAs
// (16 SMs) holds W and Q in distributed shared memory (2 p^2 doubles spread
// over the 16 CTAs), each warp rotates one pair of a round at a time through
// DSMEM loads and stores, and the hardware cluster barrier separates the
// rounds: no global-memory round trips and no software grid barrier.
// Order and signs: singular values descending (stable in the column index);
// the largest-|.| entry of each Vs column positive (lowest index on ties),
// Us flipped with it; zero singular values get Vs columns that complete an
// orthonormal basis (Gram-Schmidt of unit vectors).  The ordering, scaling
// and signs are done in the epilogue of the FP64 sweep kernel, on all 16 SMs.
#include <cooperative_groups.h>
#include "common.cuh"
#include "internal.h"

namespace rutv {

constexpr int JC_CLUSTER = 16;   // CTAs of the cluster (non-portable size, opt-in)
constexpr int JC_NT = 128;       // 4 warps per CTA, one pair per warp at a time
constexpr int JC_WARPS = JC_NT / 32;
constexpr int JC_MAXP = 256;

// dynamic shared memory of one CTA: W and Q slots (p doubles each) + norms
__host__ __device__ constexpr size_t jc_smem(int p, int cs) {
  return (2ull * ((p + (p & 1) + cs - 1) / cs) * p + ((p + (p & 1) + cs - 1) / cs)) * sizeof(double);
}
constexpr size_t kJcSmemMax = jc_smem(JC_MAXP, 8);
__host__ __device__ constexpr size_t jc_smem32(int p, int cs) {
  return (2ull * ((p + (p & 1) + cs - 1) / cs) * p + ((p + (p & 1) + cs - 1) / cs)) * sizeof(float);
}

__device__ __forceinline__ void rr_pair(int pp, int r, int kpair, int* a, int* b) {
  auto idx = [&](int t) { return t == 0 ? 0 : ((t - 1 + r) % (pp - 1)) + 1; };
  int x = idx(kpair), y = idx(pp - 1 - kpair);
  *a = min(x, y);
  *b = max(x, y);
}

// One cluster of cs CTAs (16, or 8 where 16 cannot be scheduled).  Column c
// of W (= M^T, rotated) and of Q (accumulated rotations) lives in the shared
// memory of CTA c % cs, slot c / cs, with its squared norm; a warp that
// rotates the pair (i, j) reads and writes both columns through distributed
// shared memory, and the rounds are separated by the cluster barrier.  The
// epilogue writes the ordered, signed Us, d and Vs.
//
// FP64 issues at 2 lanes/clk/SM on this GPU, so every FP64 instruction of a
// warp costs its SM sub-partition ~64 cycles; the kernel keeps their number
// per rotation small: NU = ceil(p/32) rows per lane exactly, one dot product
// per pair (the squared column norms are carried along with the exact norm
// formulas of the applied rotation and recomputed at every sweep), and the
// rotation angle t from FP32 arithmetic.  The rotation itself is exactly
// orthogonal in FP64 (c = 1/sqrt(1 + t^2), s = c t), so an FP32 angle only
// changes how much of w_i . w_j a rotation removes, not the accuracy of W, Q.
template <int NU>
__global__ void __launch_bounds__(JC_NT)
jacobi_cluster_kernel(int p, const double* __restrict__ M, int64_t ldm, const double* W0, const double* Q0,
                      double* __restrict__ Us, double* __restrict__ d, double* __restrict__ Vs, int max_sweeps,
                      double tol, int* __restrict__ err, int* __restrict__ zero_flag) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double jsm[];
  const int rank = static_cast<int>(cluster.block_rank());
  const int cs = static_cast<int>(cluster.num_blocks());   // 16, or 8 where 16 cannot be scheduled
  const int pp = p + (p & 1);
  const int slots = (pp + cs - 1) / cs;
  double* Wl = jsm;                                    // slots x p
  double* Ql = jsm + static_cast<size_t>(slots) * p;   // slots x p
  double* Nl = Ql + static_cast<size_t>(slots) * p;    // slots: squared norms of the W columns
  __shared__ double s_part[JC_CLUSTER];
  __shared__ double s_fro;
  __shared__ int s_flag[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // Load this CTA's columns: W(:, c) = M(c, :)^T and Q = I, or the given
  // starting point W0 = M^T Q0 (p x p, ld p) after the FP32 sweeps.
  for (int sl = 0; sl < slots; ++sl) {
    const int c = sl * cs + rank;
    for (int t = tid; t < p; t += JC_NT) {
      if (W0) {
        Wl[sl * p + t] = (c < p) ? W0[t + static_cast<int64_t>(c) * p] : 0.0;
        Ql[sl * p + t] = (c < p) ? Q0[t + static_cast<int64_t>(c) * p] : 0.0;
      } else {
        Wl[sl * p + t] = (c < p) ? M[c + static_cast<int64_t>(t) * ldm] : 0.0;
        Ql[sl * p + t] = (c < p && t == c) ? 1.0 : 0.0;
      }
    }
  }
  __syncthreads();
  // ||M||_F^2, summed in the same order by every CTA.
  if (warp == 0) {
    double f = 0.0;
    for (int e = lane; e < slots * p; e += 32) f = fma(Wl[e], Wl[e], f);
    f = warp_sum(f);
    if (lane == 0) s_part[rank] = f;
  }
  if (tid < 2) s_flag[tid] = 0;
  cluster.sync();
  if (tid == 0) {
    double f = 0.0;
    for (int q = 0; q < cs; ++q) f += *cluster.map_shared_rank(&s_part[q], q);
    s_fro = f;
  }
  __syncthreads();
  // Columns with ||w|| <= p u ||M||_F are at the rounding level of the block
  // and count as zero (rotating them only stirs rounding noise).
  const double pu = static_cast<double>(p) * 0x1p-53;
  const double thr2 = pu * pu * s_fro;
  const double tol2 = tol * tol;
  const int npairs = pp / 2;

  bool converged = false;
  for (int sw = 0; sw < max_sweeps && !converged; ++sw) {
    // exact squared norms of this CTA's columns at the start of the sweep
    for (int sl = warp; sl < slots; sl += JC_WARPS) {
      double f = 0.0;
      for (int t = lane; t < p; t += 32) f = fma(Wl[sl * p + t], Wl[sl * p + t], f);
      f = warp_sum(f);
      if (lane == 0) Nl[sl] = f;
    }
    if (tid == 0) s_flag[sw & 1] = 0;
    cluster.sync();
    for (int r = 0; r < pp - 1; ++r) {
      for (int k = rank * JC_WARPS + warp; k < npairs; k += cs * JC_WARPS) {
        int i, j;
        rr_pair(pp, r, k, &i, &j);
        if (j >= p) continue;
        const int oi = i % cs, oj = j % cs, si = (i / cs), sj = (j / cs);
        double* wi = cluster.map_shared_rank(Wl + si * p, oi);
        double* wj = cluster.map_shared_rank(Wl + sj * p, oj);
        double* ni = cluster.map_shared_rank(Nl + si, oi);
        double* nj = cluster.map_shared_rank(Nl + sj, oj);
        double* qi = cluster.map_shared_rank(Ql + si * p, oi);
        double* qj = cluster.map_shared_rank(Ql + sj * p, oj);
        double x[NU], y[NU], q1[NU], q2[NU];
        double g = 0.0;
#pragma unroll
        for (int u = 0; u < NU; ++u) {   // Q columns fetched with W: one round trip
          const int t = lane + 32 * u;
          x[u] = (t < p) ? wi[t] : 0.0;
          y[u] = (t < p) ? wj[t] : 0.0;
          q1[u] = (t < p) ? qi[t] : 0.0;
          q2[u] = (t < p) ? qj[t] : 0.0;
          g = fma(x[u], y[u], g);
        }
        const double a = *ni, b = *nj;
        g = warp_sum(g);   // identical in every lane
        if (g == 0.0 || a <= thr2 || b <= thr2 || !(g * g > tol2 * a * b)) continue;
        // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (b - a) / (2 g), in FP32
        // zeta is scale-invariant: bring (b - a) and g to [-2, 2] by an exact
        // power of two before rounding them to FP32 (blocks at the rounding
        // level have w_i . w_j ~ 1e-46, below the FP32 range)
        const double dba = b - a;
        const double mx = fmax(fabs(dba), fabs(g));
        const long long ex = (__double_as_longlong(mx) >> 52) & 0x7ff;
        double tt;
        float bf = 0.f, gf = 0.f, zf = 0.f;
        bool fp32_ok = ex > 0 && ex < 2046;
        if (fp32_ok) {
          const double sc = __longlong_as_double(static_cast<long long>(2046 - ex) << 52);   // 2^(1023 - ex)
          bf = static_cast<float>(dba * sc);
          gf = static_cast<float>(g * sc);
          fp32_ok = fabsf(gf) >= 0x1p-100f;
          if (fp32_ok) zf = bf / (2.0f * gf);
        }
        if (fp32_ok) {
          // for |zeta| > 2^60, zeta^2 would overflow: t -> 1 / (2 zeta)
          const float tf = (fabsf(zf) > 0x1p60f) ? 0.5f / zf
                                                  : copysignf(1.0f, zf) / (fabsf(zf) + sqrtf(fmaf(zf, zf, 1.0f)));
          tt = static_cast<double>(tf);
        } else {
          const double zeta = (b - a) / (2.0 * g);   // rare: outside the FP32 range
          tt = (fabs(zeta) > 0x1p500) ? 0.5 / zeta
                                      : copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
        }
        const double c = rsqrt(fma(tt, tt, 1.0));
        const double sn = c * tt;
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          const int t = lane + 32 * u;
          if (t < p) {
            wi[t] = fma(c, x[u], -sn * y[u]);
            wj[t] = fma(sn, x[u], c * y[u]);
            qi[t] = fma(c, q1[u], -sn * q2[u]);
            qj[t] = fma(sn, q1[u], c * q2[u]);
          }
        }
        if (lane == 0) {
          // squared norms after the applied rotation (c, s)
          const double cc = c * c, ss = sn * sn, csg = 2.0 * c * sn * g;
          *ni = fma(cc, a, fma(ss, b, -csg));
          *nj = fma(ss, a, fma(cc, b, csg));
          s_flag[sw & 1] = 1;
        }
      }
      cluster.sync();
    }
    // A sweep without rotations anywhere in the cluster: converged.
    int any = 0;
    for (int q = 0; q < cs; ++q) any |= *cluster.map_shared_rank(&s_flag[sw & 1], q);
    converged = (any == 0);
  }
  if (!converged && rank == 0 && tid == 0) atomicOr(err, kDevErrNoConv);

  // Epilogue on the 16 SMs: sigma_c = ||w_c||, the order (descending, stable
  // in c), Vs = w / sigma, Us = Q, each pair signed so that the largest-|.|
  // entry of its Vs column is positive (lowest index on ties).  sigma at the
  // rounding level of the block (<= p u ||M||_F) counts as zero; those Vs
  // columns are left zero and the completion kernel fills them.
  cluster.sync();
  for (int sl = warp; sl < slots; sl += JC_WARPS) {
    const int c = sl * cs + rank;
    double f = 0.0;
    for (int t = lane; t < p; t += 32) f = fma(Wl[sl * p + t], Wl[sl * p + t], f);
    f = warp_sum(f);
    if (lane == 0) Nl[sl] = (c < p) ? sqrt(f) : -1.0;
  }
  cluster.sync();
  const double cut = pu * sqrt(s_fro);
  for (int sl = warp; sl < slots; sl += JC_WARPS) {
    const int c = sl * cs + rank;
    if (c >= p) continue;
    double sc = Nl[sl];
    if (sc <= cut) sc = 0.0;
    int cnt = 0;
    for (int o = lane; o < p; o += 32) {
      double so = *cluster.map_shared_rank(Nl + o / cs, o % cs);
      if (so <= cut) so = 0.0;
      cnt += (so > sc) || (so == sc && o < c);
    }
    const int r = __reduce_add_sync(0xffffffffu, cnt);
    const double* w = Wl + sl * p;
    double bv = -1.0;
    int bi = p;
    for (int t = lane; t < p; t += 32) {
      const double a = fabs(w[t]);
      if (a > bv) { bv = a; bi = t; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    const double sgn = (sc > 0.0 && w[bi] < 0.0) ? -1.0 : 1.0;
    const double inv = (sc > 0.0) ? sgn / sc : 0.0;
    double* vs = Vs + static_cast<int64_t>(r) * p;
    double* us = Us + static_cast<int64_t>(r) * p;
    const double* qc = Ql + sl * p;
    for (int t = lane; t < p; t += 32) {
      vs[t] = w[t] * inv;
      us[t] = sgn * qc[t];
    }
    if (lane == 0) {
      d[r] = sc;
      if (sc == 0.0) atomicOr(zero_flag, 1);
    }
  }
  cluster.sync();   // no CTA leaves while others may still read its shared memory
}

// The same cyclic one-sided Jacobi on the rows of M in FP32 (the FFMA pipe
// issues 64x faster than FP64 here): W = s M^T with s an exact power of two
// that brings ||M||_F near 1 (so FP32 range limits do not bite), Q = I; the
// sweeps stop at relative tolerance p 2^-24 or after max_sweeps.  The FP32
// rotations accumulate in Q, written as FP64 to Qg (p x p, ld p); the FP64
// sweeps then start from W0 = M^T Q after Q is made orthonormal in FP64.
template <int NU>
__global__ void __launch_bounds__(JC_NT)
jacobi32_cluster_kernel(int p, const double* __restrict__ M, int64_t ldm, double* __restrict__ Qg,
                        int max_sweeps) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ float jsm32[];
  const int rank = static_cast<int>(cluster.block_rank());
  const int cs = static_cast<int>(cluster.num_blocks());
  const int pp = p + (p & 1);
  const int slots = (pp + cs - 1) / cs;
  float* Wl = jsm32;
  float* Ql = jsm32 + static_cast<size_t>(slots) * p;
  float* Nl = Ql + static_cast<size_t>(slots) * p;
  __shared__ double s_part[JC_CLUSTER];
  __shared__ double s_scale;
  __shared__ int s_flag[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // ||M||_F^2 in FP64 over this CTA's rows of M, then the common scale.
  if (warp == 0) {
    double f = 0.0;
    for (int sl = 0; sl < slots; ++sl) {
      const int c = sl * cs + rank;
      if (c >= p) continue;
      for (int t = lane; t < p; t += 32) {
        const double v = M[c + static_cast<int64_t>(t) * ldm];
        f = fma(v, v, f);
      }
    }
    f = warp_sum(f);
    if (lane == 0) s_part[rank] = f;
  }
  if (tid < 2) s_flag[tid] = 0;
  cluster.sync();
  if (tid == 0) {
    double f = 0.0;
    for (int q = 0; q < cs; ++q) f += *cluster.map_shared_rank(&s_part[q], q);
    int e = 0;
    if (f > 0.0) frexp(sqrt(f), &e);
    s_scale = ldexp(1.0, -e);
  }
  __syncthreads();
  const double scale = s_scale;
  for (int sl = 0; sl < slots; ++sl) {
    const int c = sl * cs + rank;
    for (int t = tid; t < p; t += JC_NT) {
      Wl[sl * p + t] = (c < p) ? static_cast<float>(M[c + static_cast<int64_t>(t) * ldm] * scale) : 0.f;
      Ql[sl * p + t] = (c < p && t == c) ? 1.f : 0.f;
    }
  }
  __syncthreads();
  // scaled ||W||_F^2 in FP32 terms (about 1), thresholds as in the FP64 sweeps
  float fro = 0.f;
  {
    double f = 0.0;
    for (int q = 0; q < cs; ++q) f += *cluster.map_shared_rank(&s_part[q], q);
    fro = static_cast<float>(f * scale * scale);
  }
  const float pu = static_cast<float>(p) * 0x1p-24f;
  const float thr2 = pu * pu * fro;
  const float tol2 = pu * pu;
  const int npairs = pp / 2;

  bool converged = false;
  for (int sw = 0; sw < max_sweeps && !converged; ++sw) {
    for (int sl = warp; sl < slots; sl += JC_WARPS) {
      float f = 0.f;
      for (int t = lane; t < p; t += 32) f = fmaf(Wl[sl * p + t], Wl[sl * p + t], f);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
      if (lane == 0) Nl[sl] = f;
    }
    if (tid == 0) s_flag[sw & 1] = 0;
    cluster.sync();
    for (int r = 0; r < pp - 1; ++r) {
      for (int k = rank * JC_WARPS + warp; k < npairs; k += cs * JC_WARPS) {
        int i, j;
        rr_pair(pp, r, k, &i, &j);
        if (j >= p) continue;
        const int oi = i % cs, oj = j % cs, si = i / cs, sj = j / cs;
        float* wi = cluster.map_shared_rank(Wl + si * p, oi);
        float* wj = cluster.map_shared_rank(Wl + sj * p, oj);
        float* ni = cluster.map_shared_rank(Nl + si, oi);
        float* nj = cluster.map_shared_rank(Nl + sj, oj);
        float* qi = cluster.map_shared_rank(Ql + si * p, oi);
        float* qj = cluster.map_shared_rank(Ql + sj * p, oj);
        float x[NU], y[NU], q1[NU], q2[NU];
        float g = 0.f;
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          const int t = lane + 32 * u;
          x[u] = (t < p) ? wi[t] : 0.f;
          y[u] = (t < p) ? wj[t] : 0.f;
          q1[u] = (t < p) ? qi[t] : 0.f;
          q2[u] = (t < p) ? qj[t] : 0.f;
          g = fmaf(x[u], y[u], g);
        }
        const float a = *ni, b = *nj;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        if (g == 0.f || a <= thr2 || b <= thr2 || !(g * g > tol2 * a * b)) continue;
        const float zf = (b - a) / (2.0f * g);
        const float tf = (fabsf(zf) > 0x1p60f) ? 0.5f / zf
                                                : copysignf(1.0f, zf) / (fabsf(zf) + sqrtf(fmaf(zf, zf, 1.0f)));
        const float c = rsqrtf(fmaf(tf, tf, 1.0f));
        const float sn = c * tf;
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          const int t = lane + 32 * u;
          if (t < p) {
            wi[t] = fmaf(c, x[u], -sn * y[u]);
            wj[t] = fmaf(sn, x[u], c * y[u]);
            qi[t] = fmaf(c, q1[u], -sn * q2[u]);
            qj[t] = fmaf(sn, q1[u], c * q2[u]);
          }
        }
        if (lane == 0) {
          const float cc = c * c, ss = sn * sn, csg = 2.0f * c * sn * g;
          *ni = fmaf(cc, a, fmaf(ss, b, -csg));
          *nj = fmaf(ss, a, fmaf(cc, b, csg));
          s_flag[sw & 1] = 1;
        }
      }
      cluster.sync();
    }
    int any = 0;
    for (int q = 0; q < cs; ++q) any |= *cluster.map_shared_rank(&s_flag[sw & 1], q);
    converged = (any == 0);
  }
  for (int sl = 0; sl < slots; ++sl) {
    const int c = sl * cs + rank;
    if (c >= p) continue;
    for (int t = tid; t < p; t += JC_NT) Qg[t + static_cast<int64_t>(c) * p] = static_cast<double>(Ql[sl * p + t]);
  }
  cluster.sync();
}

// F = 1.5 I - 0.5 E in place: one Newton-Schulz step Q <- Q F with E = Q^T Q
// pulls Q to the nearest orthonormal matrix (error squared per step).
__global__ void polar_step_kernel(int p, double* E) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= static_cast<int64_t>(p) * p) return;
  const int i = static_cast<int>(t % p), j = static_cast<int>(t / p);
  E[t] = (i == j ? 1.5 : 0.0) - 0.5 * E[t];
}

// Basis completion for zero singular values (they sort last): the Vs
// columns of those are built by two-pass Gram-Schmidt of unit vectors
// against the others, then signed like the rest.  Runs as one CTA and
// returns at once unless the sweep kernel flagged a zero singular value.
__global__ void __launch_bounds__(256)
jacobi_complete_kernel(int p, double* __restrict__ Us, const double* __restrict__ d, double* __restrict__ Vs,
                       int* __restrict__ zero_flag) {
  __shared__ double red[8];
  __shared__ int s_need;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_need = *zero_flag;
    *zero_flag = 0;
  }
  __syncthreads();
  if (!s_need) return;
  for (int r = 0; r < p; ++r) {
    if (d[r] > 0.0) continue;
    double* u = Vs + static_cast<int64_t>(r) * p;
    for (int e = 0; e < p; ++e) {
      for (int t = tid; t < p; t += blockDim.x) u[t] = (t == e) ? 1.0 : 0.0;
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        for (int q = 0; q < r; ++q) {
          const double* uq = Vs + static_cast<int64_t>(q) * p;
          double s = 0.0;
          for (int t = tid; t < p; t += blockDim.x) s = fma(uq[t], u[t], s);
          s = warp_sum(s);
          if (lane == 0) red[warp] = s;
          __syncthreads();
          double dot = 0.0;
          for (int w = 0; w < 8; ++w) dot += red[w];
          __syncthreads();
          for (int t = tid; t < p; t += blockDim.x) u[t] -= dot * uq[t];
          __syncthreads();
        }
      }
      double s = 0.0;
      for (int t = tid; t < p; t += blockDim.x) s = fma(u[t], u[t], s);
      s = warp_sum(s);
      if (lane == 0) red[warp] = s;
      __syncthreads();
      double nrm2 = 0.0;
      for (int w = 0; w < 8; ++w) nrm2 += red[w];
      __syncthreads();
      if (nrm2 > 0.25) {
        const double inv = 1.0 / sqrt(nrm2);
        for (int t = tid; t < p; t += blockDim.x) u[t] *= inv;
        __syncthreads();
        break;
      }
    }
    // sign rule on the completed column
    if (warp == 0) {
      double bv = -1.0;
      int bi = p;
      for (int t = lane; t < p; t += 32) {
        const double a = fabs(u[t]);
        if (a > bv) { bv = a; bi = t; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (u[bi] < 0.0) {
        double* us = Us + static_cast<int64_t>(r) * p;
        for (int t = lane; t < p; t += 32) { u[t] = -u[t]; us[t] = -us[t]; }
      }
    }
    __syncthreads();
  }
}

namespace {

cudaLaunchConfig_t cluster_cfg(cudaStream_t s, int csize, size_t smem, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csize);
  cfg.blockDim = dim3(JC_NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

template <typename K>
cudaError_t prepare(K kern, int csize, size_t smem_max) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem_max));
  if (e == cudaSuccess && csize > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

template <int NU>
cudaError_t launch64(cudaStream_t s, int csize, int p, const double* M, int64_t ldm, const double* W0,
                     const double* Q0, double* Us, double* d, double* Vs, int max_sweeps, double tol, int* err,
                     int* zflag) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = prepare(jacobi_cluster_kernel<NU>, csize, kJcSmemMax);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = cluster_cfg(s, csize, jc_smem(p, csize), at);
  return cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel<NU>, p, M, ldm, W0, Q0, Us, d, Vs, max_sweeps, tol, err,
                            zflag);
}

template <int NU>
cudaError_t launch32(cudaStream_t s, int csize, int p, const double* M, int64_t ldm, double* Qg, int sweeps) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = prepare(jacobi32_cluster_kernel<NU>, csize, jc_smem32(JC_MAXP, 8));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = cluster_cfg(s, csize, jc_smem32(p, csize), at);
  return cudaLaunchKernelEx(&cfg, jacobi32_cluster_kernel<NU>, p, M, ldm, Qg, sweeps);
}

cudaError_t run64(cudaStream_t s, int csize, int p, const double* M, int64_t ldm, const double* W0, const double* Q0,
                  double* Us, double* d, double* Vs, int max_sweeps, double tol, int* err, int* zf) {
  if (p <= 32) return launch64<1>(s, csize, p, M, ldm, W0, Q0, Us, d, Vs, max_sweeps, tol, err, zf);
  if (p <= 64) return launch64<2>(s, csize, p, M, ldm, W0, Q0, Us, d, Vs, max_sweeps, tol, err, zf);
  if (p <= 128) return launch64<4>(s, csize, p, M, ldm, W0, Q0, Us, d, Vs, max_sweeps, tol, err, zf);
  return launch64<8>(s, csize, p, M, ldm, W0, Q0, Us, d, Vs, max_sweeps, tol, err, zf);
}

cudaError_t run32(cudaStream_t s, int csize, int p, const double* M, int64_t ldm, double* Qg, int sweeps) {
  if (p <= 32) return launch32<1>(s, csize, p, M, ldm, Qg, sweeps);
  if (p <= 64) return launch32<2>(s, csize, p, M, ldm, Qg, sweeps);
  if (p <= 128) return launch32<4>(s, csize, p, M, ldm, Qg, sweeps);
  return launch32<8>(s, csize, p, M, ldm, Qg, sweeps);
}

// Largest cluster size (16 with the non-portable opt-in, else 8) that can be scheduled.
int cluster_size() {
  static int csize = 0;
  if (csize) return csize;
  csize = 8;
  if (prepare(jacobi_cluster_kernel<8>, JC_CLUSTER, kJcSmemMax) == cudaSuccess) {
    cudaLaunchAttribute qa[1];
    cudaLaunchConfig_t q = cluster_cfg(nullptr, JC_CLUSTER, jc_smem(JC_MAXP, JC_CLUSTER), qa);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, jacobi_cluster_kernel<8>, &q) == cudaSuccess && nclusters > 0)
      csize = JC_CLUSTER;
  }
  cudaGetLastError();
  return csize;
}

constexpr int kPreconditionMinP = 32;   // below this the FP64 sweeps alone are cheaper
constexpr int kFp32Sweeps = 20;

}  // namespace

int64_t jacobi_work_elems(int p) { return jacobi_work_elems_for(p); }

cudaError_t jacobi_svd(cudaStream_t s, int p, const double* M, int64_t ldm, double* Us, double* d,
                       double* Vs, int max_sweeps, double* work, unsigned* bar) {
  if (p < 1) return cudaSuccess;
  if (p > JC_MAXP) return cudaErrorInvalidValue;
  const int64_t pe = static_cast<int64_t>(p) * p;
  double* W = work;        // W iterate
  double* V = W + pe;      // accumulated rotations Q
  double* X1 = V + pe;     // Q^T Q, then the Newton-Schulz factor
  double* X2 = X1 + pe;    // intermediate Q
  double* gw = X2 + pe;    // split-K partials of the p x p products (4 p^2)
  const int64_t gwe = 4 * pe;
  int* err = reinterpret_cast<int*>(bar + 2);
  int* zflag = reinterpret_cast<int*>(bar + 3);
  const int csize = cluster_size();
  const double tol = static_cast<double>(p) * 0x1p-53;
  const ProfToken tok = prof_begin(s, kProfJacobi);
  cudaError_t e;
  if (p >= kPreconditionMinP) {
    // FP32 sweeps, two FP64 Newton-Schulz steps on Q, W0 = M^T Q, FP64 sweeps
    e = run32(s, csize, p, M, ldm, V, kFp32Sweeps);
    note_launch();
    for (int it = 0; it < 2 && e == cudaSuccess; ++it) {
      double* Qin = (it == 0) ? V : X2;
      double* Qout = (it == 0) ? X2 : V;
      e = gemm_f64(s, true, false, p, p, p, 1.0, Qin, p, Qin, p, 0.0, X1, p, gw, gwe);
      if (e == cudaSuccess) {
        polar_step_kernel<<<static_cast<unsigned>((pe + 255) / 256), 256, 0, s>>>(p, X1);
        note_launch();
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = gemm_f64(s, false, false, p, p, p, 1.0, Qin, p, X1, p, 0.0, Qout, p, gw, gwe);
    }
    if (e == cudaSuccess) e = gemm_f64(s, true, false, p, p, p, 1.0, M, ldm, V, p, 0.0, W, p, gw, gwe);
    if (e == cudaSuccess) e = run64(s, csize, p, M, ldm, W, V, Us, d, Vs, max_sweeps, tol, err, zflag);
  } else {
    e = run64(s, csize, p, M, ldm, nullptr, nullptr, Us, d, Vs, max_sweeps, tol, err, zflag);
  }
  note_launch();
  if (e != cudaSuccess) return e;
  jacobi_complete_kernel<<<1, 256, 0, s>>>(p, Us, d, Vs, zflag);
  note_launch();
  // flops are iteration-dependent; record the p x p input and three p x p outputs
  prof_end(s, tok, 0.0, 8.0 * 4.0 * p * p);
  return cudaGetLastError();
}

}  // namespace rutv

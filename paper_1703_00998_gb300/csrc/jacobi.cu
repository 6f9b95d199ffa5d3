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
// times more slowly than on its rows.  Every sweep visits each of the
// p(p-1)/2 pairs once.
//
// GB300 design: FP64 runs at ~4 flop/clk/SM, so one SM would need tens of
// milliseconds for a 128 x 128 SVD.  One thread-block cluster of 16 CTAs
// (16 SMs) holds W and Q in shared memory, and the pairs are visited in a
// block-cyclic order (blocks of columns play a round-robin tournament, two
// blocks per CTA; see the block layout below): each CTA rotates the pairs of
// its two blocks in local shared memory, separated by __syncthreads, and the
// hardware cluster barrier is needed only once per round of blocks (P - 1 = 31
// per sweep instead of p - 1 = 127), when each CTA passes a block to its
// neighbour through distributed shared memory.  No global-memory round trips
// and no software grid barrier.
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

// Sweep counters (diagnostics): FP32 sweeps, FP64 sweeps, FP64 launches; added
// by CTA 0 of each launch, read and cleared by randutv_jacobi_sweeps.
__device__ unsigned long long g_jb_sweeps[3];
constexpr int JC_NT = 128;       // 4 warps per CTA, one pair per warp at a time
constexpr int JC_WARPS = JC_NT / 32;
constexpr int JC_MAXP = 256;
constexpr size_t kJcSmemLimit = 226 * 1024;   // dynamic; the static arrays need the rest of 227 KB

// Block layout.  The p columns (padded with zero columns) form P = 2 cs
// blocks of bs = ceil(p / P) consecutive columns; column c is entry c % bs of
// block c / bs.  The blocks play a round-robin tournament: P - 1 rounds, in
// each of which the cs CTAs of the cluster host P / 2 disjoint block pairs.
// CTA k hosts the players at positions k (its top seat) and P - 1 - k (its
// bottom seat); between rounds every player but the one at position 0 moves
// one position down the cycle 1, 2, ..., P - 1 (so after P - 1 rounds every
// block is home again).  Within a round a CTA rotates all bs^2 column pairs
// across its two blocks in bs sub-rounds of bs disjoint pairs, separated by
// __syncthreads only; in the first pairing round it also rotates the pairs inside each of
// its two blocks.  Every column pair meets exactly once per sweep, as in the
// plain cyclic order, but the cluster synchronises only once per round.
// Each seat holds bs columns of W and of Q (p entries each) and their
// squared norms; a seat moves to the next CTA by distributed-shared-memory
// stores into that CTA's second buffer, and the buffers swap every round.
__host__ __device__ constexpr int jb_bs(int p, int cs) { return (p + 2 * cs - 1) / (2 * cs); }
__host__ __device__ constexpr size_t jb_smem(int p, int cs, size_t real_bytes) {
  return (8ull * jb_bs(p, cs) * p + 4ull * jb_bs(p, cs)) * real_bytes;
}

__device__ __forceinline__ void rr_pair(int pp, int r, int kpair, int* a, int* b) {
  auto idx = [&](int t) { return t == 0 ? 0 : ((t - 1 + r) % (pp - 1)) + 1; };
  int x = idx(kpair), y = idx(pp - 1 - kpair);
  *a = min(x, y);
  *b = max(x, y);
}

// Home seat of block B (its place at the start of every sweep).
__device__ __forceinline__ void jb_home(int B, int cs, int* cta, int* seat) {
  if (B < cs) { *cta = B; *seat = 0; }
  else { *cta = 2 * cs - 1 - B; *seat = 1; }
}

template <typename Real>
struct JbSeats {
  Real* base;   // [buf][seat][bs][2p]: W column then Q column
  Real* nrm;    // [buf][seat][bs]
  int p, bs;
  __device__ Real* w(int buf, int seat, int i) const {
    return base + (static_cast<size_t>((buf * 2 + seat) * bs + i)) * 2 * p;
  }
  __device__ Real* q(int buf, int seat, int i) const { return w(buf, seat, i) + p; }
  __device__ Real* n(int buf, int seat, int i) const { return nrm + (buf * 2 + seat) * bs + i; }
};

// Rotation angle t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (b - a) / (2 g).
// FP64 columns: zeta from FP32 arithmetic after an exact power-of-two scaling
// of (b - a) and g into [-2, 2] (blocks at the rounding level have
// w_i . w_j ~ 1e-46, below the FP32 range), FP64 where that still fails.  The
// rotation itself is exactly orthogonal in the columns' precision
// (c = 1/sqrt(1 + t^2), s = c t), so an FP32 angle only changes how much of
// w_i . w_j a rotation removes, not the accuracy of W and Q.
__device__ __forceinline__ double jb_angle(double a, double b, double g) {
  const double dba = b - a;
  const double mx = fmax(fabs(dba), fabs(g));
  const long long ex = (__double_as_longlong(mx) >> 52) & 0x7ff;
  bool fp32_ok = ex > 0 && ex < 2046;
  float zf = 0.f;
  if (fp32_ok) {
    const double sc = __longlong_as_double(static_cast<long long>(2046 - ex) << 52);   // 2^(1023 - ex)
    const float bf = static_cast<float>(dba * sc);
    const float gf = static_cast<float>(g * sc);
    fp32_ok = fabsf(gf) >= 0x1p-100f;
    if (fp32_ok) zf = bf / (2.0f * gf);
  }
  if (fp32_ok) {
    // for |zeta| > 2^60, zeta^2 would overflow: t -> 1 / (2 zeta)
    const float tf = (fabsf(zf) > 0x1p60f) ? 0.5f / zf
                                            : copysignf(1.0f, zf) / (fabsf(zf) + sqrtf(fmaf(zf, zf, 1.0f)));
    return static_cast<double>(tf);
  }
  const double zeta = (b - a) / (2.0 * g);   // rare: outside the FP32 range
  return (fabs(zeta) > 0x1p500) ? 0.5 / zeta : copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
}

__device__ __forceinline__ float jb_angle(float a, float b, float g) {
  const float zf = (b - a) / (2.0f * g);
  return (fabsf(zf) > 0x1p60f) ? 0.5f / zf : copysignf(1.0f, zf) / (fabsf(zf) + sqrtf(fmaf(zf, zf, 1.0f)));
}

// rho^2 = g^2 / (a b) for the convergence test of a sweep (a heuristic
// maximum, so FP32 accuracy suffices): FP64 divisions run on the slow FP64
// pipe and every lane of the warp executes them, so the FP64 form scales
// g^2 and a b by the same power of two (a b into [1, 2)) and divides in FP32.
__device__ __forceinline__ float jb_ratio(double gg, double ab) {
  const long long eb = (__double_as_longlong(ab) >> 52) & 0x7ff;
  if (eb == 0 || eb >= 2046) return static_cast<float>(gg / ab);   // zero, subnormal, huge: rare
  const double sc = __longlong_as_double(static_cast<long long>(2046 - eb) << 52);   // 2^(1023 - eb)
  return __fdividef(static_cast<float>(gg * sc), static_cast<float>(ab * sc));
}
__device__ __forceinline__ float jb_ratio(float gg, float ab) { return __fdividef(gg, ab); }

__device__ __forceinline__ double jb_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float jb_rsqrt(float x) { return rsqrtf(x); }

template <typename Real>
__device__ __forceinline__ Real jb_warp_sum(Real v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One warp rotates the local column pair (wi, wj) with (qi, qj) and the
// squared norms *ni, *nj, unless the pair is already orthogonal to the
// tolerance (|w_i . w_j| <= tol ||w_i|| ||w_j||) or a column is at the
// rounding level of the block (||w||^2 <= thr2).  Each lane owns NU = ceil(p/32)
// rows; one dot product per pair: the squared norms are carried along with
// the exact norm formulas of the applied rotation (recomputed every sweep).
// Returns whether a rotation was applied (identical in all lanes).
template <typename Real, int NU>
__device__ __forceinline__ bool jb_rotate(int p, int lane, Real* wi, Real* wj, Real* qi, Real* qj, Real* ni,
                                          Real* nj, Real thr2, Real tol2, float* rho2) {
  Real x[NU], y[NU], q1[NU], q2[NU];
  Real g = 0;
#pragma unroll
  for (int u = 0; u < NU; ++u) {
    const int t = lane + 32 * u;
    x[u] = (t < p) ? wi[t] : Real(0);
    y[u] = (t < p) ? wj[t] : Real(0);
    q1[u] = (t < p) ? qi[t] : Real(0);
    q2[u] = (t < p) ? qj[t] : Real(0);
    g = fma(x[u], y[u], g);
  }
  const Real a = *ni, b = *nj;
  g = jb_warp_sum(g);   // identical in every lane
  const Real gg = g * g, ab = a * b;
  const bool live = a > thr2 && b > thr2;
  if (live) *rho2 = fmaxf(*rho2, jb_ratio(gg, ab));   // the sweep's largest g^2 / (a b)
  if (g == Real(0) || !live || !(gg > tol2 * ab)) return false;
  const Real tt = jb_angle(a, b, g);
  const Real c = jb_rsqrt(fma(tt, tt, Real(1)));
  const Real sn = c * tt;
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
  __syncwarp();
  if (lane == 0) {
    const Real cc = c * c, ss = sn * sn, csg = Real(2) * c * sn * g;
    *ni = fma(cc, a, fma(ss, b, -csg));
    *nj = fma(ss, a, fma(cc, b, csg));
  }
  return true;
}

// The sweeps of the block-cyclic order on the seats of this CTA (buffer
// *cur at entry and exit).  Returns whether the last sweep converged (the
// same in every CTA).  Converged: a sweep applied no rotation (every pair
// already orthogonal to the tolerance), or, with early_stop (the FP32
// stage, which the FP64 sweeps refine anyway), the largest relative
// off-diagonal rho = |w_i . w_j| / (||w_i|| ||w_j||) the sweep met
// satisfies rho^2 <= tol / 10, so that the next sweep would meet about
// rho^2 and rotate little.  The FP64 stage does not stop early: its last
// rotations' rho' ~ rho^2 / gap is above the tolerance where singular values
// cluster (relative gaps ~ 1e-2..1e-3), and it would leave Vs about
// 1e-13 from orthogonal.
template <typename Real, int NU>
__device__ bool jb_sweeps(const JbSeats<Real>& S, int* cur_io, int p, int cs, int rank, int max_sweeps, Real thr2,
                          Real tol2, int* s_flag, int* sweeps_done, bool early_stop) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bs = S.bs, P = 2 * cs;
  const int bsp = bs + (bs & 1);
  int cur = *cur_io;
  bool converged = false;
  int sw = 0;
  for (; sw < max_sweeps && !converged; ++sw) {
    // exact squared norms of this CTA's columns at the start of the sweep
    for (int e = warp; e < 2 * bs; e += JC_WARPS) {
      const Real* w = S.w(cur, e / bs, e % bs);
      Real f = 0;
      for (int t = lane; t < p; t += 32) f = fma(w[t], w[t], f);
      f = jb_warp_sum(f);
      if (lane == 0) *S.n(cur, e / bs, e % bs) = f;
    }
    if (tid == 0) { s_flag[sw & 1] = 0; s_flag[2 + (sw & 1)] = 0; }
    bool rotated = false;
    float rho2 = 0.0f;
    __syncthreads();
    for (int r = 0; r < P - 1; ++r) {
      if (r == 0 && bs > 1) {
        // pairs inside each of the two blocks: bsp - 1 sub-rounds
        for (int sub = 0; sub < bsp - 1; ++sub) {
          for (int kk = warp; kk < bsp; kk += JC_WARPS) {
            const int seat = kk / (bsp / 2), kp = kk % (bsp / 2);
            int a, b;
            rr_pair(bsp, sub, kp, &a, &b);
            if (b >= bs) continue;
            rotated |= jb_rotate<Real, NU>(p, lane, S.w(cur, seat, a), S.w(cur, seat, b), S.q(cur, seat, a),
                                           S.q(cur, seat, b), S.n(cur, seat, a), S.n(cur, seat, b), thr2, tol2,
                                           &rho2);
          }
          __syncthreads();
        }
      }
      // pairs across the two blocks: bs sub-rounds of bs disjoint pairs
      for (int sub = 0; sub < bs; ++sub) {
        for (int i = warp; i < bs; i += JC_WARPS) {
          const int j = (i + sub) % bs;
          rotated |= jb_rotate<Real, NU>(p, lane, S.w(cur, 0, i), S.w(cur, 1, j), S.q(cur, 0, i), S.q(cur, 1, j),
                                         S.n(cur, 0, i), S.n(cur, 1, j), thr2, tol2, &rho2);
        }
        __syncthreads();
      }
      // move the seats (top: k -> k-1, k = 1 -> bottom of 0, k = 0 stays;
      // bottom: k -> k+1, k = cs-1 -> its own top) into the other buffer
      const int nx = cur ^ 1;
      int dt_cta, dt_seat, db_cta, db_seat;
      if (rank == 0) { dt_cta = 0; dt_seat = 0; }
      else if (rank == 1) { dt_cta = 0; dt_seat = 1; }
      else { dt_cta = rank - 1; dt_seat = 0; }
      if (rank < cs - 1) { db_cta = rank + 1; db_seat = 1; }
      else { db_cta = rank; db_seat = 0; }
      Real* dt = cluster.map_shared_rank(S.w(nx, dt_seat, 0), dt_cta);
      Real* db = cluster.map_shared_rank(S.w(nx, db_seat, 0), db_cta);
      Real* dtn = cluster.map_shared_rank(S.n(nx, dt_seat, 0), dt_cta);
      Real* dbn = cluster.map_shared_rank(S.n(nx, db_seat, 0), db_cta);
      const Real* st = S.w(cur, 0, 0);
      const Real* sb = S.w(cur, 1, 0);
      const int len = bs * 2 * p;
      for (int e = tid; e < len; e += JC_NT) {
        dt[e] = st[e];
        db[e] = sb[e];
      }
      if (tid < bs) {
        dtn[tid] = *S.n(cur, 0, tid);
        dbn[tid] = *S.n(cur, 1, tid);
      }
      cur = nx;
      cluster.sync();
    }
    // a sweep without rotations anywhere in the cluster, or one whose largest relative
    // off-diagonal already puts the next sweep below the tolerance: converged
    if (rotated) s_flag[sw & 1] = 1;   // benign race: every writer stores 1
    if (lane == 0 && rho2 > 0.0f) atomicMax(&s_flag[2 + (sw & 1)], __float_as_int(rho2));   // non-negative floats
    cluster.sync();
    int any = 0;
    float rmax = 0.0f;
    for (int q = 0; q < cs; ++q) {
      any |= *cluster.map_shared_rank(&s_flag[sw & 1], q);
      rmax = fmaxf(rmax, __int_as_float(*cluster.map_shared_rank(&s_flag[2 + (sw & 1)], q)));
    }
    const float tol = sqrtf(static_cast<float>(tol2));
    converged = (any == 0) || (early_stop && rmax <= 0.1f * tol);
  }
  *cur_io = cur;
  *sweeps_done = sw;
  return converged;
}

// FP64 sweeps, then the epilogue on the 16 SMs: sigma_c = ||w_c||, the order
// (descending, stable in c), Vs = w / sigma, Us = Q, each pair signed so
// that the largest-|.| entry of its Vs column is positive (lowest index on
// ties).  sigma at the rounding level of the block (<= p u ||M||_F) counts as
// zero; those Vs columns are left zero and the completion kernel fills them.
// Start: W(:, c) = M(c, :)^T and Q = I, or W0 = M^T Q0 (p x p, ld p) after
// the FP32 sweeps.
template <int NU>
__global__ void __launch_bounds__(JC_NT, 1)
jacobi_block64_kernel(int p, const double* __restrict__ M, int64_t ldm, const double* W0, const double* Q0,
                      double* __restrict__ Us, double* __restrict__ d, double* __restrict__ Vs, int max_sweeps,
                      double tol, int* __restrict__ err, int* __restrict__ zero_flag) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double jsm[];
  const int rank = static_cast<int>(cluster.block_rank());
  const int cs = static_cast<int>(cluster.num_blocks());
  const int bs = jb_bs(p, cs);
  JbSeats<double> S{jsm, jsm + 8ull * bs * p, p, bs};
  __shared__ double s_part[JC_CLUSTER];
  __shared__ double s_fro;
  __shared__ int s_flag[4];   // per sweep parity: rotated, largest rho^2 (float bits)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // this CTA's two home blocks: rank (top) and 2 cs - 1 - rank (bottom)
  for (int seat = 0; seat < 2; ++seat) {
    const int B = seat == 0 ? rank : 2 * cs - 1 - rank;
    for (int i = 0; i < bs; ++i) {
      const int c = B * bs + i;
      double* w = S.w(0, seat, i);
      double* q = S.q(0, seat, i);
      for (int t = tid; t < p; t += JC_NT) {
        if (c >= p) { w[t] = 0.0; q[t] = 0.0; }
        else if (W0) { w[t] = W0[t + static_cast<int64_t>(c) * p]; q[t] = Q0[t + static_cast<int64_t>(c) * p]; }
        else { w[t] = M[c + static_cast<int64_t>(t) * ldm]; q[t] = (t == c) ? 1.0 : 0.0; }
      }
    }
  }
  __syncthreads();
  // ||M||_F^2, summed in the same order by every CTA
  if (warp == 0) {
    double f = 0.0;
    for (int e = 0; e < 2 * bs; ++e) {
      const double* w = S.w(0, e / bs, e % bs);
      for (int t = lane; t < p; t += 32) f = fma(w[t], w[t], f);
    }
    f = warp_sum(f);
    if (lane == 0) s_part[rank] = f;
  }
  if (tid < 4) s_flag[tid] = 0;
  cluster.sync();
  if (tid == 0) {
    double f = 0.0;
    for (int q = 0; q < cs; ++q) f += *cluster.map_shared_rank(&s_part[q], q);
    s_fro = f;
  }
  __syncthreads();
  // columns with ||w|| <= p u ||M||_F are at the rounding level of the block
  // and count as zero (rotating them only stirs rounding noise)
  const double pu = static_cast<double>(p) * 0x1p-53;
  const double thr2 = pu * pu * s_fro;
  int cur = 0;
  int nsw = 0;
  const bool converged = jb_sweeps<double, NU>(S, &cur, p, cs, rank, max_sweeps, thr2, tol * tol, s_flag, &nsw, false);
  if (!converged && rank == 0 && tid == 0) atomicOr(err, kDevErrNoConv);
  if (rank == 0 && tid == 0) {
    atomicAdd(&g_jb_sweeps[1], static_cast<unsigned long long>(nsw));
    atomicAdd(&g_jb_sweeps[2], 1ull);
  }

  // every block is at its home seat again (buffer cur): exact norms
  for (int e = warp; e < 2 * bs; e += JC_WARPS) {
    const int seat = e / bs, i = e % bs;
    const int c = (seat == 0 ? rank : 2 * cs - 1 - rank) * bs + i;
    const double* w = S.w(cur, seat, i);
    double f = 0.0;
    for (int t = lane; t < p; t += 32) f = fma(w[t], w[t], f);
    f = warp_sum(f);
    if (lane == 0) *S.n(cur, seat, i) = (c < p) ? sqrt(f) : -1.0;
  }
  cluster.sync();
  const double cut = pu * sqrt(s_fro);
  for (int e = warp; e < 2 * bs; e += JC_WARPS) {
    const int seat = e / bs, i = e % bs;
    const int c = (seat == 0 ? rank : 2 * cs - 1 - rank) * bs + i;
    if (c >= p) continue;
    double sc = *S.n(cur, seat, i);
    if (sc <= cut) sc = 0.0;
    int cnt = 0;
    for (int o = lane; o < p; o += 32) {
      int oc, os;
      jb_home(o / bs, cs, &oc, &os);
      double so = *cluster.map_shared_rank(S.n(cur, os, o % bs), oc);
      if (so <= cut) so = 0.0;
      cnt += (so > sc) || (so == sc && o < c);
    }
    const int r = __reduce_add_sync(0xffffffffu, cnt);
    const double* w = S.w(cur, seat, i);
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
    const double* qc = S.q(cur, seat, i);
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

// The same block-cyclic one-sided Jacobi on the rows of M in FP32 (the FFMA
// pipe issues 64x faster than FP64 here): W = s M^T with s an exact power of
// two that brings ||M||_F near 1 (so FP32 range limits do not bite), Q = I;
// the sweeps stop at relative tolerance p 2^-24 or after max_sweeps.  The
// FP32 rotations accumulate in Q, written as FP64 to Qg (p x p, ld p); the
// FP64 sweeps then start from W0 = M^T Q after Q is made orthonormal in FP64.
template <int NU>
__global__ void __launch_bounds__(JC_NT, 1)
jacobi_block32_kernel(int p, const double* __restrict__ M, int64_t ldm, double* __restrict__ Qg, int max_sweeps) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ float jsm32[];
  const int rank = static_cast<int>(cluster.block_rank());
  const int cs = static_cast<int>(cluster.num_blocks());
  const int bs = jb_bs(p, cs);
  JbSeats<float> S{jsm32, jsm32 + 8ull * bs * p, p, bs};
  __shared__ double s_part[JC_CLUSTER];
  __shared__ double s_scale;
  __shared__ int s_flag[4];   // per sweep parity: rotated, largest rho^2 (float bits)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // ||M||_F^2 in FP64 over this CTA's rows of M, then the common scale
  if (warp == 0) {
    double f = 0.0;
    for (int e = 0; e < 2 * bs; ++e) {
      const int c = (e < bs ? rank : 2 * cs - 1 - rank) * bs + e % bs;
      if (c >= p) continue;
      for (int t = lane; t < p; t += 32) {
        const double v = M[c + static_cast<int64_t>(t) * ldm];
        f = fma(v, v, f);
      }
    }
    f = warp_sum(f);
    if (lane == 0) s_part[rank] = f;
  }
  if (tid < 4) s_flag[tid] = 0;
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
  for (int seat = 0; seat < 2; ++seat) {
    const int B = seat == 0 ? rank : 2 * cs - 1 - rank;
    for (int i = 0; i < bs; ++i) {
      const int c = B * bs + i;
      float* w = S.w(0, seat, i);
      float* q = S.q(0, seat, i);
      for (int t = tid; t < p; t += JC_NT) {
        w[t] = (c < p) ? static_cast<float>(M[c + static_cast<int64_t>(t) * ldm] * scale) : 0.f;
        q[t] = (c < p && t == c) ? 1.f : 0.f;
      }
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
  int cur = 0;
  int nsw = 0;
  jb_sweeps<float, NU>(S, &cur, p, cs, rank, max_sweeps, pu * pu * fro, pu * pu, s_flag, &nsw, true);
  if (rank == 0 && tid == 0) atomicAdd(&g_jb_sweeps[0], static_cast<unsigned long long>(nsw));
  for (int seat = 0; seat < 2; ++seat) {
    const int B = seat == 0 ? rank : 2 * cs - 1 - rank;
    for (int i = 0; i < bs; ++i) {
      const int c = B * bs + i;
      if (c >= p) continue;
      const float* q = S.q(cur, seat, i);
      for (int t = tid; t < p; t += JC_NT) Qg[t + static_cast<int64_t>(c) * p] = static_cast<double>(q[t]);
    }
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
  static PerDeviceOnce once;
  cudaError_t e = per_device_once(once, [&] { return prepare(jacobi_block64_kernel<NU>, csize, kJcSmemLimit); });
  if (e != cudaSuccess) return e;
  const size_t smem = jb_smem(p, csize, sizeof(double));
  if (smem > kJcSmemLimit) return cudaErrorInvalidConfiguration;   // p > 240 needs the 16-CTA cluster
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = cluster_cfg(s, csize, smem, at);
  return cudaLaunchKernelEx(&cfg, jacobi_block64_kernel<NU>, p, M, ldm, W0, Q0, Us, d, Vs, max_sweeps, tol, err,
                            zflag);
}

template <int NU>
cudaError_t launch32(cudaStream_t s, int csize, int p, const double* M, int64_t ldm, double* Qg, int sweeps) {
  static PerDeviceOnce once;
  cudaError_t e = per_device_once(once, [&] { return prepare(jacobi_block32_kernel<NU>, csize, kJcSmemLimit); });
  if (e != cudaSuccess) return e;
  const size_t smem = jb_smem(p, csize, sizeof(float));
  if (smem > kJcSmemLimit) return cudaErrorInvalidConfiguration;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = cluster_cfg(s, csize, smem, at);
  return cudaLaunchKernelEx(&cfg, jacobi_block32_kernel<NU>, p, M, ldm, Qg, sweeps);
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
// Cached per device (the query depends on the device's limits).
int cluster_size() {
  static std::mutex mu;
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    dev = -1;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && cached[dev]) return cached[dev];
  int csize = 8;
  if (prepare(jacobi_block64_kernel<8>, JC_CLUSTER, kJcSmemLimit) == cudaSuccess) {
    cudaLaunchAttribute qa[1];
    cudaLaunchConfig_t q = cluster_cfg(nullptr, JC_CLUSTER, jb_smem(JC_MAXP, JC_CLUSTER, sizeof(double)), qa);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, jacobi_block64_kernel<8>, &q) == cudaSuccess && nclusters > 0)
      csize = JC_CLUSTER;
  }
  cudaGetLastError();
  if (dev >= 0) cached[dev] = csize;
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

cudaError_t jacobi_sweep_counts(unsigned long long out[3], bool reset) {
  cudaError_t e = cudaMemcpyFromSymbol(out, g_jb_sweeps, sizeof(unsigned long long) * 3);
  if (e == cudaSuccess && reset) {
    const unsigned long long z[3] = {0, 0, 0};
    e = cudaMemcpyToSymbol(g_jb_sweeps, z, sizeof(z));
  }
  return e;
}

}  // namespace rutv

extern "C" int randutv_jacobi_sweeps(int64_t* fp32_sweeps, int64_t* fp64_sweeps, int64_t* svds, int reset) {
  unsigned long long c[3] = {0, 0, 0};
  if (rutv::jacobi_sweep_counts(c, reset != 0) != cudaSuccess) {
    cudaGetLastError();
    return RANDUTV_ECUDA;
  }
  if (fp32_sweeps) *fp32_sweeps = static_cast<int64_t>(c[0]);
  if (fp64_sweeps) *fp64_sweeps = static_cast<int64_t>(c[1]);
  if (svds) *svds = static_cast<int64_t>(c[2]);
  return RANDUTV_OK;
}

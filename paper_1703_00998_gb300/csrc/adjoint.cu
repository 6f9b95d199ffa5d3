// The rank-k approximation of randUTV, A_k = U(:, 1:k) T(1:k, :) V^T
// (eq. Ak_randUTV, k a multiple of b), and its vector-Jacobian product at
// fixed Gaussian matrices, FP64.
//
// The first k/b randomized steps of Fig. 4 fix U(:, 1:k), and A = U T V^T
// holds after every step, so A_k = U_k U_k^T A; the small SVDs rotate only
// inside the finished blocks and leave span(U_k), the trailing block and
// the trailing bases unchanged, so the map is that of the steps without
// them: per step the sketch Y = (X^T X)^q X^T G, the Householder QR of Y and
// its application to T(:, J2 J3), the Householder QR of the panel and its
// application to U(:, I2 I3) and T(I2 I3, J2 J3).
//
// The reverse pass is written by hand: for F = U_k W, W = U_k^T A,
//   Abar = U_k U_k^T Fbar + Tbar_0,  Ubar_k = Fbar W^T + A Fbar^T U_k,
// then step by step backwards through the two block-reflector applications
// (Q = I - V S V^T: Cbar <- Cbar Q^T or Q Cbar, and the products Qbar V,
// Qbar^T V formed from thin factors; each step's Gaussian, sketches,
// reflectors and WY factors are kept from the forward pass, O((m + n) b)
// per step, and T and U entering each step, and T between its two
// applications, are walked back from the final T and U with those
// reflectors when the reverse pass reaches the step, instead of being
// stored), the compact-WY factor (S^-1 =
// striu(V^T V) + diag(1/tau): Sbar = triu(-V^T Qbar V), Mbar = triu(-S^T
// Sbar S^T), Vbar += V (N + N^T) with N = striu(Mbar), taubar = -diag(Mbar)
// / tau^2), the Householder QR reflector by reflector (the intermediate
// panels recomputed backwards from [R; 0] with the involutions H_j, the
// dlarfg derivative per column) and the sketch's products.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>
#include "common.cuh"
#include "internal.h"

namespace rutv {
namespace {

constexpr int AD_MAXW = 32;     // block size limit of the reverse kernels
constexpr int HR_NT = 256;      // threads of the QR reverse kernel
constexpr int HR_NW = HR_NT / 32;

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reverse of the Householder QR of an L x w panel (w <= 32), one CTA.
// In: the explicit reflectors V (L x w, ld L, unit lower trapezoidal), tau,
// R (w x w, ld ldr), the cotangents Vbar (L x w, ld L; only the entries
// below the diagonal are read; overwritten as scratch) and taubar (w).
// Out: Pbar (L x w, ld L), the cotangent of the panel.  P (L x w, ld L) is
// scratch for the intermediate panels.  Each thread owns rows tid + k HR_NT.
__global__ void __launch_bounds__(HR_NT) hqr_reverse_kernel(int L, int w, const double* __restrict__ V,
                                                            const double* __restrict__ tau,
                                                            const double* __restrict__ R, int ldr, double* Vbar,
                                                            const double* __restrict__ taubar, double* P,
                                                            double* Pbar) {
  __shared__ double red[HR_NW][2 * AD_MAXW + 2];
  __shared__ double vec[2 * AD_MAXW + 2];
  __shared__ double sred[HR_NW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the panel after all reflectors is [R; 0]; its cotangent is zero
  for (int64_t e = tid; e < static_cast<int64_t>(L) * w; e += HR_NT) {
    const int r = static_cast<int>(e % L), c = static_cast<int>(e / L);
    P[e] = (r <= c && r < w) ? R[r + static_cast<int64_t>(c) * ldr] : 0.0;
    Pbar[e] = 0.0;
  }
  __syncthreads();
  for (int j = w - 1; j >= 0; --j) {
    const double t = tau[j], beta = R[j + static_cast<int64_t>(j) * ldr];
    const double* vj = V + static_cast<int64_t>(j) * L;
    // pass 1: v^T P(:, c), v^T Pbar(:, c) for c > j and v^T v over rows >= j
    double wn[AD_MAXW], db[AD_MAXW], vv = 0.0;
#pragma unroll
    for (int c = 0; c < AD_MAXW; ++c) wn[c] = db[c] = 0.0;
    for (int r = j + tid; r < L; r += HR_NT) {
      const double v = (r == j) ? 1.0 : vj[r];
      vv = fma(v, v, vv);
#pragma unroll
      for (int c = 0; c < AD_MAXW; ++c) {
        if (c > j && c < w) {
          wn[c] = fma(v, P[r + static_cast<int64_t>(c) * L], wn[c]);
          db[c] = fma(v, Pbar[r + static_cast<int64_t>(c) * L], db[c]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < AD_MAXW; ++c) {
      if (c > j && c < w) {
        const double a = wsum(wn[c]), d = wsum(db[c]);
        if (lane == 0) {
          red[warp][c] = a;
          red[warp][AD_MAXW + c] = d;
        }
      }
    }
    vv = wsum(vv);
    if (lane == 0) red[warp][2 * AD_MAXW] = vv;
    __syncthreads();
    if (tid < 2 * AD_MAXW + 1) {
      const int c = tid < 2 * AD_MAXW ? tid % AD_MAXW : 0;
      double s = 0.0;
      if (tid == 2 * AD_MAXW || (c > j && c < w))
        for (int i = 0; i < HR_NW; ++i) s += red[i][tid];
      vec[tid] = s;
    }
    __syncthreads();
    const double* swn = vec;
    const double* sdb = vec + AD_MAXW;
    const double svv = vec[2 * AD_MAXW];
    // w_c = v^T P_c before H_j = v^T P_c after it times (1 - tau v^T v)
    double tb = taubar[j];
    for (int c = j + 1; c < w; ++c) tb -= sdb[c] * swn[c] * (1.0 - t * svv);
    // pass 2: the panel before H_j and the cotangents of columns c > j and of v
    double gpart = 0.0;
    for (int r = j + tid; r < L; r += HR_NT) {
      const double v = (r == j) ? 1.0 : vj[r];
      double sa = 0.0, sb = 0.0;
      for (int c = j + 1; c < w; ++c) {
        const int64_t o = r + static_cast<int64_t>(c) * L;
        const double wc = swn[c] * (1.0 - t * svv);
        const double cn = P[o], cbn = Pbar[o];
        const double cc = cn - t * v * swn[c];
        sa = fma(cbn, wc, sa);
        sb = fma(cc, sdb[c], sb);
        P[o] = cc;
        Pbar[o] = cbn - t * v * sdb[c];
      }
      if (r > j) {
        const double vb = Vbar[r + static_cast<int64_t>(j) * L] - t * (sa + sb);
        Vbar[r + static_cast<int64_t>(j) * L] = vb;
        gpart = fma(vb, -t * beta * v, gpart);      // vb_r x_r with x_r = -tau beta v_r
      }
    }
    gpart = wsum(gpart);
    if (lane == 0) sred[warp] = gpart;
    __syncthreads();
    double gsum = 0.0;
    for (int i = 0; i < HR_NW; ++i) gsum += sred[i];
    // dlarfg derivative: x = beta (e_0 - tau v), alpha = beta (1 - tau)
    const double alpha = beta * (1.0 - t);
    const double nu = fabs(beta), sg = copysign(1.0, alpha);
    double ab = 0.0, nub = 0.0, inv_ab = 0.0;
    if (t != 0.0) {
      inv_ab = 1.0 / (alpha - beta);
      const double g = -gsum * inv_ab * inv_ab;
      const double bb = -g + tb * alpha / (beta * beta);
      nub = -sg * bb;
      ab = g - tb / beta + nub * alpha / nu;
    }
    for (int r = j + tid; r < L; r += HR_NT) {
      const int64_t o = r + static_cast<int64_t>(j) * L;
      if (r == j) {
        Pbar[o] = ab;
        P[o] = alpha;
      } else {
        const double x = -t * beta * vj[r];
        Pbar[o] = (t != 0.0) ? Vbar[o] * inv_ab + nub * x / nu : 0.0;
        P[o] = x;
      }
    }
    __syncthreads();
  }
}

// The same reverse over a cooperative grid: CTA b owns rows [b rpb, (b+1)
// rpb) of the panel (rpb a multiple of 32; lane = row within each group of
// 32, warp = a group of columns), so the FP64 work of a reflector is spread
// over many SMs (one SM issues ~4 FP64 flop per clock here).  Each reflector
// needs two sums over all rows: the products v^T P(:, c), v^T Pbar(:, c),
// v^T v (pass 1) and the dlarfg cotangent's v^T Vbar part (pass 2); each CTA
// adds its partial sums into `acc` (w x HG_ACC, zeroed by the host) with
// FP64 atomics, and one bounded grid barrier follows each.  Scalar FP64
// work (taubar's correction, the dlarfg derivative) runs in one thread and
// is broadcast through shared memory.
constexpr int HG_NT = 256;
constexpr int HG_NW = HG_NT / 32;
constexpr int HG_ACC = 2 * AD_MAXW + 2;   // per reflector: v^T P, v^T Pbar (w each), v^T v, the Vbar sum
constexpr int HG_MAX_RPB = 256;

__global__ void __launch_bounds__(HG_NT, 1)
hqr_reverse_grid_kernel(int L, int w, const double* __restrict__ V, const double* __restrict__ tau,
                        const double* __restrict__ R, int ldr, double* Vbar, const double* __restrict__ taubar,
                        double* P, double* Pbar, double* acc, GridBarrier gb, int rpb) {
  __shared__ double s_wn[AD_MAXW], s_db[AD_MAXW], s_wc[AD_MAXW];
  __shared__ double s_sc[8];
  __shared__ double red[HG_NW][HG_MAX_RPB];
  __shared__ double s_part[HG_NW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = gridDim.x;
  const int r_lo = blockIdx.x * rpb;
  const int nr = max(0, min(L, r_lo + rpb) - r_lo);
  // the panel after all reflectors is [R; 0]; its cotangent is zero
  for (int e = tid; e < nr * w; e += HG_NT) {
    const int r = r_lo + e % nr, c = e / nr;
    const int64_t o = r + static_cast<int64_t>(c) * L;
    P[o] = (r <= c && r < w) ? R[r + static_cast<int64_t>(c) * ldr] : 0.0;
    Pbar[o] = 0.0;
  }
  __syncthreads();
  for (int j = w - 1; j >= 0; --j) {
    const double t = tau[j], beta = R[j + static_cast<int64_t>(j) * ldr];
    const double* vj = V + static_cast<int64_t>(j) * L;
    double* aj = acc + static_cast<int64_t>(j) * HG_ACC;
    const bool has = r_lo + nr > j;   // this CTA holds rows >= j
    // pass 1: partial v^T P(:, c), v^T Pbar(:, c) (c > j) and v^T v over rows >= j
    if (has) {
      for (int c = j + 1 + warp; c < w; c += HG_NW) {
        double s1 = 0.0, s2 = 0.0;
        for (int rl = lane; rl < nr; rl += 32) {
          const int r = r_lo + rl;
          if (r < j) continue;
          const double v = (r == j) ? 1.0 : vj[r];
          const int64_t o = r + static_cast<int64_t>(c) * L;
          s1 = fma(v, P[o], s1);
          s2 = fma(v, Pbar[o], s2);
        }
        s1 = wsum(s1);
        s2 = wsum(s2);
        if (lane == 0) {
          atomicAdd(aj + c, s1);
          atomicAdd(aj + AD_MAXW + c, s2);
        }
      }
      if (warp == HG_NW - 1) {
        double vv = 0.0;
        for (int rl = lane; rl < nr; rl += 32) {
          const int r = r_lo + rl;
          if (r < j) continue;
          const double v = (r == j) ? 1.0 : vj[r];
          vv = fma(v, v, vv);
        }
        vv = wsum(vv);
        if (lane == 0) atomicAdd(aj + 2 * AD_MAXW, vv);
      }
    }
    if (!grid_barrier(gb, nb)) return;
    if (tid > j && tid < w) {
      s_wn[tid] = __ldcg(aj + tid);
      s_db[tid] = __ldcg(aj + AD_MAXW + tid);
    }
    if (tid == 0) s_sc[0] = __ldcg(aj + 2 * AD_MAXW);
    __syncthreads();
    // w_c = v^T P_c before H_j = v^T P_c after it times (1 - tau v^T v);
    // taubar_j - sum_c db_c w_c by one warp (a chain of FP64 steps in one
    // thread would cost 64 cycles of the FP64 pipe per step)
    if (tid > j && tid < w) s_wc[tid] = s_wn[tid] * (1.0 - t * s_sc[0]);
    if (warp == 0) {
      const double one = 1.0 - t * s_sc[0];
      double d = (lane > j && lane < w) ? s_db[lane] * s_wn[lane] * one : 0.0;
      d = wsum(d);
      if (lane == 0) s_sc[1] = taubar[j] - d;
    }
    __syncthreads();
    // pass 2: the panel before H_j (columns c > j) and its cotangent; each
    // thread's part of sum_c (Pbar w_c + P_c db_c) per row into red
    for (int rl = lane; rl < nr; rl += 32) {
      const int r = r_lo + rl;
      double sab = 0.0;
      if (r >= j) {
        const double v = (r == j) ? 1.0 : vj[r];
        for (int c = j + 1 + warp; c < w; c += HG_NW) {
          const int64_t o = r + static_cast<int64_t>(c) * L;
          const double cn = P[o], cbn = Pbar[o];
          const double cc = cn - t * v * s_wn[c];
          sab = fma(cbn, s_wc[c], sab);
          sab = fma(cc, s_db[c], sab);
          P[o] = cc;
          Pbar[o] = cbn - t * v * s_db[c];
        }
      }
      red[warp][rl] = sab;
    }
    __syncthreads();
    double gp = 0.0;
    for (int rl = tid; rl < nr; rl += HG_NT) {
      const int r = r_lo + rl;
      if (r > j) {
        double sab = 0.0;
#pragma unroll
        for (int g = 0; g < HG_NW; ++g) sab += red[g][rl];
        const int64_t o = r + static_cast<int64_t>(j) * L;
        const double vb = Vbar[o] - t * sab;
        Vbar[o] = vb;
        gp = fma(vb, -t * beta * vj[r], gp);      // vb_r x_r with x_r = -tau beta v_r
      }
    }
    gp = wsum(gp);
    if (lane == 0) s_part[warp] = gp;
    __syncthreads();
    if (tid == 0 && has) {
      double g = 0.0;
      for (int i = 0; i < HG_NW; ++i) g += s_part[i];
      atomicAdd(aj + 2 * AD_MAXW + 1, g);
    }
    if (!grid_barrier(gb, nb)) return;
    // dlarfg derivative: x = beta (e_0 - tau v), alpha = beta (1 - tau)
    if (tid == 0) {
      const double gsum = __ldcg(aj + 2 * AD_MAXW + 1);
      const double tb = s_sc[1];
      const double alpha = beta * (1.0 - t);
      const double nu = fabs(beta), sg = copysign(1.0, alpha);
      double ab = 0.0, nub = 0.0, inv_ab = 0.0;
      if (t != 0.0) {
        inv_ab = 1.0 / (alpha - beta);
        const double gg = -gsum * inv_ab * inv_ab;
        const double bb = -gg + tb * alpha / (beta * beta);
        nub = -sg * bb;
        ab = gg - tb / beta + nub * alpha / nu;
      }
      s_sc[2] = ab;
      s_sc[3] = inv_ab;
      s_sc[4] = (t != 0.0) ? nub / nu : 0.0;
      s_sc[5] = alpha;
    }
    __syncthreads();
    for (int rl = tid; rl < nr; rl += HG_NT) {
      const int r = r_lo + rl;
      if (r < j) continue;
      const int64_t o = r + static_cast<int64_t>(j) * L;
      if (r == j) {
        Pbar[o] = s_sc[2];
        P[o] = s_sc[5];
      } else {
        const double x = -t * beta * vj[r];
        Pbar[o] = (t != 0.0) ? Vbar[o] * s_sc[3] + s_sc[4] * x : 0.0;
        P[o] = x;
      }
    }
    __syncthreads();
  }
}

// b x b part of the compact-WY adjoint (one CTA of 32 x 32 threads): from
// VtQV = V^T Qbar V, S and tau, Nsym = N + N^T with N = striu(Mbar), Mbar =
// triu(-S^T Sbar S^T), Sbar = triu(-VtQV), and taubar = -diag(Mbar) / tau^2.
__global__ void __launch_bounds__(1024) wy_small_adjoint_kernel(int w, const double* __restrict__ VtQV,
                                                                const double* __restrict__ S,
                                                                const double* __restrict__ tau, double* Nsym,
                                                                double* taubar) {
  __shared__ double sS[AD_MAXW][AD_MAXW + 1], sB[AD_MAXW][AD_MAXW + 1], sX[AD_MAXW][AD_MAXW + 1];
  const int i = threadIdx.x % AD_MAXW, j = threadIdx.x / AD_MAXW;
  const bool in = i < w && j < w;
  sS[i][j] = in ? S[i + j * w] : 0.0;
  sB[i][j] = (in && i <= j) ? -VtQV[i + j * w] : 0.0;
  __syncthreads();
  double x = 0.0;
  for (int l = 0; l < w; ++l) x = fma(sS[l][i], sB[l][j], x);     // (S^T Sbar)(i, j)
  sX[i][j] = x;
  __syncthreads();
  double mb = 0.0;
  if (in && i <= j)
    for (int l = 0; l < w; ++l) mb -= sX[i][l] * sS[j][l];         // -(S^T Sbar S^T)(i, j)
  sB[i][j] = mb;
  __syncthreads();
  if (in) {
    Nsym[i + j * w] = (i < j ? sB[i][j] : 0.0) + (j < i ? sB[j][i] : 0.0);
    if (i == j) taubar[i] = -sB[i][i] / (tau[i] * tau[i]);
  }
}

// Y (m x n, ld ldy) += X (m x n, ld ldx)
__global__ void add_kernel(int64_t m, int64_t n, const double* __restrict__ X, int64_t ldx, double* Y, int64_t ldy) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= m * n) return;
  const int64_t r = t % m, c = t / m;
  Y[r + c * ldy] += X[r + c * ldx];
}

}  // namespace
}  // namespace rutv

// ---------------------------------------------------------------------------
// Host side.

struct randutv_rank_k_state {
  int64_t m = 0, n = 0, k = 0;
  int b = 0, q = 0, s = 0;
  void* base = nullptr;                 // one device allocation for everything below
  uint64_t seed = 0;
  double *A = nullptr, *U = nullptr, *W = nullptr;
  double* gin = nullptr;                // copy of the injected Gaussian streams (or null: drawn from seed)
  double* Tfin = nullptr;                // T after the last step of the forward pass
  // each step's factors, kept from the forward (O((m + n) b) per step); the
  // reverse pass forms T after the step's right application again from the
  // checkpoint (one block-reflector application) instead of storing it
  struct Factors {
    double *G, *Ys, *Zs, *Vv, *tv, *Rv, *Sv, *Vu, *tu, *Ru, *Su;
  };
  std::vector<Factors> fs;
  // the reverse pass walks T and U back step by step with the kept
  // reflectors: recP holds T entering the step, recT T between its two
  // applications, recU U entering it
  double *recT = nullptr, *recP = nullptr, *recU = nullptr;
  // scratch
  double *work = nullptr, *gram = nullptr, *pq = nullptr, *c1 = nullptr, *c2 = nullptr, *c3 = nullptr,
         *c4 = nullptr, *big1 = nullptr, *big2 = nullptr, *Tbar = nullptr, *Ubar = nullptr, *vbar = nullptr,
         *nsym = nullptr, *taub = nullptr, *pbar = nullptr, *pwork = nullptr;
  double* hacc = nullptr;               // sums of the grid QR reverse (AD_MAXW x (2 AD_MAXW + 2))
  double* oz = nullptr;                 // Ozaki-scheme GEMM workspace (null: every product on DFMA)
  size_t ozb = 0;
  int64_t work_elems = 0;
  unsigned* flags = nullptr;
};

namespace rutv {
namespace {

using State = randutv_rank_k_state;

#define AD_CK(call)                                              \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return e_;                            \
  } while (0)

// The products go through the Ozaki-scheme GEMM (FP64-accurate, BF16 tensor
// cores) when the options ask for it and the product fills its tiles, else
// through the FP64 DFMA GEMM, as in the factorization.
cudaError_t g64(State& S, cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc) {
  if (S.oz && m >= 64 && n >= 32 && k >= 32 && gemm_oz_work_bytes(m, n, k) <= S.ozb)
    return gemm_oz(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, S.oz, S.ozb,
                   reinterpret_cast<int*>(S.flags + 2));
  return gemm_f64(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, S.work, S.work_elems);
}

// Householder QR of a copy of the L x w panel P (ld ldp): V (L x w), tau, R
// (w x w), S (w x w).
cudaError_t qr_panel(State& S, cudaStream_t s, int64_t L, int w, const double* P, int64_t ldp, double* V, double* tau,
                     double* R, double* Sf) {
  AD_CK(copy_matrix(s, L, w, P, ldp, S.pwork, L));
  AD_CK(panel_qr(s, L, w, S.pwork, L, tau, V, R, S.pq, S.flags));
  AD_CK(g64(S, s, true, false, w, w, L, 1.0, V, L, V, L, 0.0, S.gram, w));
  return tfactor_from_gram(s, w, S.gram, tau, Sf);
}

// C (M x K) <- C Q (right == true, Q = I - V S V^T, V K x w) or Q^T C (C K x M),
// with the transposed factor when trans (C Q^T, Q C).
cudaError_t wy_apply(State& S, cudaStream_t s, bool right, bool trans, int64_t M, int64_t K, int w, const double* V,
                     const double* Sf, double* C, int64_t ldc) {
  if (right) {   // C - (C V) S' V^T, S' = S or S^T
    AD_CK(g64(S, s, false, false, M, w, K, 1.0, C, ldc, V, K, 0.0, S.c1, M));
    AD_CK(g64(S, s, false, trans, M, w, w, 1.0, S.c1, M, Sf, w, 0.0, S.c2, M));
    return g64(S, s, false, true, M, K, w, -1.0, S.c2, M, V, K, 1.0, C, ldc);
  }
  // Q^T C = C - V S^T (V^T C);  Q C = C - V S (V^T C)
  AD_CK(g64(S, s, true, false, w, M, K, 1.0, V, K, C, ldc, 0.0, S.c1, w));
  AD_CK(g64(S, s, !trans, false, w, M, w, 1.0, Sf, w, S.c1, w, 0.0, S.c2, w));
  return g64(S, s, false, false, K, M, w, -1.0, V, K, S.c2, w, 1.0, C, ldc);
}

// Adjoint of Q = I - V S V^T (V L x w) given QV = Qbar V and QtV = Qbar^T V
// (L x w each): Vbar (into S.vbar) and taubar (into S.taub).
cudaError_t wy_adjoint(State& S, cudaStream_t s, int64_t L, int w, const double* V, const double* Sf,
                       const double* tau, const double* QV, const double* QtV) {
  AD_CK(g64(S, s, false, true, L, w, w, -1.0, QV, L, Sf, w, 0.0, S.vbar, L));
  AD_CK(g64(S, s, false, false, L, w, w, -1.0, QtV, L, Sf, w, 1.0, S.vbar, L));
  AD_CK(g64(S, s, true, false, w, w, L, 1.0, V, L, QV, L, 0.0, S.gram, w));
  wy_small_adjoint_kernel<<<1, AD_MAXW * AD_MAXW, 0, s>>>(w, S.gram, Sf, tau, S.nsym, S.taub);
  note_launch();
  AD_CK(cudaGetLastError());
  return g64(S, s, false, false, L, w, w, 1.0, V, L, S.nsym, w, 1.0, S.vbar, L);
}

// Reverse of the Householder QR: S.vbar, S.taub -> Pbar (L x w, ld L).
cudaError_t qr_reverse(State& S, cudaStream_t s, int64_t L, int w, const double* V, const double* tau, const double* R,
                       double* Pbar) {
  // rows per CTA: a multiple of 32 with the grid within one wave of the SMs
  int rpb = 32;
  while (static_cast<int64_t>(rpb) * (kNumSMs - 4) < L && rpb < HG_MAX_RPB) rpb += 32;
  const int nb = static_cast<int>((L + rpb - 1) / rpb);
  if (static_cast<int64_t>(rpb) * nb < L || nb > kNumSMs) {
    // too tall for one wave of row blocks: the one-CTA form
    hqr_reverse_kernel<<<1, HR_NT, 0, s>>>(static_cast<int>(L), w, V, tau, R, w, S.vbar, S.taub, S.pwork, Pbar);
    note_launch();
    return cudaGetLastError();
  }
  AD_CK(cudaMemsetAsync(S.hacc, 0, sizeof(double) * AD_MAXW * HG_ACC, s));
  AD_CK(cudaMemsetAsync(S.flags, 0, 2 * sizeof(unsigned), s));
  GridBarrier gb{S.flags, S.flags + 1, reinterpret_cast<int*>(S.flags + 2)};
  int Li = static_cast<int>(L), ldr = w;
  const double* taub = S.taub;
  double *vbar = S.vbar, *pw = S.pwork, *acc = S.hacc;
  void* args[] = {&Li, &w, &V, &tau, &R, &ldr, &vbar, &taub, &pw, &Pbar, &acc, &gb, &rpb};
  cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(hqr_reverse_grid_kernel), dim3(nb),
                                              dim3(HG_NT), args, 0, s);
  note_launch();
  return e;
}

cudaError_t add(cudaStream_t s, int64_t m, int64_t n, const double* X, int64_t ldx, double* Y, int64_t ldy) {
  const int64_t t = m * n;
  if (t == 0) return cudaSuccess;
  add_kernel<<<static_cast<unsigned>((t + 255) / 256), 256, 0, s>>>(m, n, X, ldx, Y, ldy);
  note_launch();
  return cudaGetLastError();
}

// Step i of the map on T (m x n) and U (m x m), both in place; the step's
// Gaussian, sketches, reflectors and factors go to S.fs[i - 1].
cudaError_t step_forward(State& S, cudaStream_t s, int i, double* T, double* U) {
  const int64_t m = S.m, n = S.n;
  const int b = S.b, q = S.q;
  auto& P = S.fs[i - 1];
  const int64_t r0 = static_cast<int64_t>(b) * (i - 1), kr = m - r0, kc = n - r0;
  if (S.gin) {
    int64_t goff = 0;
    for (int j = 1; j < i; ++j) goff += (m - static_cast<int64_t>(b) * (j - 1)) * b;
    AD_CK(cudaMemcpyAsync(P.G, S.gin + goff, sizeof(double) * kr * b, cudaMemcpyDeviceToDevice, s));
  } else {
    AD_CK(launch_gaussian(s, S.seed, i, kr, b, P.G, kr));
  }
  const double* X = T + r0 + r0 * m;
  // Ys holds Y_0 .. Y_q (kc x b each), Zs holds Z_1 .. Z_q (kr x b each)
  AD_CK(g64(S, s, true, false, kc, b, kr, 1.0, X, m, P.G, kr, 0.0, P.Ys, kc));
  for (int t = 1; t <= q; ++t) {
    double* Z = P.Zs + (t - 1) * kr * b;
    AD_CK(g64(S, s, false, false, kr, b, kc, 1.0, X, m, P.Ys + (t - 1) * kc * b, kc, 0.0, Z, kr));
    AD_CK(g64(S, s, true, false, kc, b, kr, 1.0, X, m, Z, kr, 0.0, P.Ys + t * kc * b, kc));
  }
  AD_CK(qr_panel(S, s, kc, b, P.Ys + q * kc * b, kc, P.Vv, P.tv, P.Rv, P.Sv));
  AD_CK(wy_apply(S, s, true, false, m, kc, b, P.Vv, P.Sv, T + r0 * m, m));
  AD_CK(qr_panel(S, s, kr, b, T + r0 + r0 * m, m, P.Vu, P.tu, P.Ru, P.Su));
  AD_CK(wy_apply(S, s, true, false, m, kr, b, P.Vu, P.Su, U + r0 * m, m));
  return wy_apply(S, s, false, false, kc, kr, b, P.Vu, P.Su, T + r0 + r0 * m, m);
}

cudaError_t forward(State& S, cudaStream_t s, const double* A, int64_t lda, double* F, int64_t ldf) {
  const int64_t m = S.m, n = S.n;
  AD_CK(copy_matrix(s, m, n, A, lda, S.A, m));
  double* T = S.big1;                    // the running T (m x n)
  AD_CK(copy_matrix(s, m, n, A, lda, T, m));
  AD_CK(set_identity(s, m, S.U, m));
  for (int i = 1; i <= S.s; ++i) AD_CK(step_forward(S, s, i, T, S.U));
  AD_CK(copy_matrix(s, m, n, T, m, S.Tfin, m));
  // W = U_k^T A, F = U_k W
  AD_CK(g64(S, s, true, false, S.k, n, m, 1.0, S.U, m, S.A, m, 0.0, S.W, S.k));
  return g64(S, s, false, false, m, n, S.k, 1.0, S.U, m, S.W, S.k, 0.0, F, ldf);
}

cudaError_t reverse(State& S, cudaStream_t s, const double* Fb, int64_t ldfb, double* Ab, int64_t ldab) {
  const int64_t m = S.m, n = S.n, k = S.k;
  const int b = S.b, q = S.q;
  double* Tb = S.Tbar;
  double* Ub = S.Ubar;
  // Abar = U_k (U_k^T Fbar); Ubar_k = Fbar W^T + A (Fbar^T U_k); Tbar = 0
  AD_CK(g64(S, s, true, false, k, n, m, 1.0, S.U, m, Fb, ldfb, 0.0, S.big2, k));
  AD_CK(g64(S, s, false, false, m, n, k, 1.0, S.U, m, S.big2, k, 0.0, Ab, ldab));
  AD_CK(cudaMemsetAsync(Ub, 0, sizeof(double) * m * m, s));
  AD_CK(g64(S, s, false, true, m, k, n, 1.0, Fb, ldfb, S.W, k, 0.0, Ub, m));
  AD_CK(g64(S, s, true, false, n, k, m, 1.0, Fb, ldfb, S.U, m, 0.0, S.big2, n));
  AD_CK(g64(S, s, false, false, m, k, n, 1.0, S.A, m, S.big2, n, 1.0, Ub, m));
  AD_CK(cudaMemsetAsync(Tb, 0, sizeof(double) * m * n, s));
  AD_CK(copy_matrix(s, m, n, S.Tfin, m, S.recP, m));
  AD_CK(copy_matrix(s, m, m, S.U, m, S.recU, m));
  for (int i = S.s; i >= 1; --i) {
    // T and U entering the step, and T between its two applications, walked
    // back from those after it with the step's own reflectors (orthogonal:
    // the inverse of C Q is C Q^T, of Q^T C is Q C)
    const auto& P = S.fs[i - 1];
    {
      const int64_t q0 = static_cast<int64_t>(b) * (i - 1), kr0 = m - q0, kc0 = n - q0;
      AD_CK(copy_matrix(s, m, n, S.recP, m, S.recT, m));
      AD_CK(wy_apply(S, s, false, true, kc0, kr0, b, P.Vu, P.Su, S.recT + q0 + q0 * m, m));   // Qu T(r0:, r0:)
      AD_CK(copy_matrix(s, m, n, S.recT, m, S.recP, m));
      AD_CK(wy_apply(S, s, true, true, m, kc0, b, P.Vv, P.Sv, S.recP + q0 * m, m));           // T(:, r0:) Qv^T
      AD_CK(wy_apply(S, s, true, true, m, kr0, b, P.Vu, P.Su, S.recU + q0 * m, m));           // U(:, r0:) Qu^T
    }
    const double* Tprev = S.recP;
    const double* Uprev = S.recU;
    const int64_t r0 = static_cast<int64_t>(b) * (i - 1), kr = m - r0, kc = n - r0;
    double* T2b = S.big2;                                 // Tbar(r0:, r0:) after the step (kr x kc, ld kr)
    AD_CK(copy_matrix(s, kr, kc, Tb + r0 + r0 * m, m, T2b, kr));
    double* Ubb = S.big1;                                 // Ubar(:, r0:) after the step (m x kr, ld m)
    AD_CK(copy_matrix(s, m, kr, Ub + r0 * m, m, Ubb, m));
    const double* T1b = S.recT + r0 + r0 * m;             // T(r0:, r0:) before the left application
    const double* Uo = Uprev + r0 * m;                    // U(:, r0:) before the right application
    // (left application of Qu^T to T and right application of Qu to U)
    AD_CK(wy_apply(S, s, false, true, kc, kr, b, P.Vu, P.Su, Tb + r0 + r0 * m, m));   // Qu Tbar_blk
    AD_CK(wy_apply(S, s, true, true, m, kr, b, P.Vu, P.Su, Ub + r0 * m, m));          // Ubar_blk Qu^T
    // QV = T1b (T2b^T Vu) + Uo^T (Ubb Vu), QtV = T2b (T1b^T Vu) + Ubb^T (Uo Vu)
    double *QV = S.c3, *QtV = S.c4;
    AD_CK(g64(S, s, true, false, kc, b, kr, 1.0, T2b, kr, P.Vu, kr, 0.0, S.c1, kc));
    AD_CK(g64(S, s, false, false, kr, b, kc, 1.0, T1b, m, S.c1, kc, 0.0, QV, kr));
    AD_CK(g64(S, s, false, false, m, b, kr, 1.0, Ubb, m, P.Vu, kr, 0.0, S.c2, m));
    AD_CK(g64(S, s, true, false, kr, b, m, 1.0, Uo, m, S.c2, m, 1.0, QV, kr));
    AD_CK(g64(S, s, true, false, kc, b, kr, 1.0, T1b, m, P.Vu, kr, 0.0, S.c1, kc));
    AD_CK(g64(S, s, false, false, kr, b, kc, 1.0, T2b, kr, S.c1, kc, 0.0, QtV, kr));
    AD_CK(g64(S, s, false, false, m, b, kr, 1.0, Uo, m, P.Vu, kr, 0.0, S.c2, m));
    AD_CK(g64(S, s, true, false, kr, b, m, 1.0, Ubb, m, S.c2, m, 1.0, QtV, kr));
    AD_CK(wy_adjoint(S, s, kr, b, P.Vu, P.Su, P.tu, QV, QtV));
    AD_CK(qr_reverse(S, s, kr, b, P.Vu, P.tu, P.Ru, S.pbar));
    AD_CK(add(s, kr, b, S.pbar, kr, Tb + r0 + r0 * m, m));
    // (right application of Qv to T(:, r0:)): C = Tprev(:, r0:), Cb = Tbar(:, r0:)
    const double* C = Tprev + r0 * m;
    double* Cb = Tb + r0 * m;
    AD_CK(g64(S, s, false, false, m, b, kc, 1.0, Cb, m, P.Vv, kc, 0.0, S.c2, m));     // Cb Vv
    AD_CK(g64(S, s, true, false, kc, b, m, 1.0, C, m, S.c2, m, 0.0, QV, kc));          // C^T (Cb Vv)
    AD_CK(g64(S, s, false, false, m, b, kc, 1.0, C, m, P.Vv, kc, 0.0, S.c1, m));      // C Vv
    AD_CK(g64(S, s, true, false, kc, b, m, 1.0, Cb, m, S.c1, m, 0.0, QtV, kc));        // Cb^T (C Vv)
    AD_CK(wy_adjoint(S, s, kc, b, P.Vv, P.Sv, P.tv, QV, QtV));
    double* Yb = S.pbar;                                                               // kc x b
    AD_CK(qr_reverse(S, s, kc, b, P.Vv, P.tv, P.Rv, Yb));
    AD_CK(wy_apply(S, s, true, true, m, kc, b, P.Vv, P.Sv, Cb, m));                   // Cb Qv^T
    // sketch: Y_t = X^T Z_t, Z_t = X Y_{t-1}, Y_0 = X^T G
    const double* X = Tprev + r0 + r0 * m;
    double* Xb = Tb + r0 + r0 * m;
    double* Ycur = Yb;                   // cotangent of Y_t
    for (int t = q; t >= 1; --t) {
      const double* Z = P.Zs + (t - 1) * kr * b;
      const double* Yp = P.Ys + (t - 1) * kc * b;
      double* Zb = S.c3;                 // kr x b
      AD_CK(g64(S, s, false, false, kr, b, kc, 1.0, X, m, Ycur, kc, 0.0, Zb, kr));
      AD_CK(g64(S, s, false, true, kr, kc, b, 1.0, Z, kr, Ycur, kc, 1.0, Xb, m));
      AD_CK(g64(S, s, false, true, kr, kc, b, 1.0, Zb, kr, Yp, kc, 1.0, Xb, m));
      double* Yn = S.c4;                 // kc x b
      AD_CK(g64(S, s, true, false, kc, b, kr, 1.0, X, m, Zb, kr, 0.0, Yn, kc));
      AD_CK(cudaMemcpyAsync(S.pbar, Yn, sizeof(double) * kc * b, cudaMemcpyDeviceToDevice, s));
      Ycur = S.pbar;
    }
    AD_CK(g64(S, s, false, true, kr, kc, b, 1.0, P.G, kr, Ycur, kc, 1.0, Xb, m));
  }
  return add(s, m, n, Tb, m, Ab, ldab);
}

int ad_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return RANDUTV_OK;
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  set_last_error(buf);
  return e == cudaErrorMemoryAllocation ? RANDUTV_ENOMEM : RANDUTV_ECUDA;
}

}  // namespace
}  // namespace rutv

extern "C" {

int randutv_rank_k(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q, int64_t k, double* F,
                   int64_t ldf, const randutv_opts* opts, randutv_rank_k_state** state) {
  using namespace rutv;
  randutv_opts o;
  randutv_opts_default(&o);
  if (opts) o = *opts;
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (!A) return -3;
  if (lda < m) return -4;
  if (b < 1) return -5;
  if (q < 0) return -6;
  if (k < b || k % b) return -7;
  if (!F) return -8;
  if (ldf < m) return -9;
  if (b > AD_MAXW) {
    set_last_error("rank-k map: block size above 32");
    return RANDUTV_EUNSUPPORTED;
  }
  if (k >= std::min(m, n)) {
    set_last_error("rank-k map: k must be below min(m, n) (randomized steps only)");
    return RANDUTV_EUNSUPPORTED;
  }
  if (o.p != 0) return -10;
  auto* S = new (std::nothrow) State;
  if (!S) return RANDUTV_ENOMEM;
  S->m = m;
  S->n = n;
  S->k = k;
  S->b = b;
  S->q = q;
  S->s = static_cast<int>(k / b);
  const int64_t mx = std::max(m, n);
  S->work_elems = std::max<int64_t>(24 * mx * b, 64ll * b * b);
  // sizes (doubles)
  std::vector<std::pair<double**, int64_t>> items;
  items.push_back({&S->A, m * n});
  items.push_back({&S->U, m * m});
  items.push_back({&S->W, k * n});
  items.push_back({&S->Tfin, m * n});
  // every step's factors, each sized for the first (largest) step
  S->fs.resize(S->s);
  for (int i = 0; i < S->s; ++i) {
    auto& P = S->fs[i];
    items.push_back({&P.G, m * b});
    items.push_back({&P.Ys, (q + 1) * n * b});
    items.push_back({&P.Zs, std::max<int64_t>(1, q * m * b)});
    items.push_back({&P.Vv, n * b});
    items.push_back({&P.tv, b});
    items.push_back({&P.Rv, b * b});
    items.push_back({&P.Sv, b * b});
    items.push_back({&P.Vu, m * b});
    items.push_back({&P.tu, b});
    items.push_back({&P.Ru, b * b});
    items.push_back({&P.Su, b * b});
  }
  items.push_back({&S->recT, m * n});
  items.push_back({&S->recP, m * n});
  items.push_back({&S->recU, m * m});
  int64_t gtot = 0;
  for (int i = 0; i < S->s; ++i) gtot += (m - static_cast<int64_t>(b) * i) * b;
  if (o.g_inject) items.push_back({&S->gin, gtot});
  items.push_back({&S->work, S->work_elems});
  items.push_back({&S->gram, b * b});
  items.push_back({&S->pq, panel_qr_part_elems(mx, b)});
  for (double** p : {&S->c1, &S->c2, &S->c3, &S->c4, &S->vbar, &S->pbar, &S->pwork}) items.push_back({p, mx * b});
  items.push_back({&S->big1, std::max(m * n, m * m)});
  items.push_back({&S->big2, std::max(m * n, m * m)});
  items.push_back({&S->Tbar, m * n});
  items.push_back({&S->Ubar, m * m});
  items.push_back({&S->nsym, b * b});
  items.push_back({&S->taub, b});
  items.push_back({&S->hacc, 32 * 66});
  if (o.fp64_emulation && gemm_oz_supported()) {
    // the largest products: m x n x k (the first forward product), mx x mx x b and thin mx x b x mx
    S->ozb = std::max({gemm_oz_work_bytes(m, n, std::max<int64_t>(m, k)), gemm_oz_work_bytes(mx, mx, b),
                       gemm_oz_work_bytes(mx, b, mx), gemm_oz_work_bytes(b, mx, mx), gemm_oz_work_bytes(mx, mx, mx)});
    items.push_back({&S->oz, static_cast<int64_t>((S->ozb + 7) / 8)});
  }
  size_t total = 0;
  for (auto& it : items) total += (static_cast<size_t>(it.second) * sizeof(double) + 255) & ~static_cast<size_t>(255);
  total += 256;
  cudaStream_t s = current_stream();
  cudaError_t e = cudaMalloc(&S->base, total);
  if (e != cudaSuccess) {
    delete S;
    return ad_status(e, "randutv_rank_k allocation");
  }
  char* p = static_cast<char*>(S->base);
  for (auto& it : items) {
    *it.first = reinterpret_cast<double*>(p);
    p += (static_cast<size_t>(it.second) * sizeof(double) + 255) & ~static_cast<size_t>(255);
  }
  S->flags = reinterpret_cast<unsigned*>(p);
  e = cudaMemsetAsync(S->flags, 0, 256, s);
  if (e == cudaSuccess && S->oz) e = cudaMemsetAsync(S->oz, 0, gemm_oz_head_bytes(), s);   // split-tile head
  S->seed = o.seed;
  if (e == cudaSuccess && o.g_inject)
    e = cudaMemcpyAsync(S->gin, o.g_inject, sizeof(double) * gtot, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = forward(*S, s, A, lda, F, ldf);
  unsigned herr[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(herr, S->flags, sizeof(herr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int st = ad_status(e, "randutv_rank_k");
  if (st == RANDUTV_OK && (herr[2] & kDevErrTimeout)) st = RANDUTV_ETIMEOUT;
  if (st != RANDUTV_OK || !state) {
    cudaFree(S->base);
    delete S;
    if (state) *state = nullptr;
    return st;
  }
  *state = S;
  return RANDUTV_OK;
}

int randutv_rank_k_vjp(randutv_rank_k_state* state, const double* Fbar, int64_t ldfb, double* Abar, int64_t ldab) {
  using namespace rutv;
  if (!state) return -1;
  if (!Fbar) return -2;
  if (ldfb < state->m) return -3;
  if (!Abar) return -4;
  if (ldab < state->m) return -5;
  cudaStream_t s = current_stream();
  cudaError_t e = reverse(*state, s, Fbar, ldfb, Abar, ldab);
  unsigned herr[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(herr, state->flags, sizeof(herr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  const int st = ad_status(e, "randutv_rank_k_vjp");
  if (st == RANDUTV_OK && (herr[2] & kDevErrTimeout)) return RANDUTV_ETIMEOUT;
  return st;
}

int randutv_rank_k_free(randutv_rank_k_state* state) {
  if (!state) return -1;
  cudaStreamSynchronize(rutv::current_stream());
  cudaFree(state->base);
  delete state;
  return RANDUTV_OK;
}

}  // extern "C"

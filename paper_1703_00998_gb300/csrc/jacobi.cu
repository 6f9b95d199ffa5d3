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
// milliseconds for a 128 x 128 SVD; instead one cooperative launch gives each
// pair of a round its own CTA (p/2 CTAs) and separates the rounds by a grid
// barrier.  W and Q live in global memory (L2-resident, 2 p^2 doubles).
// Order and signs: singular values descending (stable in the column index);
// the largest-|.| entry of each Vs column positive (lowest index on ties),
// Us flipped with it; zero singular values get Vs columns that complete an
// orthonormal basis (Gram-Schmidt of unit vectors).
#include "common.cuh"
#include "internal.h"

namespace rutv {

constexpr int JC_NT = 128;

__device__ __forceinline__ void rr_pair(int pp, int r, int kpair, int* a, int* b) {
  auto idx = [&](int t) { return t == 0 ? 0 : ((t - 1 + r) % (pp - 1)) + 1; };
  int x = idx(kpair), y = idx(pp - 1 - kpair);
  *a = min(x, y);
  *b = max(x, y);
}

constexpr int JC_MAXR = 4;   // rows per thread: p <= JC_NT * JC_MAXR = 512

__global__ void __launch_bounds__(JC_NT)
jacobi_sweeps_kernel(int p, int pp, double* __restrict__ W, double* __restrict__ V, int max_sweeps,
                     double tol, unsigned* __restrict__ sweep_flag, GridBarrier gb) {
  __shared__ double red[3][JC_NT / 32];
  __shared__ double s_cs[2];
  __shared__ int s_rot;
  __shared__ double s_thr2;
  const int nb = gridDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // Columns whose norm is at the rounding level of the whole block,
  // ||w|| <= p u ||M||_F, are treated as zero: rotating them only stirs
  // rounding noise and would never meet the relative stopping test.
  {
    double f = 0.0;
    for (int64_t e = tid; e < static_cast<int64_t>(p) * p; e += JC_NT) {
      const double x = __ldcg(W + e);
      f = fma(x, x, f);
    }
    f = warp_sum(f);
    if (lane == 0) red[0][warp] = f;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < JC_NT / 32; ++w) t += red[0][w];
      const double pu = static_cast<double>(p) * 0x1p-53;
      s_thr2 = pu * pu * t;
    }
    __syncthreads();
  }
  const double thr2 = s_thr2;
  for (int sw = 0; sw < max_sweeps; ++sw) {
    for (int r = 0; r < pp - 1; ++r) {
      int i, j;
      rr_pair(pp, r, blockIdx.x, &i, &j);
      if (j < p) {
        double* wi = W + static_cast<int64_t>(i) * p;
        double* wj = W + static_cast<int64_t>(j) * p;
        double x[JC_MAXR], y[JC_MAXR];
        double a = 0.0, b = 0.0, g = 0.0;
#pragma unroll
        for (int u = 0; u < JC_MAXR; ++u) {
          const int t = tid + u * JC_NT;
          x[u] = (t < p) ? __ldcg(wi + t) : 0.0;
          y[u] = (t < p) ? __ldcg(wj + t) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < JC_MAXR; ++u) {
          a = fma(x[u], x[u], a); b = fma(y[u], y[u], b); g = fma(x[u], y[u], g);
        }
        a = warp_sum(a); b = warp_sum(b); g = warp_sum(g);
        if (lane == 0) { red[0][warp] = a; red[1][warp] = b; red[2][warp] = g; }
        __syncthreads();
        if (tid == 0) {
          a = b = g = 0.0;
          for (int w = 0; w < JC_NT / 32; ++w) { a += red[0][w]; b += red[1][w]; g += red[2][w]; }
          int rot = 0;
          if (g != 0.0 && a > thr2 && b > thr2 && fabs(g) > tol * sqrt(a) * sqrt(b)) {
            const double zeta = (b - a) / (2.0 * g);
            const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
            const double c = 1.0 / sqrt(fma(t, t, 1.0));
            s_cs[0] = c;
            s_cs[1] = c * t;
            rot = 1;
          }
          s_rot = rot;
        }
        __syncthreads();
        if (s_rot) {
          const double c = s_cs[0], s = s_cs[1];
          double* vi = V + static_cast<int64_t>(i) * p;
          double* vj = V + static_cast<int64_t>(j) * p;
#pragma unroll
          for (int u = 0; u < JC_MAXR; ++u) {
            const int t = tid + u * JC_NT;
            if (t < p) {
              wi[t] = c * x[u] - s * y[u];
              wj[t] = s * x[u] + c * y[u];
              const double q1 = __ldcg(vi + t), q2 = __ldcg(vj + t);
              vi[t] = c * q1 - s * q2;
              vj[t] = s * q1 + c * q2;
            }
          }
          if (tid == 0) atomicOr(sweep_flag + sw, 1u);
        }
      }
      if (!grid_barrier(gb, nb)) return;
    }
    if (ld_acquire_u32(sweep_flag + sw) == 0u) return;  // a sweep without rotations: converged
  }
  if (blockIdx.x == 0 && tid == 0) atomicOr(gb.err, kDevErrNoConv);
}

// Sort, normalise, complete, sign-fix; one CTA.
__global__ void __launch_bounds__(256)
jacobi_finish_kernel(int p, const double* __restrict__ W, const double* __restrict__ V,
                     double* __restrict__ Us, double* __restrict__ d, double* __restrict__ Vs,
                     double* __restrict__ sig, int* __restrict__ perm) {
  const int tid = threadIdx.x;
  for (int c = tid; c < p; c += blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < p; ++t) s = fma(W[t + static_cast<int64_t>(c) * p], W[t + static_cast<int64_t>(c) * p], s);
    sig[c] = sqrt(s);
  }
  __syncthreads();
  {
    // negligible columns (see the sweep kernel) count as exact zeros
    __shared__ double s_cut;
    if (tid == 0) {
      double f = 0.0;
      for (int c = 0; c < p; ++c) f = fma(sig[c], sig[c], f);
      s_cut = static_cast<double>(p) * 0x1p-53 * sqrt(f);
    }
    __syncthreads();
    const double cut = s_cut;
    for (int c = tid; c < p; c += blockDim.x)
      if (sig[c] <= cut) sig[c] = 0.0;
    __syncthreads();
  }
  for (int c = tid; c < p; c += blockDim.x) {
    int rank = 0;
    const double sc = sig[c];
    for (int o = 0; o < p; ++o) rank += (sig[o] > sc) || (sig[o] == sc && o < c);
    perm[rank] = c;
  }
  __syncthreads();
  for (int64_t e = tid; e < static_cast<int64_t>(p) * p; e += blockDim.x) {
    const int t = static_cast<int>(e % p), r = static_cast<int>(e / p);
    const int c = perm[r];
    const double s = sig[c];
    Vs[t + static_cast<int64_t>(r) * p] = (s > 0.0) ? W[t + static_cast<int64_t>(c) * p] / s : 0.0;
    Us[t + static_cast<int64_t>(r) * p] = V[t + static_cast<int64_t>(c) * p];
    if (t == 0) d[r] = s;
  }
  __syncthreads();
  // Complete the basis for zero singular values (columns with sigma = 0 are last).
  __shared__ double red[8];
  for (int r = 0; r < p; ++r) {
    if (sig[perm[r]] > 0.0) continue;
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
          if ((tid & 31) == 0) red[tid >> 5] = s;
          __syncthreads();
          double dot = 0.0;
          for (int w = 0; w < static_cast<int>(blockDim.x) / 32; ++w) dot += red[w];
          __syncthreads();
          for (int t = tid; t < p; t += blockDim.x) u[t] -= dot * uq[t];
          __syncthreads();
        }
      }
      double s = 0.0;
      for (int t = tid; t < p; t += blockDim.x) s = fma(u[t], u[t], s);
      s = warp_sum(s);
      if ((tid & 31) == 0) red[tid >> 5] = s;
      __syncthreads();
      double nrm2 = 0.0;
      for (int w = 0; w < static_cast<int>(blockDim.x) / 32; ++w) nrm2 += red[w];
      __syncthreads();
      if (nrm2 > 0.25) {
        const double inv = 1.0 / sqrt(nrm2);
        for (int t = tid; t < p; t += blockDim.x) u[t] *= inv;
        __syncthreads();
        break;
      }
    }
  }
  __syncthreads();
  // Sign convention on Vs columns.
  for (int r = tid; r < p; r += blockDim.x) {
    double* v = Vs + static_cast<int64_t>(r) * p;
    int best = 0;
    double bv = fabs(v[0]);
    for (int t = 1; t < p; ++t) {
      const double a = fabs(v[t]);
      if (a > bv) { bv = a; best = t; }
    }
    if (v[best] < 0.0) {
      double* u = Us + static_cast<int64_t>(r) * p;
      for (int t = 0; t < p; ++t) { v[t] = -v[t]; u[t] = -u[t]; }
    }
  }
}

__global__ void jacobi_init_kernel(int p, const double* __restrict__ M, int64_t ldm, double* __restrict__ W,
                                   double* __restrict__ V) {
  const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (e >= static_cast<int64_t>(p) * p) return;
  const int t = static_cast<int>(e % p), c = static_cast<int>(e / p);
  W[e] = M[c + t * ldm];   // W = M^T
  V[e] = (t == c) ? 1.0 : 0.0;
}

int64_t jacobi_work_elems(int p) {
  // W, V (p x p each), sig (p), perm (p ints), sweep flags (<= 64 unsigned)
  return 2ll * p * p + 2ll * p + 64;
}

cudaError_t jacobi_svd(cudaStream_t s, int p, const double* M, int64_t ldm, double* Us, double* d,
                       double* Vs, int max_sweeps, double* work, unsigned* bar) {
  if (p < 1) return cudaSuccess;
  if (p > JC_NT * JC_MAXR) return cudaErrorInvalidValue;
  if (max_sweeps > 64) max_sweeps = 64;
  double* W = work;
  double* V = W + static_cast<int64_t>(p) * p;
  double* sig = V + static_cast<int64_t>(p) * p;
  int* perm = reinterpret_cast<int*>(sig + p);
  unsigned* flags = reinterpret_cast<unsigned*>(sig + 2 * p);
  const int64_t pe = static_cast<int64_t>(p) * p;
  const ProfToken tok = prof_begin(s, kProfJacobi);
  jacobi_init_kernel<<<static_cast<unsigned>((pe + 255) / 256), 256, 0, s>>>(p, M, ldm, W, V);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (p >= 2) {
    if ((e = cudaMemsetAsync(flags, 0, 64 * sizeof(unsigned), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s)) != cudaSuccess) return e;
    int pp = p + (p & 1);
    double tol = static_cast<double>(p) * 0x1p-53;
    GridBarrier gb{bar, bar + 1, reinterpret_cast<int*>(bar + 2)};
    void* args[] = {&p, &pp, &W, &V, &max_sweeps, &tol, &flags, &gb};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(jacobi_sweeps_kernel), dim3(pp / 2),
                                    dim3(JC_NT), args, 0, s);
    note_launch();
    if (e != cudaSuccess) return e;
  }
  jacobi_finish_kernel<<<1, 256, 0, s>>>(p, W, V, Us, d, Vs, sig, perm);
  note_launch(2);
  // flops are iteration-dependent; record the p x p input and three p x p outputs
  prof_end(s, tok, 0.0, 8.0 * 4.0 * p * p);
  return cudaGetLastError();
}

}  // namespace rutv

// Batched randUTV of many small FP32 matrices (m, n <= 512): Fig. 4 run on
// each matrix by one CTA, all matrices in ONE persistent kernel that takes
// them from a device work queue, largest first.  Each matrix stops early
// once its trailing block is small (Section 1.1 (ii): ||T22||_F <= tol
// ||A||_F before a step) and ends with the rectangular final blocks of
// Section 5.2 (tall: QR of the columns, then an SVD of R) and of the Remark
// on m < n (wide: QR of the rows, then an SVD of L = R^T).
//
// Per CTA (512 threads) the whole step stays on chip except the matrix
// itself: the b-wide operands (G, the samples Y, the reflector blocks, the
// products W = C V) live in shared memory as row-major panels, panels are
// factored with one row per thread in registers, the b x b SVD is a
// one-sided Jacobi in shared memory, and T, U, V are read and written in
// place in global memory (L2-resident while the CTA works on them).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>
#include "common.cuh"
#include "internal.h"
#include "philox.cuh"

namespace rutv {
namespace {

constexpr int BT_NT = 512;           // threads per CTA
constexpr int BT_NW = BT_NT / 32;    // warps per CTA
constexpr int BT_MAXD = 512;         // largest m, n (one panel row per thread)
constexpr int LDW = 36;              // row stride (floats) of the panel buffers
constexpr int LDQ = 36;              // leading dimension of the small column-major matrices
constexpr int KCH = 16;              // K chunk of the staged A^T B product
constexpr int LDAT = 514;            // row stride of its staging tile (2 mod 32: no bank conflicts)

// One matrix of the batch: sizes, block size and element offsets into the
// packed A/T, U, V and Gaussian-stream buffers.
struct BMat {
  int m, n, b, pad;
  int64_t a, u, v, g;
};

struct BtSmem {
  float P0[BT_MAXD * LDW];   // panel buffers: row i at [i * LDW], columns 0..31
  float P1[BT_MAXD * LDW];
  float At[KCH * LDAT];      // staging tile of A^T B
  float S[32 * LDQ];         // T factor of the current reflector block
  float R[32 * LDQ];         // R of a panel, then Us
  float Vs[32 * LDQ];        // right singular vectors of the small SVD
  float d[32];               // singular values, descending
  float sig[32];
  float redv[2][BT_NW][33];  // vector reductions (two alternating buffers)
  float vec[2][32];
  float reds[2][3 * BT_NW];  // scalar reductions
  double redd[2][BT_NW];
  int rank[32];
};

struct BtArgs {
  const BMat* tab;
  const int* order;
  int count;
  const float* A;
  float* T;
  float* U;
  float* V;
  const float* gin;
  int form_uv, q, max_sweeps;
  float tol;
  uint32_t k0, k1;
  int* k_out;
  int* info;
  int* err;
  unsigned* head;
  unsigned* done;
  unsigned long long* tns;
};

// Alternating-buffer parities of the reductions: identical in every thread,
// so one barrier per scalar reduction suffices (a buffer is rewritten only
// after every thread passed the next reduction's barrier).
struct Red {
  int ps = 0, pv = 0, pd = 0;
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// (sum of a, sum of b, max of c) over the CTA, returned to every thread.
__device__ float3 block_sum2_max(BtSmem& sm, Red& rd, float a, float b, float c) {
  a = warp_sum(a);
  b = warp_sum(b);
#pragma unroll
  for (int o = 16; o; o >>= 1) c = fmaxf(c, __shfl_xor_sync(0xffffffffu, c, o));
  float* buf = sm.reds[rd.ps];
  rd.ps ^= 1;
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    buf[w] = a;
    buf[BT_NW + w] = b;
    buf[2 * BT_NW + w] = c;
  }
  __syncthreads();
  float sa = 0.f, sb = 0.f, mc = 0.f;
#pragma unroll
  for (int i = 0; i < BT_NW; ++i) {
    sa += buf[i];
    sb += buf[BT_NW + i];
    mc = fmaxf(mc, buf[2 * BT_NW + i]);
  }
  return make_float3(sa, sb, mc);
}

__device__ double block_sum_d(BtSmem& sm, Red& rd, double a) {
  a = warp_sum_d(a);
  double* buf = sm.redd[rd.pd];
  rd.pd ^= 1;
  if ((threadIdx.x & 31) == 0) buf[threadIdx.x >> 5] = a;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < BT_NW; ++i) s += buf[i];
  return s;
}

// Butterfly ("transpose") reduction: after it lane l holds the warp-wide sum
// of v[l % NB] (31 shuffles for NB = 32, 16 for NB = 16).
template <int NB>
__device__ __forceinline__ float warp_vsum(float (&v)[NB]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = NB / 2; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const float send = up ? v[i] : v[i + s];
      const float keep = up ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  float r = v[0];
  if (NB == 16) r += __shfl_xor_sync(0xffffffffu, r, 16);
  return r;
}

// CTA-wide sum of the vector v (NB entries per thread); the result is in
// shared memory, valid until the second reduction after this one.
template <int NB>
__device__ const float* block_vsum(BtSmem& sm, Red& rd, float (&v)[NB]) {
  const float r = warp_vsum<NB>(v);
  float(*buf)[33] = sm.redv[rd.pv];
  float* out = sm.vec[rd.pv];
  rd.pv ^= 1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane < NB) buf[w][lane] = r;
  __syncthreads();
  if (threadIdx.x < NB) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < BT_NW; ++i) s += buf[i][threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
  return out;
}

// Two standard normals from one Philox block in FP32 (Box-Muller): u1, u2
// from the top 23 bits of words x1 and x3, u = (floor(w / 2^9) + 1/2) 2^-23,
// exact in FP32 and inside (0, 1).
__device__ __forceinline__ float2 box_muller_f32(U4 w) {
  const float u1 = (static_cast<float>(w.x1 >> 9) + 0.5f) * 0x1p-23f;
  const float u2 = (static_cast<float>(w.x3 >> 9) + 0.5f) * 0x1p-23f;
  const float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  return make_float2(r * c, r * s);
}

// G (kr x b) of step `step` of matrix `idx` into the panel buffer P (zero
// columns b..NB-1): injected (column-major, ld kr) or drawn with counter
// (row / 2, column, step, idx) under key (k0, k1).
template <int NB>
__device__ __noinline__ void fill_gaussian(float* P, int kr, int b, uint32_t k0, uint32_t k1, uint32_t step, uint32_t idx,
                              const float* gin) {
  const int tid = threadIdx.x;
  if (gin) {
    for (int e = tid; e < kr * b; e += BT_NT) {
      const int r = e % kr, c = e / kr;
      P[r * LDW + c] = gin[e];
    }
  } else {
    const int np = (kr + 1) / 2;
    for (int e = tid; e < np * b; e += BT_NT) {
      const int p = e % np, c = e / np;
      const float2 z = box_muller_f32(philox4x32_10(U4{static_cast<uint32_t>(p), static_cast<uint32_t>(c), step, idx},
                                                    k0, k1));
      P[(2 * p) * LDW + c] = z.x;
      if (2 * p + 1 < kr) P[(2 * p + 1) * LDW + c] = z.y;
    }
  }
  if (b < NB)
    for (int e = tid; e < kr * (NB - b); e += BT_NT) P[(e / (NB - b)) * LDW + b + e % (NB - b)] = 0.f;
  __syncthreads();
}

// Thread layout of the skinny products C (M x NB) = op(A) B: one output row
// per thread, rows in warps of 32, and KS = floor(16 / warps per row set)
// groups of warps splitting K (KS * Mp <= 512).
struct SkinnyMap {
  int Mp, nwr, KS, kg, i;
  bool act;
  __device__ SkinnyMap(int M) {
    Mp = (M + 31) & ~31;
    nwr = Mp >> 5;
    KS = BT_NW / nwr;
    const int w = threadIdx.x >> 5;
    kg = w / nwr;
    i = (w % nwr) * 32 + (threadIdx.x & 31);
    act = kg < KS;
  }
};

// Store the accumulators of a skinny product into C (row-major, ld LDW),
// summing the KS partial products through C's own buffer when K was split.
template <int NB>
__device__ __forceinline__ void skinny_store(const SkinnyMap& mp, float (&acc)[NB], float* C, int M) {
  if (mp.KS == 1) {
    if (mp.act && mp.i < M) {
      float4* c4 = reinterpret_cast<float4*>(C + mp.i * LDW);
#pragma unroll
      for (int j = 0; j < NB / 4; ++j) c4[j] = make_float4(acc[4 * j], acc[4 * j + 1], acc[4 * j + 2], acc[4 * j + 3]);
    }
    __syncthreads();
    return;
  }
  // partial of group g, column c, row i at C[(g * NB + c) * Mp + i]
  // (KS * Mp <= 512, so this fits the 512 x LDW buffer)
  if (mp.act) {
#pragma unroll
    for (int c = 0; c < NB; ++c) C[(mp.kg * NB + c) * mp.Mp + mp.i] = acc[c];
  }
  __syncthreads();
  const int tot = NB * mp.Mp;
  float out[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const int o = threadIdx.x + j * BT_NT;
    float s = 0.f;
    if (o < tot) {
      const int c = o / mp.Mp, ii = o % mp.Mp;
      for (int g = 0; g < mp.KS; ++g) s += C[(g * NB + c) * mp.Mp + ii];
    }
    out[j] = s;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const int o = threadIdx.x + j * BT_NT;
    if (o < tot) {
      const int c = o / mp.Mp, ii = o % mp.Mp;
      if (ii < M) C[ii * LDW + c] = out[j];
    }
  }
  __syncthreads();
}

// C (M x NB, shared, row-major) = A^T B with A global column-major K x M
// (ld lda) and B shared row-major K x NB.  A is staged through shared
// memory KCH rows at a time so that its loads are coalesced.
template <int NB>
__device__ __noinline__ void gemm_tn_small(BtSmem& sm, const float* A, int lda, int K, int M, const float* B, float* C) {
  if (M <= 0) return;
  const SkinnyMap mp(M);
  float acc[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) acc[c] = 0.f;
  // each thread stages at most KCH * 512 / BT_NT = 16 elements per chunk;
  // the next chunk is loaded into registers while the current one is used
  constexpr int PER = KCH * BT_MAXD / BT_NT;
  float pre[PER];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + u * BT_NT;
      const int kk = e % KCH, ii = e / KCH, k = k0 + kk;
      pre[u] = (e < KCH * M && k < K) ? A[k + static_cast<int64_t>(ii) * lda] : 0.f;
    }
  };
  fetch(0);
  for (int k0 = 0; k0 < K; k0 += KCH) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + u * BT_NT;
      if (e < KCH * M) sm.At[(e % KCH) * LDAT + e / KCH] = pre[u];
    }
    __syncthreads();
    if (k0 + KCH < K) fetch(k0 + KCH);
    if (mp.act && mp.i < M) {
      for (int kk = mp.kg; kk < KCH; kk += mp.KS) {
        const int k = k0 + kk;
        if (k >= K) break;
        const float a = sm.At[kk * LDAT + mp.i];
        const float4* b4 = reinterpret_cast<const float4*>(B + k * LDW);
#pragma unroll
        for (int j = 0; j < NB / 4; ++j) {
          const float4 bb = b4[j];
          acc[4 * j] = fmaf(a, bb.x, acc[4 * j]);
          acc[4 * j + 1] = fmaf(a, bb.y, acc[4 * j + 1]);
          acc[4 * j + 2] = fmaf(a, bb.z, acc[4 * j + 2]);
          acc[4 * j + 3] = fmaf(a, bb.w, acc[4 * j + 3]);
        }
      }
    }
  }
  __syncthreads();
  skinny_store<NB>(mp, acc, C, M);
}

// C (M x NB, shared, row-major) = A B with A global column-major M x K (ld
// lda) and B shared row-major K x NB.  Rows of A are read coalesced along M;
// each B row is a broadcast.
template <int NB>
__device__ __noinline__ void gemm_nn_small(const float* A, int lda, int M, int K, const float* B, float* C) {
  if (M <= 0) return;
  const SkinnyMap mp(M);
  float acc[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) acc[c] = 0.f;
  if (mp.act && mp.i < M) {
    const int kper = (K + mp.KS - 1) / mp.KS;
    const int kb = mp.kg * kper, ke = min(K, kb + kper);
    const float* a = A + mp.i;
    // eight loads in flight per thread: the next group of columns is
    // fetched while the current one is multiplied
    float nxt[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) nxt[u] = (kb + u < ke) ? a[static_cast<int64_t>(kb + u) * lda] : 0.f;
    for (int k = kb; k < ke; k += 8) {
      float av[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) av[u] = nxt[u];
#pragma unroll
      for (int u = 0; u < 8; ++u) nxt[u] = (k + 8 + u < ke) ? a[static_cast<int64_t>(k + 8 + u) * lda] : 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (k + u >= ke) break;
        const float4* b4 = reinterpret_cast<const float4*>(B + (k + u) * LDW);
#pragma unroll
        for (int j = 0; j < NB / 4; ++j) {
          const float4 bb = b4[j];
          acc[4 * j] = fmaf(av[u], bb.x, acc[4 * j]);
          acc[4 * j + 1] = fmaf(av[u], bb.y, acc[4 * j + 1]);
          acc[4 * j + 2] = fmaf(av[u], bb.z, acc[4 * j + 2]);
          acc[4 * j + 3] = fmaf(av[u], bb.w, acc[4 * j + 3]);
        }
      }
    }
  }
  skinny_store<NB>(mp, acc, C, M);
}

// C (M x N, global column-major, ld ldc) = beta C + alpha A B^T with A
// (M x K) and B (N x K) shared row-major (ld LDW, K <= 32, columns K..K4-1
// zero).  Tiles of 128 x 64, a 4 x 4 block per thread.  With want_ss the
// CTA-wide sum of squares of the new C over rows >= srow is returned.
__device__ __noinline__ double gemm_update(BtSmem& sm, Red& rd, float* C, int ldc, int M, int N, const float* A, const float* B,
                              int K, float alpha, float beta, int srow, bool want_ss) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int K4 = (K + 3) & ~3;
  double ssd = 0.0;
  for (int tm = 0; tm < M; tm += 128) {
    for (int tn = 0; tn < N; tn += 64) {
      float acc[4][4];
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[s][t] = 0.f;
      int ii[4], jj[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) ii[s] = tm + lane + 32 * s;
#pragma unroll
      for (int t = 0; t < 4; ++t) jj[t] = tn + warp + 16 * t;
      // the tile's old values are fetched before the products so that
      // their latency overlaps the FMA loop
      float cold[4][4];
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int s = 0; s < 4; ++s)
          cold[s][t] = (beta != 0.f && ii[s] < M && jj[t] < N) ? C[ii[s] + static_cast<int64_t>(jj[t]) * ldc] : 0.f;
      for (int k = 0; k < K4; k += 4) {
        float4 a[4], bq[4];
#pragma unroll
        for (int s = 0; s < 4; ++s)
          a[s] = ii[s] < M ? *reinterpret_cast<const float4*>(A + ii[s] * LDW + k) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int t = 0; t < 4; ++t)
          bq[t] = jj[t] < N ? *reinterpret_cast<const float4*>(B + jj[t] * LDW + k) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            float v = acc[s][t];
            v = fmaf(a[s].x, bq[t].x, v);
            v = fmaf(a[s].y, bq[t].y, v);
            v = fmaf(a[s].z, bq[t].z, v);
            v = fmaf(a[s].w, bq[t].w, v);
            acc[s][t] = v;
          }
      }
      float ss = 0.f;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (jj[t] >= N) continue;
        float* col = C + static_cast<int64_t>(jj[t]) * ldc;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          if (ii[s] >= M) continue;
          float v = alpha * acc[s][t];
          if (beta != 0.f) v = fmaf(beta, cold[s][t], v);
          col[ii[s]] = v;
          if (ii[s] >= srow) ss = fmaf(v, v, ss);
        }
      }
      ssd += static_cast<double>(ss);
    }
  }
  double r = 0.0;
  if (want_ss) r = block_sum_d(sm, rd, ssd);
  __syncthreads();
  return r;
}

// W (M x NB, shared row-major) <- W S with S upper triangular (column-major,
// ld LDQ, zero outside its leading block).
template <int NB>
__device__ __noinline__ void mul_tri(float* W, int M, const float* S) {
  for (int i = threadIdx.x; i < M; i += BT_NT) {
    float x[NB];
    const float4* w4 = reinterpret_cast<const float4*>(W + i * LDW);
#pragma unroll
    for (int j = 0; j < NB / 4; ++j) {
      const float4 v = w4[j];
      x[4 * j] = v.x;
      x[4 * j + 1] = v.y;
      x[4 * j + 2] = v.z;
      x[4 * j + 3] = v.w;
    }
    // (W S)(i, c) needs x[0..c] only: overwrite from the last column down
#pragma unroll
    for (int c = NB - 1; c >= 0; --c) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k <= c; ++k) s = fmaf(x[k], S[c * LDQ + k], s);
      x[c] = s;
    }
    float4* o4 = reinterpret_cast<float4*>(W + i * LDW);
#pragma unroll
    for (int j = 0; j < NB / 4; ++j) o4[j] = make_float4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
  }
  __syncthreads();
}

// Householder QR (dlarfg convention: v(j) = 1, beta = -sign(alpha) ||x||,
// tau = (beta - alpha) / beta, tau = 0 when the part below the diagonal is
// zero; a column whose entries would under- or overflow when squared is
// normed after scaling by a power of two) of the M x w panel held one row
// per thread: thread r < M holds row r in x (zero beyond w; threads r >= M
// hold zeros).  On return thread r holds
// R(r, c) for c >= r (r < w) and the reflector entries v_c(r) for c < r, and
// sm.S holds the upper triangular S with H_0 ... H_{w-1} = I - V S V^T
// (S(j, j) = tau_j, S(0:j, j) = -tau_j S(0:j, 0:j) V(:, 0:j)^T v_j).
// Per column: one scalar reduction (the norm, alpha, max |x|) and one
// vector reduction (the products of v_j with every other column: the update
// for c > j and the Gram entries of S for c < j).
template <int NB>
__device__ __forceinline__ void panel_qr_regs(BtSmem& sm, Red& rd, float (&x)[NB], int M, int w) {
  const int r = threadIdx.x;
  for (int e = r; e < 32 * LDQ; e += BT_NT) sm.S[e] = 0.f;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j >= w) break;
    const float xj = x[j];
    const float3 t = block_sum2_max(sm, rd, (r > j && r < M) ? xj * xj : 0.f, r == j ? xj : 0.f,
                                    (r >= j && r < M) ? fabsf(xj) : 0.f);
    float s1 = t.x, alpha = t.y, sc = 1.f;
    if (t.z > 0.f && (t.z < 0x1p-40f || t.z > 0x1p40f)) {
      // squares of this column would under- or overflow FP32: take the norm
      // of the column scaled by a power of two (v and tau are scale free,
      // beta is scaled back exactly)
      int e;
      frexpf(t.z, &e);
      sc = ldexpf(1.f, -e);
      const float xs = xj * sc;
      s1 = block_sum2_max(sm, rd, (r > j && r < M) ? xs * xs : 0.f, 0.f, 0.f).x;
      alpha *= sc;
    }
    float tau = 0.f, beta = alpha / sc, scal = 0.f;
    if (s1 > 0.f) {
      const float bs = -copysignf(hypotf(alpha, sqrtf(s1)), alpha);
      tau = (bs - alpha) / bs;
      scal = sc / (alpha - bs);
      beta = bs / sc;
    }
    float vj = 0.f;
    if (r == j) {
      vj = 1.f;
      x[j] = beta;
    } else if (r > j && r < M) {
      x[j] *= scal;
      vj = x[j];
    }
    float pv[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) pv[c] = (c == j) ? 0.f : vj * x[c];
    const float* dot = block_vsum<NB>(sm, rd, pv);
    const float tv = tau * vj;
#pragma unroll
    for (int c = j + 1; c < NB; ++c)
      if (c < w) x[c] = fmaf(-tv, dot[c], x[c]);
    if (r < j) {
      float s = 0.f;
      for (int k = r; k < j; ++k) s = fmaf(sm.S[k * LDQ + r], dot[k], s);
      sm.S[j * LDQ + r] = -tau * s;
    } else if (r == j) {
      sm.S[j * LDQ + j] = tau;
    }
  }
  __syncthreads();
}

// Write the reflectors of a factored panel (unit lower trapezoidal, zero
// beyond column w) into the row-major buffer Vout, and with want_r its
// R (w x w) into sm.R (column-major, zero outside w x w).
template <int NB>
__device__ __forceinline__ void store_panel(BtSmem& sm, const float (&x)[NB], int M, int w, float* Vout, bool want_r) {
  const int r = threadIdx.x;
  if (r < M) {
    float v[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) v[c] = (c >= w) ? 0.f : (r > c ? x[c] : (r == c ? 1.f : 0.f));
    float4* o4 = reinterpret_cast<float4*>(Vout + r * LDW);
#pragma unroll
    for (int j = 0; j < NB / 4; ++j) o4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
  }
  if (want_r && r < 32) {
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      float v = 0.f;
      if (c < NB) v = (r < w && c < w && c >= r) ? x[c < NB ? c : 0] : 0.f;
      sm.R[c * LDQ + r] = v;
    }
  }
  __syncthreads();
}

// P (M x NB, row-major) = src(0:M, 0:w) of a global column-major block (ld),
// zero beyond column w.
template <int NB>
__device__ void stage_rows(const float* src, int ld, int M, int w, float* P) {
  for (int e = threadIdx.x; e < M * NB; e += BT_NT) {
    const int i = e % M, k = e / M;
    P[i * LDW + k] = (k < w) ? src[i + static_cast<int64_t>(k) * ld] : 0.f;
  }
  __syncthreads();
}

// P (N x NB, row-major) with P(j, k) = src(k, j) for k < K (<= NB) of a
// global column-major K x N block (ld), zero beyond column K.
template <int NB>
__device__ void stage_cols_t(const float* src, int ld, int K, int N, float* P) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < N; j += BT_NW)
    if (lane < NB) P[j * LDW + lane] = (lane < K) ? src[lane + static_cast<int64_t>(j) * ld] : 0.f;
  __syncthreads();
}

// C <- C (I - Vp S Vp^T) for the global column-major M x K block C (ld ldc),
// Vp (K x w reflectors, shared row-major) and S in sm.S; W = C Vp goes
// through P0.
template <int NB>
__device__ void apply_right(BtSmem& sm, Red& rd, float* C, int ldc, int M, int K, const float* Vp, int w) {
  if (M <= 0) return;
  gemm_nn_small<NB>(C, ldc, M, K, Vp, sm.P0);
  mul_tri<NB>(sm.P0, M, sm.S);
  gemm_update(sm, rd, C, ldc, M, K, sm.P0, Vp, w, -1.f, 1.f, 0, false);
}

// SVD of the p x p block in sm.R (column-major, ld LDQ, p <= 32, zero
// outside p x p): one-sided Jacobi (Hestenes) on its columns, R Vs = Ub
// diag(sig), in round-robin order (one warp per pair, pe/2 pairs a round).
// Then the singular values are sorted descending into sm.d, the columns
// permuted, and Us = the normalized columns re-orthonormalized by two
// Gram-Schmidt passes in that order (a column whose projection loses more
// than 99% of its norm, or a zero column, is replaced by the unit vector
// with the largest projection: R = Us D Vs^T then holds to the rounding of
// the largest singular value).  sm.R becomes Us, sm.Vs holds Vs (both zero
// outside p x p).  `tmp` is 2 * 32 * LDQ floats of free shared memory.
// Returns false when max_sweeps sweeps did not converge (outputs written).
__device__ __noinline__ bool small_svd(BtSmem& sm, int p, int max_sweeps, float* tmp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < 32 * LDQ; e += BT_NT) {
    const int r = e % LDQ, c = e / LDQ;
    sm.Vs[e] = (r == c && r < p) ? 1.f : 0.f;
  }
  __syncthreads();
  const int pe = p + (p & 1);
  const float tolj = static_cast<float>(p) * 0x1p-23f;
  bool conv = pe < 2;
  for (int sw = 0; sw < max_sweeps && !conv; ++sw) {
    int rot = 0;
    for (int rr = 0; rr < pe - 1; ++rr) {
      if (warp < pe / 2) {
        // circle method: player pe-1 fixed, the others on a circle of pe-1
        int a, b;
        if (warp == 0) {
          a = pe - 1;
          b = rr;
        } else {
          a = (rr + warp) % (pe - 1);
          b = (rr - warp + (pe - 1)) % (pe - 1);
        }
        if (a > b) {
          const int t = a;
          a = b;
          b = t;
        }
        const float xa = sm.R[a * LDQ + lane], xb = sm.R[b * LDQ + lane];
        const float al = warp_sum(xa * xa), be = warp_sum(xb * xb), ga = warp_sum(xa * xb);
        if (ga != 0.f && fabsf(ga) > tolj * sqrtf(al) * sqrtf(be)) {
          // any t gives an exact rotation as long as c and s agree, so the
          // angle uses the fast division; c = (1 + t^2)^(-1/2) from the
          // hardware reciprocal square root and one Newton step (as accurate
          // as a division by sqrtf)
          const float zeta = __fdividef(be - al, 2.f * ga);
          const float t = __fdividef(copysignf(1.f, zeta), fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
          if (t != 0.f) {
            const float x1 = fmaf(t, t, 1.f);
            float c = rsqrtf(x1);
            c = c * fmaf(-0.5f * x1 * c, c, 1.5f);
            const float s = c * t;
            sm.R[a * LDQ + lane] = c * xa - s * xb;
            sm.R[b * LDQ + lane] = s * xa + c * xb;
            const float va = sm.Vs[a * LDQ + lane], vb = sm.Vs[b * LDQ + lane];
            sm.Vs[a * LDQ + lane] = c * va - s * vb;
            sm.Vs[b * LDQ + lane] = s * va + c * vb;
            rot = 1;
          }
        }
      }
      __syncthreads();
    }
    conv = __syncthreads_or(rot) == 0;
  }
  for (int i = warp; i < p; i += BT_NW) {
    const float xv = sm.R[i * LDQ + lane];
    const float s = warp_sum(xv * xv);
    if (lane == 0) sm.sig[i] = sqrtf(s);
  }
  __syncthreads();
  if (tid < p) {
    const float si = sm.sig[tid];
    int rk = 0;
    for (int j = 0; j < p; ++j) {
      const float sj = sm.sig[j];
      rk += (sj > si) || (sj == si && j < tid);
    }
    sm.rank[tid] = rk;
    sm.d[rk] = si;
  }
  __syncthreads();
  float* Ut = tmp;
  float* Vt = tmp + 32 * LDQ;
  for (int i = warp; i < 32; i += BT_NW) {
    if (i < p) {
      const int k = sm.rank[i];
      const float si = sm.sig[i];
      const float inv = si > 0.f ? 1.f / si : 0.f;
      Ut[k * LDQ + lane] = sm.R[i * LDQ + lane] * inv;
      Vt[k * LDQ + lane] = sm.Vs[i * LDQ + lane];
    } else {
      Ut[i * LDQ + lane] = 0.f;
      Vt[i * LDQ + lane] = 0.f;
    }
  }
  __syncthreads();
  for (int e = tid; e < 32 * LDQ; e += BT_NT) {
    sm.R[e] = (e % LDQ < 32) ? Ut[e] : 0.f;
    sm.Vs[e] = (e % LDQ < 32) ? Vt[e] : 0.f;
  }
  __syncthreads();
  // two Gram-Schmidt passes per column in the sorted order; the products
  // with the earlier columns are spread over the warps (tmp holds them)
  float* dots = tmp;
  for (int k = 0; k < p; ++k) {
    float n0 = 0.f;
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = warp; j < k; j += BT_NW) {
        const float dj = warp_sum(sm.R[j * LDQ + lane] * sm.R[k * LDQ + lane]);
        if (lane == 0) dots[j] = dj;
      }
      __syncthreads();
      if (warp == 0) {
        float u = sm.R[k * LDQ + lane];
        if (pass == 0) n0 = sqrtf(warp_sum(u * u));
        for (int j = 0; j < k; ++j) u = fmaf(-dots[j], sm.R[j * LDQ + lane], u);
        sm.R[k * LDQ + lane] = u;
      }
      __syncthreads();
    }
    if (warp == 0) {
      float u = sm.R[k * LDQ + lane];
      float n1 = sqrtf(warp_sum(u * u));
      if (!(n0 > 0.f) || !(n1 > 0.01f * n0)) {
        // basis completion: the unit vector e_t (t < p) with the largest
        // component outside span(u_0..u_{k-1}); it is at least 1/sqrt(p)
        int best = 0;
        float bn = -1.f;
        for (int t = 0; t < p; ++t) {
          float e = (lane == t) ? 1.f : 0.f;
          for (int j = 0; j < k; ++j) {
            const float qv = sm.R[j * LDQ + lane];
            e = fmaf(-warp_sum(qv * e), qv, e);
          }
          const float en = warp_sum(e * e);
          if (en > bn) {
            bn = en;
            best = t;
          }
        }
        u = (lane == best) ? 1.f : 0.f;
        for (int pass = 0; pass < 2; ++pass)
          for (int j = 0; j < k; ++j) {
            const float qv = sm.R[j * LDQ + lane];
            u = fmaf(-warp_sum(qv * u), qv, u);
          }
        n1 = sqrtf(warp_sum(u * u));
      }
      sm.R[k * LDQ + lane] = (lane < p) ? u / n1 : 0.f;
    }
    __syncthreads();
  }
  __syncthreads();
  return conv;
}

// Load thread r's row of the row-major panel buffer P (r < M) into x.
template <int NB>
__device__ __forceinline__ void load_row(float (&x)[NB], const float* P, int M) {
  const int r = threadIdx.x;
#pragma unroll
  for (int c = 0; c < NB; ++c) x[c] = 0.f;
  if (r < M) {
    const float4* p4 = reinterpret_cast<const float4*>(P + r * LDW);
#pragma unroll
    for (int j = 0; j < NB / 4; ++j) {
      const float4 v = p4[j];
      x[4 * j] = v.x;
      x[4 * j + 1] = v.y;
      x[4 * j + 2] = v.z;
      x[4 * j + 3] = v.w;
    }
  }
}

// Thread r's row of the global column-major block X (rows < M, columns < w;
// with trans the row of X^T, i.e. column r of X).
template <int NB>
__device__ __forceinline__ void load_panel(float (&x)[NB], const float* X, int ld, int M, int w, bool trans) {
  const int r = threadIdx.x;
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    float v = 0.f;
    if (r < M && c < w) v = trans ? X[c + static_cast<int64_t>(r) * ld] : X[r + static_cast<int64_t>(c) * ld];
    x[c] = v;
  }
}

// Zero the global column-major M x N block X (ld).
__device__ void zero_block(float* X, int ld, int M, int N) {
  for (int e = threadIdx.x; e < M * N; e += BT_NT) X[e % M + static_cast<int64_t>(e / M) * ld] = 0.f;
}

// Factor a panel held one row per thread: loaded from the shared row-major
// buffer P (when non-null) or from the global block X (ld, rows M, columns
// w, transposed when trans), factored in registers, its reflectors written
// to Vout and, with want_r, its R to sm.R.
template <int NB>
__device__ __noinline__ void factor_panel(BtSmem& sm, Red& rd, const float* P, const float* X, int ld, bool trans, int M,
                                          int w, float* Vout, bool want_r) {
  float x[NB];
  if (P)
    load_row<NB>(x, P, M);
  else
    load_panel<NB>(x, X, ld, M, w, trans);
  panel_qr_regs<NB>(sm, rd, x, M, w);
  store_panel<NB>(sm, x, M, w, Vout, want_r);
}

// One step of Fig. 4 with both I3 and J3 non-empty, at r0 = b (step - 1).
// Returns ||T(I3, J3)||_F^2 after the step (the next step's trailing block).
template <int NB>
__device__ __noinline__ double regular_step(BtSmem& sm, Red& rd, const BtArgs& g, float* T, float* U, float* V, int m, int n,
                               int b, int r0, int step, int idx, const float* gstep, bool& ok) {
  const int kr = m - r0, kc = n - r0, c1 = r0 + b;
  float* X = T + r0 + static_cast<int64_t>(r0) * m;
  // Section 4.3 steps 1-2: G, then Y = (X^T X)^q X^T G
  fill_gaussian<NB>(sm.P0, kr, b, g.k0, g.k1, static_cast<uint32_t>(step), static_cast<uint32_t>(idx), gstep);
  gemm_tn_small<NB>(sm, X, m, kr, kc, sm.P0, sm.P1);
  for (int it = 0; it < g.q; ++it) {
    gemm_nn_small<NB>(X, m, kr, kc, sm.P1, sm.P0);
    gemm_tn_small<NB>(sm, X, m, kr, kc, sm.P0, sm.P1);
  }
  // Section 4.3 step 3: Householder QR of Y; VV applied to T(:, [J2 J3]) and V
  factor_panel<NB>(sm, rd, sm.P1, nullptr, 0, false, kc, b, sm.P1, false);
  apply_right<NB>(sm, rd, T + static_cast<int64_t>(r0) * m, m, m, kc, sm.P1, b);
  if (g.form_uv) apply_right<NB>(sm, rd, V + static_cast<int64_t>(r0) * n, n, n, kc, sm.P1, b);
  // Remark 1: QR of the new panel T([I2 I3], J2); UU into U and T([I2 I3], J3)
  factor_panel<NB>(sm, rd, nullptr, X, m, false, kr, b, sm.P1, true);
  zero_block(X, m, kr, b);
  if (g.form_uv) apply_right<NB>(sm, rd, U + static_cast<int64_t>(r0) * m, m, m, kr, sm.P1, b);
  float* X13 = T + r0 + static_cast<int64_t>(c1) * m;
  gemm_tn_small<NB>(sm, X13, m, kr, kc - b, sm.P1, sm.P0);
  mul_tri<NB>(sm.P0, kc - b, sm.S);
  const double nxt = gemm_update(sm, rd, X13, m, kr, kc - b, sm.P1, sm.P0, b, -1.f, 1.f, b, true);
  // Fig. 4: SVD of R = Us D Vs^T, rotated into T, U and V
  ok &= small_svd(sm, b, g.max_sweeps, sm.P0);
  if (threadIdx.x < b) X[threadIdx.x + static_cast<int64_t>(threadIdx.x) * m] = sm.d[threadIdx.x];
  stage_cols_t<NB>(X13, m, b, kc - b, sm.P0);
  gemm_update(sm, rd, X13, m, b, kc - b, sm.R, sm.P0, b, 1.f, 0.f, 0, false);
  if (g.form_uv) {
    stage_rows<NB>(U + static_cast<int64_t>(r0) * m, m, m, b, sm.P0);
    gemm_update(sm, rd, U + static_cast<int64_t>(r0) * m, m, m, b, sm.P0, sm.R, b, 1.f, 0.f, 0, false);
  }
  if (r0 > 0) {
    stage_rows<NB>(T + static_cast<int64_t>(r0) * m, m, r0, b, sm.P0);
    gemm_update(sm, rd, T + static_cast<int64_t>(r0) * m, m, r0, b, sm.P0, sm.Vs, b, 1.f, 0.f, 0, false);
  }
  if (g.form_uv) {
    stage_rows<NB>(V + static_cast<int64_t>(r0) * n, n, n, b, sm.P0);
    gemm_update(sm, rd, V + static_cast<int64_t>(r0) * n, n, n, b, sm.P0, sm.Vs, b, 1.f, 0.f, 0, false);
  }
  return nxt;
}

// The last block X = T(r0:m, r0:n) (Fig. 4, else branch): a full SVD, done
// through a QR of the columns when X is tall (Section 5.2, third
// modification) or of the rows when it is wide (Remark on m < n).
template <int NB>
__device__ __noinline__ void final_block(BtSmem& sm, Red& rd, const BtArgs& g, float* T, float* U, float* V, int m, int n,
                            int r0, bool& ok) {
  const int kr = m - r0, kc = n - r0;
  float* X = T + r0 + static_cast<int64_t>(r0) * m;
  int p;
  if (kr > kc) {
    p = kc;
    factor_panel<NB>(sm, rd, nullptr, X, m, false, kr, kc, sm.P1, true);
    if (g.form_uv) apply_right<NB>(sm, rd, U + static_cast<int64_t>(r0) * m, m, m, kr, sm.P1, kc);
  } else if (kr < kc) {
    p = kr;
    factor_panel<NB>(sm, rd, nullptr, X, m, true, kc, kr, sm.P1, true);
    // core L = R^T: transpose sm.R in place
    for (int e = threadIdx.x; e < 32 * 32; e += BT_NT) {
      const int r = e % 32, c = e / 32;
      if (r < c) {
        const float t = sm.R[c * LDQ + r];
        sm.R[c * LDQ + r] = sm.R[r * LDQ + c];
        sm.R[r * LDQ + c] = t;
      }
    }
    __syncthreads();
    if (r0 > 0) apply_right<NB>(sm, rd, T + static_cast<int64_t>(r0) * m, m, r0, kc, sm.P1, kr);
    if (g.form_uv) apply_right<NB>(sm, rd, V + static_cast<int64_t>(r0) * n, n, n, kc, sm.P1, kr);
  } else {
    p = kr;
    for (int e = threadIdx.x; e < 32 * LDQ; e += BT_NT) {
      const int r = e % LDQ, c = e / LDQ;
      sm.R[e] = (r < p && c < p) ? X[r + static_cast<int64_t>(c) * m] : 0.f;
    }
    __syncthreads();
  }
  zero_block(X, m, kr, kc);
  __syncthreads();
  ok &= small_svd(sm, p, g.max_sweeps, sm.P0);
  if (threadIdx.x < p) X[threadIdx.x + static_cast<int64_t>(threadIdx.x) * m] = sm.d[threadIdx.x];
  if (r0 > 0) {
    stage_rows<NB>(T + static_cast<int64_t>(r0) * m, m, r0, p, sm.P0);
    gemm_update(sm, rd, T + static_cast<int64_t>(r0) * m, m, r0, p, sm.P0, sm.Vs, p, 1.f, 0.f, 0, false);
  }
  if (g.form_uv) {
    stage_rows<NB>(U + static_cast<int64_t>(r0) * m, m, m, p, sm.P0);
    gemm_update(sm, rd, U + static_cast<int64_t>(r0) * m, m, m, p, sm.P0, sm.R, p, 1.f, 0.f, 0, false);
    stage_rows<NB>(V + static_cast<int64_t>(r0) * n, n, n, p, sm.P0);
    gemm_update(sm, rd, V + static_cast<int64_t>(r0) * n, n, n, p, sm.P0, sm.Vs, p, 1.f, 0.f, 0, false);
  }
}

// Factor one matrix of the batch (T = A copied, U = V = I, then Fig. 4 with
// the early stop of Section 1.1 (ii)).  Returns the info word.
template <int NB>
__device__ int factor_one(BtSmem& sm, const BtArgs& g, const BMat& mt, int idx, int& kreach) {
  const int m = mt.m, n = mt.n, b = mt.b;
  const float* A = g.A + mt.a;
  float* T = g.T + mt.a;
  float* U = g.form_uv ? g.U + mt.u : nullptr;
  float* V = g.form_uv ? g.V + mt.v : nullptr;
  Red rd;
  float ssf = 0.f;
  for (int e = threadIdx.x; e < m * n; e += BT_NT) {
    const float a = A[e];
    T[e] = a;
    ssf = fmaf(a, a, ssf);
  }
  const double nrmA2 = block_sum_d(sm, rd, static_cast<double>(ssf));
  if (g.form_uv) {
    for (int e = threadIdx.x; e < m * m; e += BT_NT) U[e] = (e % m == e / m) ? 1.f : 0.f;
    for (int e = threadIdx.x; e < n * n; e += BT_NT) V[e] = (e % n == e / n) ? 1.f : 0.f;
  }
  __syncthreads();
  if (!isfinite(nrmA2)) {
    kreach = 0;
    return RANDUTV_ENAN;
  }
  const double thr2 = static_cast<double>(g.tol) * g.tol * nrmA2;
  double cur2 = nrmA2;
  bool ok = true;
  kreach = min(m, n);
  const int nsteps = min((m + b - 1) / b, (n + b - 1) / b);
  int64_t goff = 0;
  for (int i = 1; i <= nsteps; ++i) {
    const int r0 = b * (i - 1);
    if (g.tol > 0.f && cur2 <= thr2) {
      kreach = r0;
      break;
    }
    if (r0 + b < m && r0 + b < n) {
      const float* gstep = g.gin ? g.gin + mt.g + goff : nullptr;
      cur2 = regular_step<NB>(sm, rd, g, T, U, V, m, n, b, r0, i, idx, gstep, ok);
      goff += static_cast<int64_t>(m - r0) * b;
    } else {
      final_block<NB>(sm, rd, g, T, U, V, m, n, r0, ok);
    }
  }
  return ok ? 0 : RANDUTV_ENOCONV;
}

__global__ void __launch_bounds__(BT_NT, 1) batched_kernel(BtArgs g) {
  extern __shared__ __align__(16) unsigned char bt_smem[];
  BtSmem& sm = *reinterpret_cast<BtSmem*>(bt_smem);
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = static_cast<int>(atomicAdd(g.head, 1u));
    __syncthreads();
    const int t = s_item;
    __syncthreads();
    if (t >= g.count) break;
    const int idx = g.order[t];
    const BMat mt = g.tab[idx];
    const unsigned long long t0 = global_ns();
    int kreach = 0;
    const int st = mt.b <= 16 ? factor_one<16>(sm, g, mt, idx, kreach) : factor_one<32>(sm, g, mt, idx, kreach);
    if (threadIdx.x == 0) {
      g.k_out[idx] = kreach;
      if (g.info) g.info[idx] = st;
      if (st) atomicOr(g.err, st == RANDUTV_ENOCONV ? kDevErrNoConv : kDevErrNaN);
      if (g.tns) g.tns[idx] = global_ns() - t0;
    }
  }
  // the last CTA out rewinds the queue for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(g.done, 1u);
    if (prev == gridDim.x - 1) {
      *g.head = 0u;
      *g.done = 0u;
      __threadfence();
    }
  }
}

__global__ void batched_gaussian_kernel(uint32_t k0, uint32_t k1, uint32_t step, uint32_t idx, int k, int w, float* G,
                                        int64_t ldg) {
  const int np = (k + 1) / 2;
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= static_cast<int64_t>(np) * w) return;
  const int p = static_cast<int>(t % np), c = static_cast<int>(t / np);
  const float2 z = box_muller_f32(philox4x32_10(U4{static_cast<uint32_t>(p), static_cast<uint32_t>(c), step, idx}, k0, k1));
  G[2 * p + c * ldg] = z.x;
  if (2 * p + 1 < k) G[2 * p + 1 + c * ldg] = z.y;
}

}  // namespace
}  // namespace rutv

// ---------------------------------------------------------------------------
// Host side: the plan (sizes, block sizes, packed offsets, the device work
// table in queue order) and the entry points.

struct randutv_batched_plan {
  int64_t count = 0;
  int bfix = 0;                       // requested block size (0: per size class)
  int tuned[8] = {32, 32, 32, 32, 32, 32, 32, 32};
  std::vector<int> m, n;
  std::vector<rutv::BMat> tab;
  std::vector<int> order;
  int64_t tot_a = 0, tot_u = 0, tot_v = 0, tot_g = 0;
  rutv::BMat* d_tab = nullptr;
  int* d_order = nullptr;
  unsigned* d_ctr = nullptr;          // {queue head, CTAs done}
  int* d_err = nullptr;
  int grid = 0;
  cudaStream_t ps = nullptr;          // private stream of the graph launches
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaGraphExec_t exec = nullptr;
  rutv::BtArgs key;                   // arguments of the captured graph (compared bytewise)
};

namespace rutv {
namespace {

constexpr size_t kBtSmemBytes = sizeof(BtSmem);
static_assert(sizeof(BtSmem) + 64 <= 232448, "batched kernel shared memory above the per-CTA limit");

int size_class(int m, int n) { return (std::min(m, n) - 1) / 64; }

int64_t gauss_elems(int m, int n, int b) {
  int64_t t = 0;
  for (int i = 1; static_cast<int64_t>(b) * i < std::min(m, n); ++i) t += static_cast<int64_t>(m - b * (i - 1)) * b;
  return t;
}

int bt_status(cudaError_t e) {
  if (e == cudaSuccess) return RANDUTV_OK;
  set_last_error(cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? RANDUTV_ENOMEM : RANDUTV_ECUDA;
}

// Block sizes, offsets and queue order (largest m n min(m, n) first) on the
// host, then the table and order uploaded.
// The host part of a plan: per matrix its block size (the fixed one, else
// its size class's, capped at min(m, n)) and packed offsets, the totals, and
// the queue order (largest m n min(m, n) first, ties by index).
void batched_layout(int64_t c, const int* ms, const int* ns, int bfix, const int* tuned, BMat* tab, int* order,
                    int64_t* totals) {
  int64_t a = 0, u = 0, v = 0, g = 0;
  for (int64_t i = 0; i < c; ++i) {
    const int m = ms[i], n = ns[i];
    const int bb = bfix ? bfix : tuned[size_class(m, n)];
    BMat& t = tab[i];
    t = BMat{};
    t.m = m;
    t.n = n;
    t.b = std::min(bb, std::min(m, n));
    t.a = a;
    t.u = u;
    t.v = v;
    t.g = g;
    a += static_cast<int64_t>(m) * n;
    u += static_cast<int64_t>(m) * m;
    v += static_cast<int64_t>(n) * n;
    g += gauss_elems(m, n, t.b);
  }
  totals[0] = a;
  totals[1] = u;
  totals[2] = v;
  totals[3] = g;
  for (int64_t i = 0; i < c; ++i) order[i] = static_cast<int>(i);
  std::stable_sort(order, order + c, [ms, ns](int x, int y) {
    const double cx = double(ms[x]) * ns[x] * std::min(ms[x], ns[x]);
    const double cy = double(ms[y]) * ns[y] * std::min(ms[y], ns[y]);
    return cx > cy;
  });
}

int relayout(randutv_batched_plan* p) {
  const int64_t c = p->count;
  p->tab.assign(c, BMat{});
  p->order.resize(c);
  int64_t tot[4];
  batched_layout(c, p->m.data(), p->n.data(), p->bfix, p->tuned, p->tab.data(), p->order.data(), tot);
  p->tot_a = tot[0];
  p->tot_u = tot[1];
  p->tot_v = tot[2];
  p->tot_g = tot[3];
  if (c == 0) return RANDUTV_OK;
  // a launch still running (asynchronous calls, on the graph stream or the caller's stream) reads
  // the table: let it finish before the table changes
  cudaError_t e = cudaSuccess;
  if (p->ps) e = cudaStreamSynchronize(p->ps);
  if (e == cudaSuccess) e = cudaStreamSynchronize(current_stream());
  if (e == cudaSuccess) e = cudaMemcpy(p->d_tab, p->tab.data(), sizeof(BMat) * c, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_order, p->order.data(), sizeof(int) * c, cudaMemcpyHostToDevice);
  if (p->exec) {
    cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
  }
  return bt_status(e);
}

void plan_release(randutv_batched_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  if (p->ps) cudaStreamDestroy(p->ps);
  cudaFree(p->d_tab);
  cudaFree(p->d_order);
  cudaFree(p->d_ctr);
  cudaFree(p->d_err);
  delete p;
}

cudaError_t bt_launch(const randutv_batched_plan* p, const BtArgs& a, cudaStream_t s, bool count = true) {
  cudaError_t e = cudaMemsetAsync(p->d_err, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  batched_kernel<<<p->grid, BT_NT, kBtSmemBytes, s>>>(a);
  if (count) note_launch();
  return cudaGetLastError();
}

}  // namespace
}  // namespace rutv

using rutv::BtArgs;

extern "C" {

void randutv_batched_opts_default(randutv_batched_opts* o) {
  if (!o) return;
  o->form_uv = 1;
  o->max_sweeps = 30;
  o->seed = 998;
  o->g_inject = nullptr;
  o->graph = 0;
  o->async = 0;
}

int randutv_batched_plan_create(int64_t count, const int32_t* m, const int32_t* n, int b,
                                randutv_batched_plan** plan) {
  if (count < 0 || count > (int64_t(1) << 31) - 1) return -1;
  if (count > 0 && !m) return -2;
  if (count > 0 && !n) return -3;
  if (b < 0 || b > 32) return -4;
  if (!plan) return -5;
  *plan = nullptr;
  for (int64_t i = 0; i < count; ++i) {
    if (m[i] < 1) return -2;
    if (n[i] < 1) return -3;
  }
  for (int64_t i = 0; i < count; ++i)
    if (m[i] > rutv::BT_MAXD || n[i] > rutv::BT_MAXD) {
      rutv::set_last_error("batched matrices are limited to m, n <= 512");
      return RANDUTV_EUNSUPPORTED;
    }
  auto* p = new (std::nothrow) randutv_batched_plan;
  if (!p) return RANDUTV_ENOMEM;
  std::memset(&p->key, 0, sizeof(p->key));
  p->count = count;
  p->bfix = b;
  p->m.assign(m, m + count);
  p->n.assign(n, n + count);
  const size_t c = static_cast<size_t>(std::max<int64_t>(count, 1));
  cudaError_t e = cudaMalloc(&p->d_tab, sizeof(rutv::BMat) * c);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_order, sizeof(int) * c);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_ctr, 2 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->d_ctr, 0, 2 * sizeof(unsigned));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(rutv::batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(rutv::kBtSmemBytes));
  int dev = 0, sms = 0, per = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, rutv::batched_kernel, rutv::BT_NT, rutv::kBtSmemBytes);
  if (e == cudaSuccess && per < 1) e = cudaErrorInvalidConfiguration;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->ps, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev0, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev1, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    const int st = rutv::bt_status(e);
    rutv::plan_release(p);
    return st;
  }
  p->grid = sms * per;
  const int st = rutv::relayout(p);
  if (st != RANDUTV_OK) {
    rutv::plan_release(p);
    return st;
  }
  *plan = p;
  return RANDUTV_OK;
}

int randutv_batched_layout_host(int64_t count, const int32_t* m, const int32_t* n, int b, const int32_t* b_per_class,
                                int64_t* off_a, int64_t* off_u, int64_t* off_v, int64_t* off_g, int32_t* b_out,
                                int32_t* order, int64_t* totals) {
  if (count < 0 || count > (int64_t(1) << 31) - 1) return -1;
  if (count > 0 && !m) return -2;
  if (count > 0 && !n) return -3;
  if (b < 0 || b > 32) return -4;
  int tuned[8] = {32, 32, 32, 32, 32, 32, 32, 32};
  if (b_per_class)
    for (int cl = 0; cl < 8; ++cl) {
      if (b_per_class[cl] < 1 || b_per_class[cl] > 32) return -5;
      tuned[cl] = b_per_class[cl];
    }
  for (int64_t i = 0; i < count; ++i) {
    if (m[i] < 1) return -2;
    if (n[i] < 1) return -3;
    if (m[i] > rutv::BT_MAXD || n[i] > rutv::BT_MAXD) {
      rutv::set_last_error("batched matrices are limited to m, n <= 512");
      return RANDUTV_EUNSUPPORTED;
    }
  }
  std::vector<rutv::BMat> tab(static_cast<size_t>(count));
  std::vector<int> ord(static_cast<size_t>(count));
  int64_t tot[4];
  rutv::batched_layout(count, m, n, b, tuned, tab.data(), ord.data(), tot);
  for (int64_t i = 0; i < count; ++i) {
    if (off_a) off_a[i] = tab[i].a;
    if (off_u) off_u[i] = tab[i].u;
    if (off_v) off_v[i] = tab[i].v;
    if (off_g) off_g[i] = tab[i].g;
    if (b_out) b_out[i] = tab[i].b;
    if (order) order[i] = ord[i];
  }
  if (totals)
    for (int j = 0; j < 4; ++j) totals[j] = tot[j];
  return RANDUTV_OK;
}

int randutv_batched_plan_destroy(randutv_batched_plan* plan) {
  if (!plan) return -1;
  cudaDeviceSynchronize();
  rutv::plan_release(plan);
  return RANDUTV_OK;
}

int randutv_batched_layout(const randutv_batched_plan* plan, int64_t* off_a, int64_t* off_u, int64_t* off_v,
                           int64_t* off_g, int32_t* b, int64_t* totals) {
  if (!plan) return -1;
  for (int64_t i = 0; i < plan->count; ++i) {
    const rutv::BMat& t = plan->tab[i];
    if (off_a) off_a[i] = t.a;
    if (off_u) off_u[i] = t.u;
    if (off_v) off_v[i] = t.v;
    if (off_g) off_g[i] = t.g;
    if (b) b[i] = t.b;
  }
  if (totals) {
    totals[0] = plan->tot_a;
    totals[1] = plan->tot_u;
    totals[2] = plan->tot_v;
    totals[3] = plan->tot_g;
  }
  return RANDUTV_OK;
}

int randutv_factor_batched(randutv_batched_plan* plan, const float* A, float* T, float* U, float* V, int q, double tol,
                           int32_t* k_reached, int32_t* info, const randutv_batched_opts* opts) {
  randutv_batched_opts o;
  randutv_batched_opts_default(&o);
  if (opts) o = *opts;
  if (!plan) return -1;
  const bool any = plan->count > 0;
  if (any && !A) return -2;
  if (any && !T) return -3;
  if (any && o.form_uv && !U) return -4;
  if (any && o.form_uv && !V) return -5;
  if (q < 0) return -6;
  if (!(tol >= 0.0) || std::isinf(tol)) return -7;
  if (any && !k_reached) return -8;
  if (o.max_sweeps < 1) return -10;
  if (!any) return RANDUTV_OK;
  BtArgs a;
  std::memset(&a, 0, sizeof(a));
  a.tab = plan->d_tab;
  a.order = plan->d_order;
  a.count = static_cast<int>(plan->count);
  a.A = A;
  a.T = T;
  a.U = o.form_uv ? U : nullptr;
  a.V = o.form_uv ? V : nullptr;
  a.gin = o.g_inject;
  a.form_uv = o.form_uv ? 1 : 0;
  a.q = q;
  a.max_sweeps = o.max_sweeps;
  a.tol = static_cast<float>(tol);
  a.k0 = static_cast<uint32_t>(o.seed);
  a.k1 = static_cast<uint32_t>(o.seed >> 32);
  a.k_out = k_reached;
  a.info = info;
  a.err = plan->d_err;
  a.head = plan->d_ctr;
  a.done = plan->d_ctr + 1;
  a.tns = nullptr;
  cudaStream_t s = rutv::current_stream();
  cudaError_t e = cudaSuccess;
  if (o.graph) {
    if (!plan->exec || std::memcmp(&plan->key, &a, sizeof(a)) != 0) {
      if (plan->exec) {
        cudaGraphExecDestroy(plan->exec);
        plan->exec = nullptr;
      }
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(plan->ps, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const cudaError_t le = rutv::bt_launch(plan, a, plan->ps, false);
        e = cudaStreamEndCapture(plan->ps, &graph);
        if (e == cudaSuccess) e = le;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) return rutv::bt_status(e);
      std::memcpy(&plan->key, &a, sizeof(a));
    }
    e = cudaEventRecord(plan->ev0, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->ps, plan->ev0, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(plan->exec, plan->ps);
    if (e == cudaSuccess) rutv::note_launch();
    if (e == cudaSuccess) e = cudaEventRecord(plan->ev1, plan->ps);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, plan->ev1, 0);
  } else {
    // the direct launch shares the queue counters with the graph launches: after the last of them
    e = cudaStreamWaitEvent(s, plan->ev1, 0);
    if (e == cudaSuccess) e = rutv::bt_launch(plan, a, s);
  }
  if (e != cudaSuccess) return rutv::bt_status(e);
  if (o.async) return RANDUTV_OK;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return rutv::bt_status(e);
  int err = 0;
  e = cudaMemcpy(&err, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return rutv::bt_status(e);
  if (err & rutv::kDevErrNaN) return RANDUTV_ENAN;
  if (err & rutv::kDevErrNoConv) return RANDUTV_ENOCONV;
  return RANDUTV_OK;
}

int randutv_batched_autotune(randutv_batched_plan* plan, const float* A, int q, double tol,
                             const randutv_batched_opts* opts, int32_t* choice) {
  randutv_batched_opts o;
  randutv_batched_opts_default(&o);
  if (opts) o = *opts;
  if (!plan) return -1;
  if (plan->count > 0 && !A) return -2;
  if (q < 0) return -3;
  if (!(tol >= 0.0) || std::isinf(tol)) return -4;
  if (o.max_sweeps < 1) return -5;
  const int64_t c = plan->count;
  if (c > 0) {
    float *T = nullptr, *U = nullptr, *V = nullptr;
    int* k = nullptr;
    unsigned long long* tns = nullptr;
    const int64_t ub = o.form_uv ? plan->tot_u : 1, vb = o.form_uv ? plan->tot_v : 1;
    cudaError_t e = cudaMalloc(&T, sizeof(float) * plan->tot_a);
    if (e == cudaSuccess) e = cudaMalloc(&U, sizeof(float) * ub);
    if (e == cudaSuccess) e = cudaMalloc(&V, sizeof(float) * vb);
    if (e == cudaSuccess) e = cudaMalloc(&k, sizeof(int) * c);
    if (e == cudaSuccess) e = cudaMalloc(&tns, sizeof(unsigned long long) * c);
    double tsum[2][8] = {};
    const int cand[2] = {16, 32};
    const int keep_fix = plan->bfix;
    std::vector<unsigned long long> h(c);
    cudaStream_t s = rutv::current_stream();
    for (int ci = 0; ci < 2 && e == cudaSuccess; ++ci) {
      plan->bfix = cand[ci];
      const int st = rutv::relayout(plan);
      if (st != RANDUTV_OK) {
        e = cudaErrorUnknown;
        break;
      }
      BtArgs a;
      std::memset(&a, 0, sizeof(a));
      a.tab = plan->d_tab;
      a.order = plan->d_order;
      a.count = static_cast<int>(c);
      a.A = A;
      a.T = T;
      a.U = o.form_uv ? U : nullptr;
      a.V = o.form_uv ? V : nullptr;
      a.form_uv = o.form_uv ? 1 : 0;
      a.q = q;
      a.max_sweeps = o.max_sweeps;
      a.tol = static_cast<float>(tol);
      a.k0 = static_cast<uint32_t>(o.seed);
      a.k1 = static_cast<uint32_t>(o.seed >> 32);
      a.k_out = k;
      a.err = plan->d_err;
      a.head = plan->d_ctr;
      a.done = plan->d_ctr + 1;
      a.tns = tns;
      e = rutv::bt_launch(plan, a, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e == cudaSuccess) e = cudaMemcpy(h.data(), tns, sizeof(unsigned long long) * c, cudaMemcpyDeviceToHost);
      for (int64_t i = 0; i < c && e == cudaSuccess; ++i)
        tsum[ci][rutv::size_class(plan->m[i], plan->n[i])] += static_cast<double>(h[i]);
    }
    cudaFree(T);
    cudaFree(U);
    cudaFree(V);
    cudaFree(k);
    cudaFree(tns);
    plan->bfix = keep_fix;
    if (e != cudaSuccess) {
      rutv::relayout(plan);
      return rutv::bt_status(e);
    }
    for (int cl = 0; cl < 8; ++cl)
      if (tsum[0][cl] > 0.0 || tsum[1][cl] > 0.0) plan->tuned[cl] = tsum[0][cl] < tsum[1][cl] ? 16 : 32;
  }
  if (choice)
    for (int cl = 0; cl < 8; ++cl) choice[cl] = plan->tuned[cl];
  return rutv::relayout(plan);
}

int randutv_batched_set_classes(randutv_batched_plan* plan, const int32_t* b_per_class) {
  if (!plan) return -1;
  if (!b_per_class) return -2;
  for (int cl = 0; cl < 8; ++cl)
    if (b_per_class[cl] < 1 || b_per_class[cl] > 32) return -2;
  for (int cl = 0; cl < 8; ++cl) plan->tuned[cl] = b_per_class[cl];
  return rutv::relayout(plan);
}

int randutv_batched_gaussian(uint64_t seed, int64_t index, int64_t step, int64_t k, int64_t w, float* G,
                             int64_t ldg) {
  if (index < 0 || index > 0xffffffffll) return -2;
  if (step < 1 || step > 0xffffffffll) return -3;
  if (k < 0 || k > (int64_t(1) << 30)) return -4;
  if (w < 0 || w > (int64_t(1) << 30)) return -5;
  if (!G && k > 0 && w > 0) return -6;
  if (ldg < std::max<int64_t>(1, k)) return -7;
  const int64_t total = (k + 1) / 2 * w;
  if (total == 0) return RANDUTV_OK;
  cudaStream_t s = rutv::current_stream();
  const int threads = 256;
  rutv::batched_gaussian_kernel<<<static_cast<unsigned>((total + threads - 1) / threads), threads, 0, s>>>(
      static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32), static_cast<uint32_t>(step),
      static_cast<uint32_t>(index), static_cast<int>(k), static_cast<int>(w), G, ldg);
  rutv::note_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return rutv::bt_status(e);
}

}  // extern "C"

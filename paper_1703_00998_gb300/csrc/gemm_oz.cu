// FP64 and FP32 GEMMs from BF16 tensor-core products (the Ozaki scheme):
// D = alpha op(A) op(B) + beta D, column-major, for the FP64 form's sketch
// products, block-reflector applications and rotations, and for the mixed
// form's block-reflector applications and rotations (Fig. 4).
//
// FP64 issues at ~4 flop/clk/SM on this GPU (1.2 TFLOP/s), BF16 tensor-core
// products at ~1.9 PFLOP/s.  The scheme trades the FP64 multiply-adds for
// exact integer products:
//   * slicing: each row of op(A) and each column of op(B) is split, per K
//     chunk of OZ_KC = 128, into a power-of-two scale 2^e (|x| < 2^e over the
//     chunk) and OZ_S = 8 integer slices of 7 bits, x = 2^e sum_j s_j 2^-7(j+1)
//     with |s_j| <= 127 (each an exact BF16), truncated after 56 bits;
//   * products: for the 36 slice pairs (s, t) with s + t <= 7, the tensor
//     cores form S_s T_t^T over the chunk and add it into the FP32
//     accumulator of group g = s + t (8 accumulators of 128 x 64 in tensor
//     memory).  Every product is an integer below 2^14 and a group holds at
//     most 8 x 128 of them, below 2^24: the FP32 sums are exact whatever the
//     accumulator's rounding;
//   * epilogue: the 8 exact group sums are combined in 64-bit integers
//     (H = g0 2^14 + g1 2^7 + g2, L = g3 2^28 + ... + g7) and rounded once to
//     FP64: (H 2^35 + L) 2^(eA + eB - 63).
// A chunk's result therefore has the accuracy of an FP64 dot product of
// length 128 with 56-bit inputs (error <= 128 * 2^-55 * max|a| * max|b| over
// the chunk, plus one rounding); longer K is split into chunks whose FP64
// results are summed in FP64 by a reduction kernel.
// The FP32 form (FP32 operands and result) takes 4 slices of 7 bits (28
// bits, above FP32's 24), the 10 pairs with s + t <= 3 in 4 group
// accumulators (128 x 64 tiles), W = g0 2^21 + g1 2^14 + g2 2^7 + g3 and one
// rounding to FP32 per chunk: error <= 128 * 2^-27 * max|a| * max|b| over the
// chunk plus FP32 rounding, the accuracy class of an FP32 GEMM with round-to-
// nearest accumulation (the tensor-core FP32 accumulator's truncation never
// acts: every partial sum is an exact integer below 2^24).
//
// MMA kernel, one CTA per 128 x 64 tile of D and K chunk (192 threads):
//   warp 0 (one thread): TMA loads (128B swizzle, K-major) of the 8 B slices
//     of both 64-wide K sub-blocks (128 KB, resident) and of the 16 A slice
//     sub-blocks through a 4-stage ring (16 KB each);
//   warp 1 (one thread): tcgen05.mma.kind::f16 (BF16 in, FP32 out,
//     M = 128, N = 64, K = 16), A slice s against B slices t <= 7 - s;
//   warps 2-5: tcgen05.ld of the 8 group accumulators, integer combination,
//     FP64 scaling and the alpha/beta update (or FP64 chunk partials).
// Every mbarrier wait is bounded (2 s); on expiry the CTA sets the error
// word, waits (bounded) for its copies in flight, frees its tensor memory
// and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdio>
#include <type_traits>
#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace rutv {
namespace {

constexpr int OZ_KC = 128;         // K chunk: exact FP32 group sums
constexpr int OZ_BM = 128;         // rows of a tile
constexpr int OZ_KB = 64;          // K sub-block: 64 BF16 = 128 bytes = one swizzle row
constexpr int OZ_ASTAGES = 2;
constexpr int OZ_A_BYTES = OZ_BM * OZ_KB * 2;   // 16 KB: one A slice, one sub-block
constexpr int OZ_NT = 192;
static_assert(OZ_KC == 2 * OZ_KB, "two sub-blocks per chunk");

// One form of the scheme: S slices of 7 bits per operand, tiles of 128 x BN,
// operands and result of type T.  S groups x BN columns of tensor memory
// (256 in both forms, so two CTAs share an SM and one's epilogue overlaps
// the other's products).
template <int S_, int BN_, typename T_>
struct OzCfg {
  static constexpr int S = S_, BN = BN_;
  using T = T_;
  static constexpr bool F32 = std::is_same<T_, float>::value;
  static constexpr int W = 7 * S;                           // fixed-point bits of the slices
  static constexpr int B_BYTES = BN * OZ_KB * 2;            // one B slice, one sub-block
  static constexpr int B_ALL = 2 * S * B_BYTES;
  static constexpr int SMEM = B_ALL + OZ_ASTAGES * OZ_A_BYTES + 1024 + 256;
  static constexpr uint32_t TMEM_COLS = S * BN;
  // instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, N = BN, M = 128
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((BN >> 3) << 17) | ((OZ_BM >> 4) << 24);
  static_assert(S * OZ_KC * 127 * 127 < (1 << 24), "group sums exact in FP32");
  static_assert(SMEM <= 113 * 1024 && TMEM_COLS <= 256, "two CTAs per SM");
};
using Oz64 = OzCfg<8, 32, double>;   // 56-bit slices: FP64 products
using Oz32 = OzCfg<4, 64, float>;    // 28-bit slices: FP32 products

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Bit layout of the element types: exponent field position and width, and
// (bias + mantissa bits), so that |x| = mant 2^(max(bexp, 1) - BM) with the
// implicit bit in mant.
template <typename T> struct FBits;
template <> struct FBits<double> {
  static constexpr int MB = 52, EB = 11, BM = 1075, EBIAS = 1022;
  __device__ static long long bits(double x) { return __double_as_longlong(x); }
};
template <> struct FBits<float> {
  static constexpr int MB = 23, EB = 8, BM = 150, EBIAS = 126;
  __device__ static long long bits(float x) { return static_cast<long long>(__float_as_int(x)); }
};

// Slices of an R x K operand X (element (r, k) at X[r + k ldx], or at
// X[k + r ldx] when kcontig), per K chunk: S[(j Rpad + r) Kpad + k] (BF16,
// K contiguous) and e[c Rpad + r].  Rows r >= R and columns k >= K are zero.
// One CTA of 128 threads per 32 rows x one chunk, staged through shared
// memory so that both the reads and the BF16 writes are coalesced.
// Integer arithmetic only (FP64 is the slow pipe here): the scale e is the
// largest biased exponent of the row's chunk minus the bias (so |x| < 2^e),
// and the slices are the 7-bit groups of the W-bit fixed-point magnitude
// trunc(|x| 2^(W - e)), each with the sign of x.
template <int S, typename T>
__global__ void __launch_bounds__(128)
oz_slice_kernel(int64_t R, int64_t K, const T* __restrict__ X, int64_t ldx, bool kcontig, int64_t Rpad,
                int64_t Kpad, __nv_bfloat16* __restrict__ Sl, int* __restrict__ E) {
  using F = FBits<T>;
  constexpr int W = 7 * S;
  __shared__ long long tile[32][OZ_KC + 1];
  __shared__ int s_e[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * 32;
  const int64_t k0 = static_cast<int64_t>(blockIdx.y) * OZ_KC;
  for (int idx = tid; idx < 32 * OZ_KC; idx += 128) {
    int i, kk;
    if (kcontig) { kk = idx % OZ_KC; i = idx / OZ_KC; }
    else { i = idx % 32; kk = idx / 32; }
    const int64_t r = r0 + i, k = k0 + kk;
    T v = T(0);
    if (r < R && k < K) v = kcontig ? X[k + r * ldx] : X[r + k * ldx];
    tile[i][kk] = F::bits(v);
  }
  __syncthreads();
  constexpr long long EMASK = (1ll << F::EB) - 1;
  for (int i = warp; i < 32; i += 4) {
    int be = 0;   // largest biased exponent of the row's chunk
    for (int kk = lane; kk < OZ_KC; kk += 32) be = max(be, static_cast<int>((tile[i][kk] >> F::MB) & EMASK));
    be = __reduce_max_sync(0xffffffffu, be);
    if (lane == 0) s_e[i] = (be == 0) ? 0 : be - F::EBIAS;   // zero (or subnormal-only) row: e = 0
  }
  __syncthreads();
  if (tid < 32 && r0 + tid < Rpad) E[static_cast<int64_t>(blockIdx.y) * Rpad + r0 + tid] = s_e[tid];
  // each warp writes 8 rows; a lane owns 4 consecutive k of a row
  for (int i = warp; i < 32; i += 4) {
    const int64_t r = r0 + i;
    if (r >= Rpad) continue;
    const int e = s_e[i];
    unsigned long long mag[4];
    bool neg[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long b = tile[i][lane * 4 + q];
      const int bexp = static_cast<int>((b >> F::MB) & EMASK);
      neg[q] = (b >> (F::MB + F::EB)) & 1;
      const unsigned long long mant =
          (static_cast<unsigned long long>(b) & ((1ull << F::MB) - 1)) | (bexp ? (1ull << F::MB) : 0ull);
      // |x| = mant 2^(max(bexp,1) - BM); magnitude in units of 2^(e - W)
      const int sh = max(bexp, 1) - (F::BM - W) - e;   // <= 3 (FP64) / 4 (FP32) because |x| < 2^e
      mag[q] = (sh >= 0) ? (mant << sh) : (sh > -64 ? (mant >> (-sh)) : 0ull);
    }
#pragma unroll
    for (int j = 0; j < S; ++j) {
      __nv_bfloat16 out[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int v = static_cast<int>((mag[q] >> (W - 7 * (j + 1))) & 127ull);
        out[q] = __float2bfloat16_rn(static_cast<float>(neg[q] ? -v : v));   // exact: 7 bits
      }
      uint2 pk;
      pk.x = static_cast<uint32_t>(__bfloat16_as_ushort(out[0])) |
             (static_cast<uint32_t>(__bfloat16_as_ushort(out[1])) << 16);
      pk.y = static_cast<uint32_t>(__bfloat16_as_ushort(out[2])) |
             (static_cast<uint32_t>(__bfloat16_as_ushort(out[3])) << 16);
      *reinterpret_cast<uint2*>(Sl + (static_cast<int64_t>(j) * Rpad + r) * Kpad + k0 + lane * 4) = pk;
    }
  }
}

template <class C>
__global__ void __launch_bounds__(OZ_NT, 2)
gemm_oz_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
               const int* __restrict__ eA, const int* __restrict__ eB, int MApad, int NBpad, int64_t M, int64_t N,
               typename C::T alpha, typename C::T beta, typename C::T* __restrict__ D, int64_t ldd,
               typename C::T* __restrict__ part, int* __restrict__ err) {
  using T = typename C::T;
  constexpr int S = C::S, BN = C::BN;
  extern __shared__ __align__(1024) unsigned char oz_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(oz_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  auto tileB = [&](int kb, int t) { return base + (kb * S + t) * C::B_BYTES; };
  auto tileA = [&](int st) { return base + C::B_ALL + st * OZ_A_BYTES; };
  uint64_t* bfull = reinterpret_cast<uint64_t*>(base + C::B_ALL + OZ_ASTAGES * OZ_A_BYTES);   // [2]
  uint64_t* afull = bfull + 2;                 // [OZ_ASTAGES]
  uint64_t* aempty = afull + OZ_ASTAGES;       // [OZ_ASTAGES]
  uint64_t* done = aempty + OZ_ASTAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int s_fail;
  __shared__ int s_eB[BN];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = static_cast<int>(blockIdx.x) * OZ_BM;
  const int n0 = static_cast<int>(blockIdx.y) * BN;
  const int z = static_cast<int>(blockIdx.z);
  constexpr int NA = 2 * S;   // A slice sub-blocks per CTA

  if (tid == 0) {
    s_fail = 0;
    for (int b = 0; b < 2; ++b) mbar_init(&bfull[b], 1);
    for (int st = 0; st < OZ_ASTAGES; ++st) {
      mbar_init(&afull[st], 1);
      mbar_init(&aempty[st], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < BN) s_eB[tid] = eB[static_cast<int64_t>(z) * NBpad + n0 + tid];
  if (warp == 0) {   // the S group accumulators: half of tensor memory, so two CTAs share an SM
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const unsigned long long t0 = global_ns();
  int issued_b = 0, issued_a = 0;
  const int kx0 = z * OZ_KC;

  if (warp == 0 && lane == 0) {
    // producer: B slices of a sub-block, then its S A slices through the ring
    for (int i = 0; i < NA; ++i) {
      const int kb = i / S, s = i % S, st = i % OZ_ASTAGES;
      if (s == 0) {
        mbar_expect_tx(&bfull[kb], S * C::B_BYTES);
        for (int t = 0; t < S; ++t) tma_load_2d(tileB(kb, t), &mapB, kx0 + kb * OZ_KB, t * NBpad + n0, &bfull[kb]);
        ++issued_b;
      }
      if (!mbar_wait(&aempty[st], ((i / OZ_ASTAGES) & 1) ^ 1, t0)) { s_fail = 1; break; }
      mbar_expect_tx(&afull[st], OZ_A_BYTES);
      tma_load_2d(tileA(st), &mapA, kx0 + kb * OZ_KB, s * MApad + m0, &afull[st]);
      ++issued_a;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    uint32_t inited = 0;   // groups that have received their first product
    for (int i = 0; i < NA; ++i) {
      const int kb = i / S, s = i % S, st = i % OZ_ASTAGES;
      if (s == 0 && !mbar_wait(&bfull[kb], 0, t0)) { s_fail = 1; break; }
      if (!mbar_wait(&afull[st], (i / OZ_ASTAGES) & 1, t0)) { s_fail = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t da = kmajor_sw128_desc(smem_u32(tileA(st)));
      for (int t = 0; t + s < S; ++t) {
        const int g = s + t;
        const uint64_t db = kmajor_sw128_desc(smem_u32(tileB(kb, t)));
        const uint32_t dacc = tmem + static_cast<uint32_t>(g * BN);
#pragma unroll
        for (int kk = 0; kk < OZ_KB / 16; ++kk)   // K = 16 per instruction: 32 bytes (+2 in 16 B units)
          mma_bf16(dacc, da + 2ull * kk, db + 2ull * kk, C::IDESC, (((inited >> g) & 1u) || kk > 0) ? 1u : 0u);
        inited |= 1u << g;
      }
      mma_commit(&aempty[st]);
    }
    mma_commit(done);   // arrives once every issued MMA has completed
  }
  __syncwarp();
  const bool epi = warp >= 2;
  {
    const bool waited = epi ? mbar_wait(done, 0, t0) : true;
    if (__all_sync(0xffffffffu, waited) == 0 && lane == 0) s_fail = 1;
  }
  __syncthreads();
  const bool ok = (s_fail == 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (epi && ok) {
    const int quarter = warp & 3;   // the 32 tensor-memory lanes this warp may read
    const int64_t row = m0 + quarter * 32 + lane;
    const int ea = eA[static_cast<int64_t>(z) * MApad + m0 + quarter * 32 + lane];
    for (int c0 = 0; c0 < BN; c0 += 8) {
      uint32_t r[S][8];
#pragma unroll
      for (int g = 0; g < S; ++g)
        tmem_ld8(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + static_cast<uint32_t>(g * BN + c0), r[g]);
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int64_t col = n0 + c0 + j;
          if (col >= N) break;
          long long gi[S];
#pragma unroll
          for (int g = 0; g < S; ++g) gi[g] = static_cast<long long>(__float2int_rn(__uint_as_float(r[g][j])));
          const int sc0 = ea + s_eB[c0 + j];
          T v;
          if constexpr (C::F32) {
            // W 2^-35 = g0 2^-14 + g1 2^-21 + g2 2^-28 + g3 2^-35, |W| < 2^45: one rounding to FP32
            const long long Wv = (gi[0] << 21) + (gi[1] << 14) + (gi[2] << 7) + gi[3];
            v = __ll2float_rn(Wv);
            const int sc = sc0 - 35;
            v = (sc > -126 && sc < 128) ? v * __int_as_float((127 + sc) << 23) : ldexpf(v, sc);
          } else {
            const long long H = (gi[0] << 14) + (gi[1] << 7) + gi[2];
            const long long L = (gi[3] << 28) + (gi[4] << 21) + (gi[5] << 14) + (gi[6] << 7) + gi[7];
            v = fma(static_cast<double>(H), 0x1p35, static_cast<double>(L));   // one rounding
            const int sc = sc0 - 63;
            v = (sc > -1022 && sc < 1023) ? v * __longlong_as_double(static_cast<long long>(1023 + sc) << 52)
                                          : ldexp(v, sc);
          }
          if (part) {
            part[static_cast<int64_t>(z) * M * N + row + col * M] = v;
          } else {
            T* dp = D + row + col * ldd;
            *dp = (beta == T(0)) ? alpha * v : fma(alpha, v, beta * *dp);
          }
        }
      }
    }
  }
  if (!ok && tid == 0) atomicOr(err, kDevErrTimeout);
  // drain: the producer's copies in flight must land before the CTA exits
  if (!ok && warp == 0 && lane == 0) {
    for (int b = 0; b < issued_b; ++b) mbar_wait(&bfull[b], 0, global_ns());
    for (int i = 0; i < issued_a; ++i) mbar_wait(&afull[i % OZ_ASTAGES], (i / OZ_ASTAGES) & 1, global_ns());
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
  }
}

// D = alpha sum_z part[z] + beta D (chunks in order, summed in FP64).
template <typename T>
__global__ void oz_reduce_kernel(int64_t M, int64_t N, int nch, T alpha, const T* __restrict__ part, T beta,
                                 T* __restrict__ D, int64_t ldd) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= M * N) return;
  double s = 0.0;
  for (int z = 0; z < nch; ++z) s += static_cast<double>(part[static_cast<int64_t>(z) * M * N + t]);
  T* dp = D + (t % M) + (t / M) * ldd;
  *dp = (beta == T(0)) ? static_cast<T>(alpha * s) : static_cast<T>(fma(static_cast<double>(alpha), s, static_cast<double>(beta) * static_cast<double>(*dp)));
}

template <typename T>
__global__ void oz_scale_kernel(int64_t M, int64_t N, T beta, T* __restrict__ D, int64_t ldd) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= M * N) return;
  T* dp = D + (t % M) + (t / M) * ldd;
  *dp = (beta == T(0)) ? T(0) : beta * *dp;
}

// 2-D map of a slice array: rows = slices x Rpad, Kpad BF16 per row, box
// 64 (K) x box_rows, 128B swizzle.
bool make_slice_map(CUtensorMap* map, const __nv_bfloat16* ptr, int64_t Kpad, int64_t rows, uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(Kpad), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(Kpad) * 2};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(OZ_KB), box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline int64_t rup(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline size_t al256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct OzLayout {
  int64_t MApad, NBpad, Kpad;
  int nch;
  size_t sa, ea, sb, eb, pt, total;   // byte sizes
};

template <class C>
OzLayout oz_layout(int64_t m, int64_t n, int64_t k) {
  OzLayout L;
  L.nch = static_cast<int>((k + OZ_KC - 1) / OZ_KC);
  L.MApad = rup(m, OZ_BM);
  L.NBpad = rup(n, C::BN);
  L.Kpad = static_cast<int64_t>(L.nch) * OZ_KC;
  L.sa = al256(static_cast<size_t>(C::S) * L.MApad * L.Kpad * 2);
  L.ea = al256(static_cast<size_t>(L.nch) * L.MApad * 4);
  L.sb = al256(static_cast<size_t>(C::S) * L.NBpad * L.Kpad * 2);
  L.eb = al256(static_cast<size_t>(L.nch) * L.NBpad * 4);
  L.pt = L.nch > 1 ? al256(static_cast<size_t>(L.nch) * m * n * sizeof(typename C::T)) : 0;
  L.total = L.sa + L.ea + L.sb + L.eb + L.pt;
  return L;
}

// D (m x n) = alpha op(A) op(B) + beta D, column-major: op(A) = A^T with A
// k x m (ta) or A (m x k); op(B) = B (k x n, !tb) or B^T with B n x k.
// work: oz_layout<C>(m, n, k).total bytes of device memory.
template <class C>
cudaError_t oz_run(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, typename C::T alpha,
                   const typename C::T* A, int64_t lda, const typename C::T* B, int64_t ldb, typename C::T beta,
                   typename C::T* D, int64_t ldd, void* work, size_t work_bytes, int* err, int prof_class) {
  using T = typename C::T;
  if (m <= 0 || n <= 0) return cudaSuccess;
  const ProfToken tok = prof_begin(s, prof_class);
  cudaError_t e = cudaSuccess;
  if (k <= 0) {
    oz_scale_kernel<T><<<static_cast<unsigned>((m * n + 255) / 256), 256, 0, s>>>(m, n, beta, D, ldd);
    note_launch();
    e = cudaGetLastError();
    prof_end(s, tok, 0.0, 2.0 * sizeof(T) * m * n);
    return e;
  }
  const OzLayout L = oz_layout<C>(m, n, k);
  if (work_bytes < L.total || !work) return cudaErrorInvalidValue;
  if (L.MApad * C::S >= (1ll << 31) || L.NBpad * C::S >= (1ll << 31) || L.nch > 65535) return cudaErrorInvalidValue;
  char* w = static_cast<char*>(work);
  auto* SA = reinterpret_cast<__nv_bfloat16*>(w);
  int* EA = reinterpret_cast<int*>(w + L.sa);
  auto* SB = reinterpret_cast<__nv_bfloat16*>(w + L.sa + L.ea);
  int* EB = reinterpret_cast<int*>(w + L.sa + L.ea + L.sb);
  T* part = L.nch > 1 ? reinterpret_cast<T*>(w + L.sa + L.ea + L.sb + L.eb) : nullptr;
  // op(A) rows = the m dimension, K contiguous when ta; op(B) columns = the n
  // dimension, K contiguous when !tb
  oz_slice_kernel<C::S, T><<<dim3(static_cast<unsigned>(L.MApad / 32), static_cast<unsigned>(L.nch)), 128, 0, s>>>(
      m, k, A, lda, ta, L.MApad, L.Kpad, SA, EA);
  oz_slice_kernel<C::S, T><<<dim3(static_cast<unsigned>(L.NBpad / 32), static_cast<unsigned>(L.nch)), 128, 0, s>>>(
      n, k, B, ldb, !tb, L.NBpad, L.Kpad, SB, EB);
  note_launch(2);
  e = cudaGetLastError();
  CUtensorMap ma, mb;
  if (e == cudaSuccess && (!make_slice_map(&ma, SA, L.Kpad, C::S * L.MApad, OZ_BM) ||
                           !make_slice_map(&mb, SB, L.Kpad, C::S * L.NBpad, C::BN)))
    e = cudaErrorInvalidValue;
  static bool attr = false;
  if (e == cudaSuccess && !attr) {
    e = cudaFuncSetAttribute(gemm_oz_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e == cudaSuccess) attr = true;
  }
  if (e == cudaSuccess) {
    dim3 grid(static_cast<unsigned>(L.MApad / OZ_BM), static_cast<unsigned>(L.NBpad / C::BN),
              static_cast<unsigned>(L.nch));
    gemm_oz_kernel<C><<<grid, OZ_NT, C::SMEM, s>>>(ma, mb, EA, EB, static_cast<int>(L.MApad),
                                                   static_cast<int>(L.NBpad), m, n, alpha, beta, D, ldd, part, err);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && part) {
    oz_reduce_kernel<T><<<static_cast<unsigned>((m * n + 255) / 256), 256, 0, s>>>(m, n, L.nch, alpha, part, beta,
                                                                                  D, ldd);
    note_launch();
    e = cudaGetLastError();
  }
  // flops of the product it stands for; bytes: operands once, slices written and read
  prof_end(s, tok, 2.0 * m * n * k,
           sizeof(T) * (m * k + k * n + m * n * (beta != T(0) ? 2.0 : 1.0)) + 2.0 * static_cast<double>(L.sa + L.sb));
  return e;
}

}  // namespace

size_t gemm_oz_work_bytes(int64_t m, int64_t n, int64_t k) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  return oz_layout<Oz64>(m, n, k).total;
}

size_t gemm_oz32_work_bytes(int64_t m, int64_t n, int64_t k) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  return oz_layout<Oz32>(m, n, k).total;
}

bool gemm_oz_supported() { return encode_fn() != nullptr; }

cudaError_t gemm_oz(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                    const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* D, int64_t ldd,
                    void* work, size_t work_bytes, int* err) {
  return oz_run<Oz64>(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, D, ldd, work, work_bytes, err, kProfGemmOz);
}

cudaError_t gemm_oz32(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, float alpha,
                      const float* A, int64_t lda, const float* B, int64_t ldb, float beta, float* D, int64_t ldd,
                      void* work, size_t work_bytes, int* err) {
  return oz_run<Oz32>(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, D, ldd, work, work_bytes, err, kProfGemmOz32);
}

}  // namespace rutv

namespace {

// The ABI entry points: argument checks, scratch from cudaMallocAsync on the
// bound stream, synchronised.
template <typename T>
int oz_abi(const char* name, char transa, char transb, int64_t m, int64_t n, int64_t k, T alpha, const T* A,
           int64_t lda, const T* B, int64_t ldb, T beta, T* C, int64_t ldc) {
  using namespace rutv;
  const bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
  if (!ta && transa != 'N' && transa != 'n') return -1;
  if (!tb && transb != 'N' && transb != 'n') return -2;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (k < 0) return -5;
  if (!A) return -7;
  if (lda < (ta ? k : m) || lda < 1) return -8;
  if (!B) return -9;
  if (ldb < (tb ? n : k) || ldb < 1) return -10;
  if (!C) return -12;
  if (ldc < m) return -13;
  if (!gemm_oz_supported()) {
    char msg[128];
    snprintf(msg, sizeof(msg), "%s: cuTensorMapEncodeTiled is not available", name);
    set_last_error(msg);
    return RANDUTV_EUNSUPPORTED;
  }
  cudaStream_t s = current_stream();
  const size_t wb = std::is_same<T, double>::value ? gemm_oz_work_bytes(m, n, k) : gemm_oz32_work_bytes(m, n, k);
  void* ws = nullptr;
  int herr = 0;
  cudaError_t e = cudaMallocAsync(&ws, wb + 256, s);
  if (e != cudaSuccess) { cudaGetLastError(); return RANDUTV_ENOMEM; }
  int* err = reinterpret_cast<int*>(static_cast<char*>(ws) + wb);
  e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    if constexpr (std::is_same<T, double>::value)
      e = gemm_oz(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, wb, err);
    else
      e = gemm_oz32(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, wb, err);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  cudaFreeAsync(ws, s);
  cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return RANDUTV_ECUDA;
  }
  return (herr & kDevErrTimeout) ? RANDUTV_ETIMEOUT : RANDUTV_OK;
}

}  // namespace

extern "C" int randutv_dgemm_oz(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                                const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                                int64_t ldc) {
  return oz_abi<double>("randutv_dgemm_oz", transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
}

extern "C" int randutv_sgemm_oz(char transa, char transb, int64_t m, int64_t n, int64_t k, float alpha,
                                const float* A, int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                                int64_t ldc) {
  return oz_abi<float>("randutv_sgemm_oz", transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
}

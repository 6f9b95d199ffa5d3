// FP64 and FP32 GEMMs from BF16 tensor-core products (the Ozaki scheme):
// D = alpha op(A) op(B) + beta D, column-major, for the FP64 form's sketch
// products, block-reflector applications and rotations (Fig. 4).
//
// FP64 issues at ~2 DFMA/clk/SM on this GPU (1.2 TFLOP/s), BF16 tensor-core
// products at ~1.9 PFLOP/s.  The scheme trades the FP64 multiply-adds for
// exact integer products:
//   * slicing: each row of op(A) and each column of op(B) is split, per K
//     chunk of OZ_KC = 128, into a power-of-two scale 2^e (|x| < 2^e over the
//     chunk) and S = 8 integer slices of 7 bits, x = 2^e sum_j s_j 2^-7(j+1)
//     with |s_j| <= 127 (each an exact BF16), truncated after 56 bits;
//   * products: for the 36 slice pairs (s, t) with s + t <= 7, the tensor
//     cores form S_s T_t^T over the chunk and add it into the FP32
//     accumulator of group g = s + t.  Every product is an integer below
//     2^14 and group g holds g + 1 pairs x 128 of them, below 2^24: the FP32
//     sums are exact whatever the accumulator's rounding;
//   * combination: the chunk's value is 2^(eA + eB - 63) F with
//     F = sum_g G_g 2^(49 - 7g), |F| < 2^70.  It is added, in 64-bit
//     integers, into a fixed-point accumulator whose unit is
//     2^(NA + NB - 62), where 2^NA bounds the 2-norm of the row over the
//     whole K range (from the chunk scales and an integer bound of each
//     chunk's norm the slicer records: |x| < (|s_0| + 1) 2^(e - 7)) and
//     2^NB that of the column, so that |sum_k a_k b_k| <= |a| |b| < 2^62
//     units (Cauchy-Schwarz) and the accumulator cannot overflow.  F 2^-7
//     is split into its leading part (groups 0-3) and trailing part (groups
//     4-7), each shifted to the accumulator's unit and rounded; all slices
//     of one entry carry its sign, so each part is bounded like F itself;
//   * one rounding to FP64 at the end (integer round-to-nearest-even of the
//     accumulator), then the alpha/beta update.
// The result is at least as accurate as an FP64 GEMM: the slices truncate
// each operand after 56 bits of its chunk's scale (error <= 2 * 128 *
// 2^-55 * max|a| * max|b| per chunk), the accumulator rounds each chunk
// twice to its unit, which is below 2^-60 |a| |b| (against the u sum
// |a_k| |b_k| <= 2^-53 |a| |b| of an FP64 dot product), and the final value
// is rounded once.  Integer additions are associative, so a K range split over
// several CTAs (their accumulators added with integer atomics) gives
// bit-identical results in any order.
//
// FP64 kernel (gemm_ozx_kernel): one CTA per SM (208 KB of shared memory,
// 512 tensor-memory columns), working through a contiguous range of units
// (tile, K chunk) of 128 x BN output tiles (BN = 64 for long K, 48 for short
// K; see OxT):
//   warp 0 (one thread): TMA loads (128B swizzle, K-major): per 64-wide K
//     sub-block, the B slices of the tile's BN columns side by side (one
//     operand of up to 8 BN rows, 2-stage ring) and the A slices of its 128
//     rows one by one (16 KB each, 5- or 7-stage ring);
//   warp 1 (one thread): tcgen05.mma.kind::f16 (BF16 in, FP32 out, M = 128,
//     K = 16): A slice s against the B slices t it pairs with, in one or two
//     instructions (N = BN x slices, split at 256), whose output columns land
//     in the accumulators of groups s, s + 1, .. (tensor-memory columns
//     BN g ..); slices in descending order, so that the next chunk's products
//     start on the top groups while the epilogue is still reading the others;
//   8 or 12 epilogue warps: per chunk, read the group accumulators in pairs
//     (7, 6), (5, 4), (3, 2), (1, 0) (tcgen05.ld), release each pair to the
//     MMA thread, and fold it into the 64-bit accumulators in registers (one
//     row and 32 or 16 columns per thread); at a tile's end, round to FP64
//     and update D, or (when the tile's chunks are split between CTAs) add
//     into the tile's integer accumulator with atomics, the last CTA of the
//     tile doing the update.
// The slice counts are template parameters: 8 and 8 (group 7) for FP64 data,
// 5 (FP64 data, 35 bits) and 4 (FP32 data, exact) up to group 5 for the
// mixed form's sketch.
// The FP32 form (FP32 operands and result: randutv_sgemm_oz) takes 4 slices
// of 7 bits (28 bits, above FP32's 24), the 10 pairs with s + t <= 3 in 4
// group accumulators, one CTA per 128 x 64 tile and K chunk, W = g0 2^21 +
// g1 2^14 + g2 2^7 + g3 rounded once to FP32 per chunk and chunk results
// summed in FP64 by a reduction kernel.
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
constexpr int kOzZeroScale = -2000;  // scale reported for an all-zero chunk (below any FP64 exponent)
static_assert(OZ_KC == 2 * OZ_KB, "two sub-blocks per chunk");

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t oz_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(OZ_BM >> 4) << 24);
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

// Column of the staging tile that holds k of a chunk: the low two bits of k
// rotated by k / 16, so that the 32 lanes of a warp reading k = 4 lane + q
// (q fixed) of one row hit 16 different 8-byte banks per 16 lanes.
__device__ __forceinline__ int oz_swz(int kk) { return (kk & ~3) | (((kk & 3) + (kk >> 4)) & 3); }

// Slices of an R x K operand X (element (r, k) at X[k + r ldx] when KC, the K
// index contiguous, else at X[r + k ldx]), per K chunk: S[(j Rpad + r) Kpad +
// k] (BF16, K contiguous) and e[c Rpad + r].  Rows r >= R and columns k >= K
// are zero.  One CTA of 256 threads per one chunk x 32 rows (grid x = chunk,
// y = row block); a warp owns a
// row at a time and each lane 4 consecutive k of it, so the slices are
// written 8 bytes per lane.  With K strided (column-major X) the chunk is
// first staged through shared memory so that the reads are coalesced.
// Integer arithmetic only (FP64 is the slow pipe here): the scale e is the
// largest biased exponent of the row's chunk minus the bias (so |x| < 2^e),
// and the slices are the 7-bit groups of the W-bit fixed-point magnitude
// trunc(|x| 2^(W - e)), each with the sign of x.  With NS non-null it also
// writes NS[c Rpad + r] = sum_k (|s_0| + 1)^2 over the chunk's entries (0 for
// an all-zero chunk): the chunk's squared 2-norm is below NS 2^(2e - 14),
// since |x| < (|s_0| + 1) 2^(e - 7).
template <int S, typename T, bool KC>
__global__ void __launch_bounds__(256)
oz_slice_kernel(int64_t R, int64_t K, const T* __restrict__ X, int64_t ldx, int64_t Rpad, int64_t Kpad,
                __nv_bfloat16* __restrict__ Sl, int* __restrict__ E, int* __restrict__ NS) {
  using F = FBits<T>;
  constexpr int W = 7 * S;
  constexpr long long EMASK = (1ll << F::EB) - 1;
  __shared__ long long tile[KC ? 1 : 32][KC ? 1 : OZ_KC + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 32;
  const int64_t k0 = static_cast<int64_t>(blockIdx.x) * OZ_KC;
  if constexpr (!KC) {
    for (int idx = tid; idx < 32 * OZ_KC; idx += 256) {
      const int i = idx % 32, kk = idx / 32;
      const int64_t r = r0 + i, k = k0 + kk;
      T v = T(0);
      if (r < R && k < K) v = X[r + k * ldx];
      tile[i][oz_swz(kk)] = F::bits(v);
    }
    __syncthreads();
  }
  for (int i = warp; i < 32; i += 8) {
    const int64_t r = r0 + i;
    if (r >= Rpad) continue;
    long long b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int kk = lane * 4 + q;
      if constexpr (KC) {
        T v = T(0);
        if (r < R && k0 + kk < K) v = X[k0 + kk + r * ldx];
        b[q] = F::bits(v);
      } else {
        b[q] = tile[i][oz_swz(kk)];
      }
    }
    int be = 0;   // largest biased exponent of the row's chunk
#pragma unroll
    for (int q = 0; q < 4; ++q) be = max(be, static_cast<int>((b[q] >> F::MB) & EMASK));
    be = __reduce_max_sync(0xffffffffu, be);
    // a zero (or subnormal-only) chunk reports the scale kOzZeroScale, so that it never sets a
    // row's largest scale; its slices are zero
    const bool zero = (be == 0);
    if (lane == 0) E[static_cast<int64_t>(blockIdx.x) * Rpad + r] = zero ? kOzZeroScale : be - F::EBIAS;
    const int e = zero ? 0 : be - F::EBIAS;
    int nsq = 0;
    unsigned long long mag[4];
    bool neg[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int bexp = static_cast<int>((b[q] >> F::MB) & EMASK);
      neg[q] = (b[q] >> (F::MB + F::EB)) & 1;
      const unsigned long long mant =
          (static_cast<unsigned long long>(b[q]) & ((1ull << F::MB) - 1)) | (bexp ? (1ull << F::MB) : 0ull);
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
        if (j == 0) nsq += (v + 1) * (v + 1);
      }
      uint2 pk;
      pk.x = static_cast<uint32_t>(__bfloat16_as_ushort(out[0])) |
             (static_cast<uint32_t>(__bfloat16_as_ushort(out[1])) << 16);
      pk.y = static_cast<uint32_t>(__bfloat16_as_ushort(out[2])) |
             (static_cast<uint32_t>(__bfloat16_as_ushort(out[3])) << 16);
      *reinterpret_cast<uint2*>(Sl + (static_cast<int64_t>(j) * Rpad + r) * Kpad + k0 + lane * 4) = pk;
    }
    if (NS) {
      nsq = __reduce_add_sync(0xffffffffu, nsq);
      if (lane == 0) NS[static_cast<int64_t>(blockIdx.x) * Rpad + r] = zero ? 0 : nsq;
    }
  }
}

// One slicing launch (S slices of T data; K contiguous or not).
template <int S, typename T>
void slice_launch(cudaStream_t s, int64_t R, int64_t K, const T* X, int64_t ldx, bool kcontig, int64_t Rpad,
                  int64_t Kpad, int nch, __nv_bfloat16* Sl, int* E, int* NS) {
  // chunks vary fastest: CTAs in flight together slice consecutive chunks of
  // the same rows, so each slice row is written as one contiguous run
  const dim3 g(static_cast<unsigned>(nch), static_cast<unsigned>(Rpad / 32));
  if (kcontig) oz_slice_kernel<S, T, true><<<g, 256, 0, s>>>(R, K, X, ldx, Rpad, Kpad, Sl, E, NS);
  else oz_slice_kernel<S, T, false><<<g, 256, 0, s>>>(R, K, X, ldx, Rpad, Kpad, Sl, E, NS);
}

// ============================================================ FP64 form
constexpr int OX_S = 8;                                   // largest slice count of an operand (and groups)
constexpr int OX_A_BYTES = OZ_BM * OZ_KB * 2;             // 16 KB: one A slice, one K sub-block
constexpr int OX_BST = 2;                                 // B ring stages
constexpr int OX_TILE = OZ_BM * 64;                       // outputs of the largest tile (128 x 64)
constexpr int OX_SPLIT_TILES = 2 * kNumSMs;               // tiles whose K range may be split between CTAs
constexpr int kOzWaveCTAs = kNumSMs - 16;                 // CTAs of a one-wave (stream-K) launch

// Tile shapes of the FP64 kernel: 128 x BN outputs.  BN = 64 with 8 epilogue
// warps (32 columns each) for long K, where the products dominate and the
// wider tile re-reads the 128-row operand's slices less; BN = 48 with 12
// epilogue warps (16 columns each) for short K (rank-b updates), where the
// per-tile epilogue dominates and more warps hide its latencies.  Both use
// 208 KB of shared memory and one CTA per SM.
template <int BN_>
struct OxT {
  static constexpr int BN = BN_;
  static constexpr int MT = 256 / BN;                     // B slices one MMA covers (N <= 256)
  static constexpr int BSL = BN * OZ_KB * 2;              // one B slice, one K sub-block
  static constexpr int B_BYTES = OX_S * BSL;              // a B stage: up to 8 slices side by side
  static constexpr int AST = BN == 64 ? 5 : 7;            // A ring stages
  static constexpr int EPI = BN == 64 ? 8 : 12;           // epilogue warps (EPI / 4 per TMEM lane quarter)
  static constexpr int EC = 4 * BN / EPI;                 // columns per epilogue warp: 32 or 16
  static constexpr int NT = 64 + 32 * EPI;                // 320 or 448 threads
  static constexpr int NBAR = 2 * OX_BST + 2 * AST + 2 + OX_S;
  static constexpr int SMEM = OX_BST * B_BYTES + AST * OX_A_BYTES + 1024 + 8 * NBAR + 16;
  static_assert(BN == 64 || BN == 48, "tile widths");
  static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
  static_assert(OX_S * BN <= 512, "the group accumulators fit tensor memory");
  static_assert(BSL % 1024 == 0, "B slices start on swizzle atoms");
};

struct OxParams {
  const int* eA;        // A-role chunk scales e[c RApad + r]
  const int* eB;        // B-role chunk scales
  const int* nA;        // A-role chunk norm bounds (|row chunk|_2^2 < n 2^(2e - 14))
  const int* nB;        // B-role chunk norm bounds
  int RApad, RBpad;     // padded rows of the A-role (x128) and B-role (x64) slice arrays
  int nch;             // K chunks
  int TM, ntiles;       // tiles along the A-role rows; tiles in all (tile = tn TM + tm)
  int upc;              // units (tile, chunk) per CTA
  int swap;             // 1: the tile's A-role rows are D's columns (D^T computed)
  int64_t M, N;         // valid A-role rows, B-role rows
  double alpha, beta;
  double* D;
  int64_t ldd;
  unsigned long long* acc_ws;   // split tiles: OX_TILE integer accumulators per tile (zero between calls)
  int* cnt;                     // split tiles: chunks done per tile (zero between calls)
  int* err;
};

// Bounded mbarrier wait that also gives up once another role of the CTA
// has failed (so a failure does not cascade into one 2 s wait per role).
__device__ __forceinline__ bool ox_wait(uint64_t* bar, uint32_t parity, volatile int* fail) {
  const uint32_t a = smem_u32(bar);
  unsigned long long t0 = 0;
  for (uint32_t spin = 0;; ++spin) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((spin & 255u) == 255u) {
      if (*fail) return false;
      const unsigned long long t = global_ns();
      if (t0 == 0) t0 = t;
      else if (t - t0 > 2000000000ull) { *fail = 1; return false; }
    }
  }
}

__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, uint32_t (&ra)[16], uint32_t (&rb)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(ra[0]), "=r"(ra[1]), "=r"(ra[2]), "=r"(ra[3]), "=r"(ra[4]), "=r"(ra[5]), "=r"(ra[6]), "=r"(ra[7]),
        "=r"(ra[8]), "=r"(ra[9]), "=r"(ra[10]), "=r"(ra[11]), "=r"(ra[12]), "=r"(ra[13]), "=r"(ra[14]), "=r"(ra[15])
      : "r"(ta));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(rb[0]), "=r"(rb[1]), "=r"(rb[2]), "=r"(rb[3]), "=r"(rb[4]), "=r"(rb[5]), "=r"(rb[6]), "=r"(rb[7]),
        "=r"(rb[8]), "=r"(rb[9]), "=r"(rb[10]), "=r"(rb[11]), "=r"(rb[12]), "=r"(rb[13]), "=r"(rb[14]), "=r"(rb[15])
      : "r"(tb));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// An exact group sum (an integer below 2^24 held in FP32) as an integer.
__device__ __forceinline__ int gsum(uint32_t r) { return __float2int_rz(__uint_as_float(r)); }

// round(x 2^-sh) for -62 <= sh <= 62 (halves rounded up; sh <= 0 is an exact left shift of a value
// known to fit), without overflow for |x| < 2^63 - 1.
__device__ __forceinline__ long long shift_round(long long x, int sh) {
  if (sh <= 0) return static_cast<long long>(static_cast<unsigned long long>(x) << (-sh));
  return ((x >> (sh - 1)) + 1) >> 1;
}

constexpr int kOzZeroNorm = -4000;   // norm exponent of an all-zero row or column

// Smallest N with ||x||_2 < 2^N for a row (or column) x of an operand over
// the whole K range, from its chunks' scales e_c and norm bounds n_c
// (||x_c||_2^2 < n_c 2^(2 e_c - 14)): with E the largest e_c and
// s = sum_c n_c 2^(2 (e_c - E) - 14) = m 2^t (m in [1/2, 1)), ||x||^2 <
// 2^(2E + t), so N = E + ceil(t / 2).  Also returns E.
__device__ __forceinline__ int ox_norm_exp(const int* __restrict__ e, const int* __restrict__ ns, int64_t stride,
                                           int64_t idx, int nch, int* emax) {
  int E = kOzZeroScale;
  for (int c = 0; c < nch; ++c) E = max(E, __ldg(e + c * stride + idx));
  *emax = E;
  double sum = 0.0;
  for (int c = 0; c < nch; ++c) {
    const int nc = __ldg(ns + c * stride + idx);
    if (nc > 0) {
      const int k = 2 * (__ldg(e + c * stride + idx) - E) - 14;   // <= -14
      if (k >= -1022) sum += static_cast<double>(nc) * __longlong_as_double(static_cast<long long>(1023 + k) << 52);
    }
  }
  if (sum == 0.0) return kOzZeroNorm;
  const int t = static_cast<int>((__double_as_longlong(sum) >> 52) & 0x7FF) - 1022;   // sum in [2^(t-1), 2^t)
  return E + ((t + 1) >> 1);
}

// a 2^e rounded once to FP64 (round to nearest even), by integer arithmetic
// in the normal range (FP64 conversion only outside it).
__device__ __forceinline__ double fixed_to_double(long long a, int e) {
  if (a == 0) return 0.0;
  const unsigned long long neg = static_cast<unsigned long long>(a) >> 63;
  unsigned long long m = neg ? (0ull - static_cast<unsigned long long>(a)) : static_cast<unsigned long long>(a);
  const int lz = __clzll(static_cast<long long>(m));
  m <<= lz;                                  // bit 63 set
  unsigned long long mant = m >> 11;         // 53 bits with the leading one
  const unsigned long long rem = m & 0x7FFull;
  mant += static_cast<unsigned long long>((rem > 0x400ull) | ((rem == 0x400ull) & (mant & 1ull)));
  const int be = 1023 + 63 - lz + e;        // biased exponent of the leading bit
  if (be < 1 || be > 2045) {   // subnormal or overflowing result: FP64 scaling by exact powers of two
    double v = static_cast<double>(a);
    for (; e > 1000; e -= 1000) v *= 0x1p1000;
    for (; e < -1000; e += 1000) v *= 0x1p-1000;
    return v * __longlong_as_double(static_cast<long long>(1023 + e) << 52);
  }
  return __longlong_as_double(static_cast<long long>((neg << 63) + (static_cast<unsigned long long>(be - 1) << 52) +
                                                     mant));
}

// TMA loads of the 8 B slices of K sub-block x of a CTA's units into ring stage x % OX_BST.
template <int SB, class C>
__device__ __forceinline__ bool ox_load_b(const CUtensorMap* mapB, unsigned char* sB, uint64_t* bfull, uint64_t* bempty,
                                          int nch, int TM, int RBpad, int u0, int x, volatile int* fail) {
  const int u = u0 + (x >> 1), kb = x & 1, tile = u / nch, c = u % nch, tn = tile / TM;
  const int st = x % OX_BST;
  if (!ox_wait(&bempty[st], ((x / OX_BST) & 1) ^ 1, fail)) return false;
  mbar_expect_tx(&bfull[st], SB * C::BSL);
  for (int t = 0; t < SB; ++t)
    tma_load_2d(sB + st * C::B_BYTES + t * C::BSL, mapB, c * OZ_KC + kb * OZ_KB, t * RBpad + tn * C::BN,
                &bfull[st]);
  return true;
}

// SA (SB): slices of the A-role (B-role) operand; GM: the last group formed (pairs s + t <= GM);
// BN: the tile width (OxT).
template <int SA, int SB, int GM, int BN>
__global__ void __launch_bounds__(OxT<BN>::NT, 1)
gemm_ozx_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                const OxParams p) {
  static_assert(SA >= 1 && SA <= OX_S && SB >= 1 && SB <= OX_S && GM < OX_S && GM <= SA + SB - 2, "slices");
  using C = OxT<BN>;
  extern __shared__ __align__(1024) unsigned char ox_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(ox_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* sB = base;                                   // [OX_BST][C::B_BYTES]
  unsigned char* sA = base + OX_BST * C::B_BYTES;             // [C::AST][OX_A_BYTES]
  uint64_t* bfull = reinterpret_cast<uint64_t*>(sA + C::AST * OX_A_BYTES);
  uint64_t* bempty = bfull + OX_BST;
  uint64_t* afull = bempty + OX_BST;
  uint64_t* aempty = afull + C::AST;
  uint64_t* accfull = aempty + C::AST;     // [1]: a chunk's products are complete
  uint64_t* gempty = accfull + 1;          // [OX_S]: group g read by every epilogue warp
  uint64_t* mdone = gempty + OX_S;         // [1]: every product this CTA issued is complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mdone + 1);
  __shared__ int s_fail;
  __shared__ int s_last;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nch = p.nch;
  const int W = p.ntiles * nch;
  const int u0 = static_cast<int>(blockIdx.x) * p.upc;
  const int u1 = min(W, u0 + p.upc);
  const int nx = 2 * max(0, u1 - u0);   // K sub-blocks of this CTA
  volatile int* fail = &s_fail;

  if (tid == 0) {
    s_fail = 0;
    for (int i = 0; i < OX_BST; ++i) { mbar_init(&bfull[i], 1); mbar_init(&bempty[i], 1); }
    for (int i = 0; i < C::AST; ++i) { mbar_init(&afull[i], 1); mbar_init(&aempty[i], 1); }
    mbar_init(accfull, 1);
    mbar_init(mdone, 1);
    for (int g = 0; g < OX_S; ++g) mbar_init(&gempty[g], C::EPI);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  int issued_a = 0, issued_b = 0;

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer: the B slices of sub-block x + 1 right after A slice 7 of sub-block x
      bool ok = nx == 0 || ox_load_b<SB, C>(&mapB, sB, bfull, bempty, nch, p.TM, p.RBpad, u0, 0, fail);
      issued_b = ok && nx > 0 ? 1 : 0;
      for (int x = 0; x < nx && ok; ++x) {
        const int u = u0 + (x >> 1), kb = x & 1, tile = u / nch, c = u % nch, tm = tile % p.TM;
        for (int s = SA - 1; s >= 0 && ok; --s) {
          const int st = issued_a % C::AST;
          if (!ox_wait(&aempty[st], ((issued_a / C::AST) & 1) ^ 1, fail)) { ok = false; break; }
          mbar_expect_tx(&afull[st], OX_A_BYTES);
          tma_load_2d(sA + st * OX_A_BYTES, &mapA, c * OZ_KC + kb * OZ_KB, s * p.RApad + tm * OZ_BM, &afull[st]);
          ++issued_a;
          if (s == SA - 1 && x + 1 < nx) {
            ok = ox_load_b<SB, C>(&mapB, sB, bfull, bempty, nch, p.TM, p.RBpad, u0, x + 1, fail);
            if (ok) ++issued_b;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      int ia = 0, cc = 0;
      bool ok = true;
      for (int x = 0; x < nx && ok; ++x) {
        const int kb = x & 1, sb = x % OX_BST;
        if (!ox_wait(&bfull[sb], (x / OX_BST) & 1, fail)) break;
        const uint64_t bdesc = kmajor_sw128_desc(smem_u32(sB + sb * C::B_BYTES));
        for (int s = SA - 1; s >= 0; --s) {
          const int st = ia % C::AST;
          if (!ox_wait(&afull[st], (ia / C::AST) & 1, fail)) { ok = false; break; }
          const int nt = min(SB, GM + 1 - s);   // B slices t = 0 .. nt - 1 meet A slice s (s + t <= GM)
          // the previous chunk's groups must have been read before this slice writes them first:
          // every group of the top slice, then group s
          if (kb == 0 && cc > 0) {
            const int gtop = (s == SA - 1) ? s + nt - 1 : s;
            bool w = true;
            for (int g = gtop; g >= s && w; --g) w = ox_wait(&gempty[g], (cc - 1) & 1, fail);
            if (!w) { ok = false; break; }
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t adesc = kmajor_sw128_desc(smem_u32(sA + st * OX_A_BYTES));
#pragma unroll
          for (int kk = 0; kk < OZ_KB / 16; ++kk) {   // K = 16 per instruction: 32 bytes (+2 in 16 B units)
            const uint64_t a = adesc + 2ull * kk, b = bdesc + 2ull * kk;
            const uint64_t bstep = C::BSL >> 4;        // one B slice further in the descriptor's address
            if (kb == 0 && kk == 0 && s == SA - 1) {
              // first products of the chunk: every group of the top slice starts from zero
              const int n1 = min(nt, C::MT);
              mma_bf16(tmem + s * BN, a, b, oz_idesc(n1 * BN), 0u);
              if (nt > C::MT)
                mma_bf16(tmem + (s + C::MT) * BN, a, b + C::MT * bstep, oz_idesc((nt - C::MT) * BN), 0u);
            } else if (kb == 0 && kk == 0) {
              // group s starts from zero; groups s + 1 .. already hold this chunk's products of the
              // slices above s
              mma_bf16(tmem + s * BN, a, b, oz_idesc(BN), 0u);
              if (nt > 1) {
                const int n1 = min(nt - 1, C::MT);
                mma_bf16(tmem + (s + 1) * BN, a, b + bstep, oz_idesc(n1 * BN), 1u);
                if (nt > 1 + C::MT)
                  mma_bf16(tmem + (s + 1 + C::MT) * BN, a, b + (1 + C::MT) * bstep,
                           oz_idesc((nt - 1 - C::MT) * BN), 1u);
              }
            } else {
              const int n1 = min(nt, C::MT);
              mma_bf16(tmem + s * BN, a, b, oz_idesc(n1 * BN), 1u);
              if (nt > C::MT)
                mma_bf16(tmem + (s + C::MT) * BN, a, b + C::MT * bstep, oz_idesc((nt - C::MT) * BN), 1u);
            }
          }
          mma_commit(&aempty[st]);
          ++ia;
        }
        if (!ok) break;
        mma_commit(&bempty[sb]);
        if (kb == 1) {
          mma_commit(accfull);
          ++cc;
        }
      }
      // no product may still write tensor memory when it is freed (also after a failure)
      mma_commit(mdone);
      volatile int nofail = 0;
      ox_wait(mdone, 0, &nofail);
    }
  } else {
    // ---- epilogue warps: lanes 32 (warp % 4) .. +31 of tensor memory, columns C::EC h .. + C::EC - 1
    const int ew = warp - 2, q = warp & 3, h = ew >> 2;
    const int rloc = q * 32 + lane;
    const uint32_t tl = tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(h * C::EC);
    // every epilogue warp runs the same sequence of named barriers whatever happens: after a
    // failure (a wait that ran out) the remaining chunks are skipped, not the barriers
    int cc = 0;
    bool ok = true;
    for (int u = u0; u < u1;) {
      const int tile = u / nch, c0 = u % nch, c1 = min(nch, c0 + (u1 - u)), seg = c1 - c0;
      const int tm = tile % p.TM, tn = tile / p.TM;
      const int rowA = tm * OZ_BM + rloc;
      const int colB0 = tn * BN + h * C::EC;
      const int lc = lane & (C::EC - 1);   // the column of this warp's range that the lane describes
      // norm exponents of this row and of the lane's column over the whole K range: the
      // accumulator's unit is 2^(NA + NB - 62) >= |row| |column| 2^-62, so it cannot overflow
      int EA, EBl;   // (largest chunk scales: unused beyond the norm exponents)
      const int NA = ox_norm_exp(p.eA, p.nA, p.RApad, rowA, nch, &EA);
      const int NBl = ox_norm_exp(p.eB, p.nB, p.RBpad, colB0 + lc, nch, &EBl);
      long long acc[C::EC];
#pragma unroll
      for (int j = 0; j < C::EC; ++j) acc[j] = 0;
      for (int c = c0; c < c1 && ok; ++c) {
        // chunk c's F 2^-7 has the unit 2^(eA + eB - 56): shift right by (NA - eA - 6) + (NB - eB)
        const int dA = NA - __ldg(p.eA + static_cast<int64_t>(c) * p.RApad + rowA) - 6;
        const int dBl = NBl - __ldg(p.eB + static_cast<int64_t>(c) * p.RBpad + colB0 + lc);
        // the chunk's shift of each of the columns, one byte each (-62 .. 62, offset by 64)
        // (32-column warps shuffle it when needed instead: registers)
        constexpr bool kPacked = C::EC == 16;
        uint32_t shp[kPacked ? C::EC / 4 : 1];
        if constexpr (kPacked) {
#pragma unroll
          for (int j4 = 0; j4 < C::EC / 4; ++j4) {
            uint32_t wv = 0;
#pragma unroll
            for (int bb = 0; bb < 4; ++bb) {
              const int sh = min(62, max(-62, dA + __shfl_sync(0xffffffffu, dBl, 4 * j4 + bb)));
              wv |= static_cast<uint32_t>(sh + 64) << (8 * bb);
            }
            shp[j4] = wv;
          }
        }
        const bool waited = ox_wait(accfull, cc & 1, fail);
        if (!__all_sync(0xffffffffu, waited)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // F 2^-7 = high + low with high = P0 2^35 + P1 2^21, low = P2 2^7 + (P3 >> 7) and
        // P_i = G_2i 2^7 + G_2i+1 (each an int32); high and low are each rounded once to the
        // accumulator's unit (P3 and P1 wait in `carry` for their partner pair)
        int carry[C::EC];
#pragma unroll 1
        for (int pr = 3; pr >= 0; --pr) {
#pragma unroll
          for (int hh = 0; hh < C::EC / 16; ++hh) {
            uint32_t ra[16], rb[16];
            if (2 * pr + 1 <= GM) {
              tmem_ld16x2(tl + (2 * pr + 1) * BN + hh * 16, tl + (2 * pr) * BN + hh * 16, ra, rb);
            } else {
              // group 2 pr + 1 is not formed (its accumulator is never written): zero
#pragma unroll
              for (int j = 0; j < 16; ++j) ra[j] = 0u;
              if (2 * pr <= GM) tmem_ld16(tl + (2 * pr) * BN + hh * 16, rb);
              else {
#pragma unroll
                for (int j = 0; j < 16; ++j) rb[j] = 0u;
              }
            }
            if (hh == C::EC / 16 - 1) {
              // the pair's accumulators are in registers: release them to the next chunk's products
              asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
              __syncwarp();
              if (lane == 0) { mbar_arrive(&gempty[2 * pr + 1]); mbar_arrive(&gempty[2 * pr]); }
            }
            if (pr == 3) {
#pragma unroll
              for (int j = 0; j < 16; ++j) carry[hh * 16 + j] = ((gsum(rb[j]) << 7) + gsum(ra[j])) >> 7;
            } else if (pr == 1) {
#pragma unroll
              for (int j = 0; j < 16; ++j) carry[hh * 16 + j] = (gsum(rb[j]) << 7) + gsum(ra[j]);
            } else {
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const int jj = hh * 16 + j;
                const int P = (gsum(rb[j]) << 7) + gsum(ra[j]);
                int sh;
                if constexpr (kPacked) sh = static_cast<int>((shp[jj >> 2] >> (8 * (jj & 3))) & 0xFFu) - 64;
                else sh = min(62, max(-62, dA + __shfl_sync(0xffffffffu, dBl, jj)));
                // integer wrap-around is harmless: high + low = F 2^-7 fits (|F| < 2^70 - 2^18)
                const long long t = pr == 2
                    ? (static_cast<long long>(P) << 7) + carry[jj]
                    : static_cast<long long>((static_cast<unsigned long long>(static_cast<long long>(P)) << 35) +
                                             (static_cast<unsigned long long>(static_cast<long long>(carry[jj])) << 21));
                acc[jj] += shift_round(t, sh);
              }
            }
          }
        }
        ++cc;
      }
      bool store = ok;
      if (seg < nch) {
        // K range split between CTAs: integer atomics into the tile's accumulator; the CTA that
        // completes the tile's chunk count reads the sum back, clears it and updates D
        unsigned long long* ws = p.acc_ws + static_cast<int64_t>(tile) * OX_TILE +
                                 static_cast<int64_t>(h * C::EC) * OZ_BM + rloc;
        if (ok) {
#pragma unroll
          for (int j = 0; j < C::EC; ++j) atomicAdd(ws + j * OZ_BM, static_cast<unsigned long long>(acc[j]));
        }
        __threadfence();
        asm volatile("bar.sync 1, %0;" ::"r"(32 * C::EPI) : "memory");
        if (ew == 0 && lane == 0) {
          // a failed CTA does not count its chunks: the tile is then never stored (the call
          // reports the failure)
          const int old = *fail ? 0 : atomicAdd(p.cnt + tile, seg);
          s_last = (!*fail && old + seg == nch) ? 1 : 0;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(32 * C::EPI) : "memory");
        store = s_last != 0;
        if (store) {
          __threadfence();
#pragma unroll
          for (int j = 0; j < C::EC; ++j) acc[j] = static_cast<long long>(__ldcg(ws + j * OZ_BM));
#pragma unroll
          for (int j = 0; j < C::EC; ++j) __stcg(ws + j * OZ_BM, 0ull);
          if (ew == 0 && lane == 0) p.cnt[tile] = 0;
        }
      }
      if (store) {
        // the C reads are issued together, then the rounded values stored; mode: 0 D = v,
        // 1 D = -v, 2 D = C - v, 3 D = C + v, 4 D = alpha v + beta C
        const int mode = p.beta == 0.0 ? (p.alpha == 1.0 ? 0 : (p.alpha == -1.0 ? 1 : 4))
                                       : (p.beta == 1.0 && p.alpha == -1.0 ? 2 : (p.beta == 1.0 && p.alpha == 1.0 ? 3 : 4));
#pragma unroll
        for (int h2 = 0; h2 < C::EC / 16; ++h2) {
          double cv[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int64_t colB = colB0 + h2 * 16 + j;
            cv[j] = 0.0;
            if (mode >= 2 && rowA < p.M && colB < p.N)
              cv[j] = p.swap ? p.D[colB + static_cast<int64_t>(rowA) * p.ldd] : p.D[rowA + colB * p.ldd];
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int jj = h2 * 16 + j;
            const int e = NA + __shfl_sync(0xffffffffu, NBl, jj) - 62;
            const int64_t colB = colB0 + jj;
            if (rowA < p.M && colB < p.N) {
              const double v = fixed_to_double(acc[jj], e);
              double out;
              if (mode == 0) out = v;
              else if (mode == 1) out = -v;
              else if (mode == 2) out = cv[j] - v;
              else if (mode == 3) out = cv[j] + v;
              else out = fma(p.alpha, v, p.beta * cv[j]);
              if (p.swap) p.D[colB + static_cast<int64_t>(rowA) * p.ldd] = out;
              else p.D[rowA + colB * p.ldd] = out;
            }
          }
        }
      }
      u += seg;
    }
  }
  if (warp == 0 && lane == 0 && *fail) {
    // copies in flight must land before the CTA exits: the last load of every stage
    for (int st = 0; st < OX_BST; ++st) {
      int last = -1;
      for (int x = 0; x < issued_b; ++x) if (x % OX_BST == st) last = x;
      if (last >= 0) { volatile int nofail = 0; ox_wait(&bfull[st], (last / OX_BST) & 1, &nofail); }
    }
    for (int st = 0; st < C::AST; ++st) {
      int last = -1;
      for (int i = 0; i < issued_a; ++i) if (i % C::AST == st) last = i;
      if (last >= 0) { volatile int nofail = 0; ox_wait(&afull[st], (last / C::AST) & 1, &nofail); }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && s_fail) atomicOr(p.err, kDevErrTimeout);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// ============================================================ FP32 form
constexpr int OZ_ASTAGES = 2;
constexpr int OZ_A_BYTES = OZ_BM * OZ_KB * 2;   // 16 KB: one A slice, one sub-block
constexpr int OZ_NT = 192;

// S slices of 7 bits per operand, tiles of 128 x BN, operands and result of
// type T; S groups x BN columns of tensor memory.
template <int S_, int BN_, typename T_>
struct OzCfg {
  static constexpr int S = S_, BN = BN_;
  using T = T_;
  static constexpr int W = 7 * S;                           // fixed-point bits of the slices
  static constexpr int B_BYTES = BN * OZ_KB * 2;            // one B slice, one sub-block
  static constexpr int B_ALL = 2 * S * B_BYTES;
  static constexpr int SMEM = B_ALL + OZ_ASTAGES * OZ_A_BYTES + 1024 + 256;
  static constexpr uint32_t TMEM_COLS = S * BN;
  static constexpr uint32_t IDESC = oz_idesc(BN);
  static_assert(S * OZ_KC * 127 * 127 < (1 << 24), "group sums exact in FP32");
  static_assert(SMEM <= 113 * 1024 && TMEM_COLS <= 256, "two CTAs per SM");
};
using Oz32 = OzCfg<4, 64, float>;    // 28-bit slices: FP32 products

// FP32 form: one CTA per 128 x 64 tile of D and K chunk.  warp 0 (one
// thread): TMA loads of the 4 B slices of both 64-wide K sub-blocks
// (resident) and the 8 A slice sub-blocks through a 2-stage ring; warp 1
// (one thread): A slice s against B slices t <= 3 - s into the accumulator
// of group s + t; warps 2-5: the 4 group sums combined in 64-bit integers,
// rounded once to FP32 and scaled (the alpha/beta update, or a chunk partial).
__global__ void __launch_bounds__(OZ_NT, 2)
gemm_oz32_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                 const int* __restrict__ eA, const int* __restrict__ eB, int MApad, int NBpad, int64_t M, int64_t N,
                 float alpha, float beta, float* __restrict__ D, int64_t ldd, float* __restrict__ part,
                 int* __restrict__ err) {
  using C = Oz32;
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
  if (warp == 0) {
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
        for (int kk = 0; kk < OZ_KB / 16; ++kk)
          mma_bf16(dacc, da + 2ull * kk, db + 2ull * kk, C::IDESC, (((inited >> g) & 1u) || kk > 0) ? 1u : 0u);
        inited |= 1u << g;
      }
      mma_commit(&aempty[st]);
    }
    mma_commit(done);
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
    const int quarter = warp & 3;
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
          // W 2^-35 = g0 2^-14 + g1 2^-21 + g2 2^-28 + g3 2^-35, |W| < 2^45: one rounding to FP32
          const long long Wv = (gi[0] << 21) + (gi[1] << 14) + (gi[2] << 7) + gi[3];
          float v = __ll2float_rn(Wv);
          const int sc = ea + s_eB[c0 + j] - 35;
          v = (sc > -126 && sc < 128) ? v * __int_as_float((127 + sc) << 23) : ldexpf(v, sc);
          if (part) {
            part[static_cast<int64_t>(z) * M * N + row + col * M] = v;
          } else {
            float* dp = D + row + col * ldd;
            *dp = (beta == 0.0f) ? alpha * v : fmaf(alpha, v, beta * *dp);
          }
        }
      }
    }
  }
  if (!ok && tid == 0) atomicOr(err, kDevErrTimeout);
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
__global__ void oz32_reduce_kernel(int64_t M, int64_t N, int nch, float alpha, const float* __restrict__ part,
                                   float beta, float* __restrict__ D, int64_t ldd) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= M * N) return;
  double s = 0.0;
  for (int z = 0; z < nch; ++z) s += static_cast<double>(part[static_cast<int64_t>(z) * M * N + t]);
  float* dp = D + (t % M) + (t / M) * ldd;
  *dp = (beta == 0.0f) ? static_cast<float>(alpha * s)
                       : static_cast<float>(fma(static_cast<double>(alpha), s, static_cast<double>(beta) * *dp));
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

// ---------------------------------------------------------------- FP64 host
// Workspace: the split-tile accumulators and counters first (fixed offset;
// zero between calls: each split tile's last CTA clears them), then the
// slices and scales of the call.
constexpr size_t OX_HEAD = static_cast<size_t>(OX_SPLIT_TILES) * OX_TILE * 8 + OX_SPLIT_TILES * 4;

struct OxLayout {
  bool swap;
  int SAs, SBs;              // slices of the A-role and B-role operands
  int64_t RA, RB;            // A-role and B-role rows (valid)
  int64_t RApad, RBpad, Kpad;
  int nch, TN, BN;
  size_t head, sa, ea, sb, eb, total;
};

// sm (sn): slices of op(A) (op(B)).
OxLayout ox_layout(int64_t m, int64_t n, int64_t k, int sm, int sn) {
  OxLayout L;
  L.BN = ((k + OZ_KC - 1) / OZ_KC >= 4) ? 64 : 48;   // see OxT
  L.swap = (n <= 256 && m > n);          // the thin operand takes the 128-row side; the large one is read once
  L.RA = L.swap ? n : m;
  L.RB = L.swap ? m : n;
  L.SAs = L.swap ? sn : sm;
  L.SBs = L.swap ? sm : sn;
  L.nch = static_cast<int>((k + OZ_KC - 1) / OZ_KC);
  L.RApad = rup(L.RA, OZ_BM);
  L.TN = static_cast<int>((L.RB + L.BN - 1) / L.BN);
  L.RBpad = rup(static_cast<int64_t>(L.TN) * L.BN, 32);   // the slicer works on 32-row blocks
  L.Kpad = static_cast<int64_t>(L.nch) * OZ_KC;
  L.head = al256(OX_HEAD);
  L.sa = al256(static_cast<size_t>(L.SAs) * L.RApad * L.Kpad * 2);
  L.ea = al256(2 * static_cast<size_t>(L.nch) * L.RApad * 4);   // scales, then norm bounds
  L.sb = al256(static_cast<size_t>(L.SBs) * L.RBpad * L.Kpad * 2);
  L.eb = al256(2 * static_cast<size_t>(L.nch) * L.RBpad * 4);
  L.total = L.head + L.sa + L.ea + L.sb + L.eb;
  return L;
}

// Slices of an operand: FP64 (f32 = false) or FP32 data, `slices` of them.
void launch_slices(cudaStream_t s, bool f32, int slices, int64_t R, int64_t K, const void* X, int64_t ldx,
                   bool kcontig, int64_t Rpad, int64_t Kpad, int nch, __nv_bfloat16* Sl, int* E, int* NS) {
  if (!f32 && slices == 8)
    slice_launch<8, double>(s, R, K, static_cast<const double*>(X), ldx, kcontig, Rpad, Kpad, nch, Sl, E, NS);
  else if (!f32 && slices == 5)
    slice_launch<5, double>(s, R, K, static_cast<const double*>(X), ldx, kcontig, Rpad, Kpad, nch, Sl, E, NS);
  else
    slice_launch<4, float>(s, R, K, static_cast<const float*>(X), ldx, kcontig, Rpad, Kpad, nch, Sl, E, NS);
  note_launch();
}

PerDeviceOnce g_ozx_attr[4];

template <int SA, int SB, int GM, int BN>
cudaError_t launch_ozx(PerDeviceOnce& attr, unsigned grid, cudaStream_t s, const CUtensorMap& ma, const CUtensorMap& mb,
                       const OxParams& p) {
  using C = OxT<BN>;
  cudaError_t e = per_device_once(attr, [] {
    return cudaFuncSetAttribute(gemm_ozx_kernel<SA, SB, GM, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  });
  if (e != cudaSuccess) return e;
  gemm_ozx_kernel<SA, SB, GM, BN><<<grid, C::NT, C::SMEM, s>>>(ma, mb, p);
  note_launch();
  return cudaGetLastError();
}

// D (m x n, FP64) = alpha op(A) op(B) + beta D, column-major.  op(A) (op(B))
// holds FP32 data when a32 (b32), split into sm (sn) slices; the pairs
// (slices, last group) supported are (8, 8 -> group 7), the FP64 products,
// and (4 FP32, 5 FP64 -> group 5), the sketch of the mixed form.
// keep (optional): a region that holds op(A)'s slices, scales and norm bounds
// instead of the workspace; with keep->ready they are taken as they are (the
// caller vouches that op(A) is unchanged since they were formed), otherwise
// they are formed there and keep->ready is set.
cudaError_t ozx_run(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha, const void* A,
                    int64_t lda, bool a32, int sm, const void* B, int64_t ldb, bool b32, int sn, double beta, double* D,
                    int64_t ldd, void* work, size_t work_bytes, int* err, OzKeep* keep = nullptr) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (k <= 0) {
    const ProfToken tok = prof_begin(s, kProfOther);
    oz_scale_kernel<double><<<static_cast<unsigned>((m * n + 255) / 256), 256, 0, s>>>(m, n, beta, D, ldd);
    note_launch();
    e = cudaGetLastError();
    prof_end(s, tok, 0.0, 16.0 * m * n);
    return e;
  }
  const OxLayout L = ox_layout(m, n, k, sm, sn);
  const bool cfg88 = (L.SAs == 8 && L.SBs == 8), cfg54 = (L.SAs == 5 && L.SBs == 4);
  if (!cfg88 && !cfg54) return cudaErrorInvalidValue;
  if (work_bytes < L.total || !work) return cudaErrorInvalidValue;
  if (L.RApad * OX_S >= (1ll << 31) || L.RBpad * OX_S >= (1ll << 31) || L.Kpad >= (1ll << 31)) return cudaErrorInvalidValue;
  char* w = static_cast<char*>(work);
  auto* acc_ws = reinterpret_cast<unsigned long long*>(w);
  int* cnt = reinterpret_cast<int*>(w + static_cast<size_t>(OX_SPLIT_TILES) * OX_TILE * 8);
  auto* SA = reinterpret_cast<__nv_bfloat16*>(w + L.head);
  int* EA = reinterpret_cast<int*>(w + L.head + L.sa);
  auto* SB = reinterpret_cast<__nv_bfloat16*>(w + L.head + L.sa + L.ea);
  int* EB = reinterpret_cast<int*>(w + L.head + L.sa + L.ea + L.sb);
  if (keep) {
    // op(A)'s arrays in the caller's region, laid out as in the workspace
    const size_t need = L.swap ? L.sb + L.eb : L.sa + L.ea;
    if (!keep->base || keep->bytes < need) return cudaErrorInvalidValue;
    char* kb = static_cast<char*>(keep->base);
    if (L.swap) {
      SB = reinterpret_cast<__nv_bfloat16*>(kb);
      EB = reinterpret_cast<int*>(kb + L.sb);
    } else {
      SA = reinterpret_cast<__nv_bfloat16*>(kb);
      EA = reinterpret_cast<int*>(kb + L.sa);
    }
  }
  int* NA = EA + static_cast<int64_t>(L.nch) * L.RApad;
  int* NB = EB + static_cast<int64_t>(L.nch) * L.RBpad;
  // op(A): rows = the m dimension, K contiguous when ta; op(B): columns = the n dimension, K contiguous when !tb
  const int64_t mpad = L.swap ? L.RBpad : L.RApad, npad = L.swap ? L.RApad : L.RBpad;
  {
    // slicing: operands read once, slices, scales and norm bounds written (bytes of the launches)
    const bool slice_a = !(keep && keep->ready);
    const ProfToken ts = prof_begin(s, kProfOzSlice);
    if (slice_a)
      launch_slices(s, a32, sm, m, k, A, lda, ta, mpad, L.Kpad, L.nch, L.swap ? SB : SA, L.swap ? EB : EA,
                    L.swap ? NB : NA);
    launch_slices(s, b32, sn, n, k, B, ldb, !tb, npad, L.Kpad, L.nch, L.swap ? SA : SB, L.swap ? EA : EB,
                  L.swap ? NA : NB);
    const double a_bytes = (a32 ? 4.0 : 8.0) * m * k + static_cast<double>(L.swap ? L.sb + L.eb : L.sa + L.ea);
    const double b_bytes = (b32 ? 4.0 : 8.0) * k * n + static_cast<double>(L.swap ? L.sa + L.ea : L.sb + L.eb);
    prof_end(s, ts, 0.0, (slice_a ? a_bytes : 0.0) + b_bytes);
    if (keep) keep->ready = true;
  }
  e = cudaGetLastError();
  const ProfToken tok = prof_begin(s, kProfGemmOz);
  CUtensorMap ma, mb;
  if (e == cudaSuccess && (!make_slice_map(&ma, SA, L.Kpad, L.SAs * L.RApad, OZ_BM) ||
                           !make_slice_map(&mb, SB, L.Kpad, L.SBs * L.RBpad, static_cast<uint32_t>(L.BN))))
    e = cudaErrorInvalidValue;
  if (e == cudaSuccess) {
    OxParams p;
    p.eA = EA;
    p.eB = EB;
    p.nA = NA;
    p.nB = NB;
    p.RApad = static_cast<int>(L.RApad);
    p.RBpad = static_cast<int>(L.RBpad);
    p.nch = L.nch;
    p.TM = static_cast<int>(L.RApad / OZ_BM);
    p.ntiles = p.TM * L.TN;
    p.swap = L.swap ? 1 : 0;
    p.M = L.RA;
    p.N = L.RB;
    p.alpha = alpha;
    p.beta = beta;
    p.D = D;
    p.ldd = ldd;
    p.acc_ws = acc_ws;
    p.cnt = cnt;
    p.err = err;
    const int64_t W = static_cast<int64_t>(p.ntiles) * L.nch;
    int64_t grid;
    if (L.nch >= 2 && p.ntiles <= OX_SPLIT_TILES && p.ntiles < 2 * kNumSMs) {
      // few tiles, long K: the (tile, chunk) units spread evenly over one wave, tiles split between CTAs.
      // The wave is 136 CTAs, not 152: the factorization's small SVD holds a 16-CTA cluster for
      // milliseconds on its own lane, and a one-wave kernel with CTAs left over would wait for it.
      grid = std::min<int64_t>(W, kOzWaveCTAs);
      p.upc = static_cast<int>((W + grid - 1) / grid);
    } else {
      // whole tiles per CTA, up to 8, in as few waves as that allows
      const int64_t waves = (p.ntiles + 8ll * kNumSMs - 1) / (8ll * kNumSMs);
      const int64_t tpc = (p.ntiles + waves * kNumSMs - 1) / (waves * kNumSMs);
      p.upc = static_cast<int>(tpc * L.nch);
    }
    grid = (W + p.upc - 1) / p.upc;
    const unsigned gu = static_cast<unsigned>(grid);
    if (cfg88) e = L.BN == 64 ? launch_ozx<8, 8, 7, 64>(g_ozx_attr[0], gu, s, ma, mb, p)
                              : launch_ozx<8, 8, 7, 48>(g_ozx_attr[1], gu, s, ma, mb, p);
    else e = L.BN == 64 ? launch_ozx<5, 4, 5, 64>(g_ozx_attr[2], gu, s, ma, mb, p)
                        : launch_ozx<5, 4, 5, 48>(g_ozx_attr[3], gu, s, ma, mb, p);
  }
  // flops: the BF16 slice-pair products (2 m n k each); bytes: the slices read once, D written (and read)
  const double pairs = cfg88 ? 36.0 : 17.0;
  prof_end(s, tok, pairs * 2.0 * m * n * k,
           static_cast<double>(L.sa + L.sb) + 8.0 * m * n * (beta != 0.0 ? 2.0 : 1.0));
  return e;
}

// ---------------------------------------------------------------- FP32 host
struct OzLayout {
  int64_t MApad, NBpad, Kpad;
  int nch;
  size_t sa, ea, sb, eb, pt, total;   // byte sizes
};

OzLayout oz32_layout(int64_t m, int64_t n, int64_t k) {
  using C = Oz32;
  OzLayout L;
  L.nch = static_cast<int>((k + OZ_KC - 1) / OZ_KC);
  L.MApad = rup(m, OZ_BM);
  L.NBpad = rup(n, C::BN);
  L.Kpad = static_cast<int64_t>(L.nch) * OZ_KC;
  L.sa = al256(static_cast<size_t>(C::S) * L.MApad * L.Kpad * 2);
  L.ea = al256(static_cast<size_t>(L.nch) * L.MApad * 4);
  L.sb = al256(static_cast<size_t>(C::S) * L.NBpad * L.Kpad * 2);
  L.eb = al256(static_cast<size_t>(L.nch) * L.NBpad * 4);
  L.pt = L.nch > 1 ? al256(static_cast<size_t>(L.nch) * m * n * sizeof(float)) : 0;
  L.total = L.sa + L.ea + L.sb + L.eb + L.pt;
  return L;
}

PerDeviceOnce g_oz32_attr;

cudaError_t oz32_run(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, float alpha, const float* A,
                     int64_t lda, const float* B, int64_t ldb, float beta, float* D, int64_t ldd, void* work,
                     size_t work_bytes, int* err) {
  using C = Oz32;
  if (m <= 0 || n <= 0) return cudaSuccess;
  const ProfToken tok = prof_begin(s, kProfGemmOz32);
  cudaError_t e = cudaSuccess;
  if (k <= 0) {
    oz_scale_kernel<float><<<static_cast<unsigned>((m * n + 255) / 256), 256, 0, s>>>(m, n, beta, D, ldd);
    note_launch();
    e = cudaGetLastError();
    prof_end(s, tok, 0.0, 8.0 * m * n);
    return e;
  }
  const OzLayout L = oz32_layout(m, n, k);
  if (work_bytes < L.total || !work) return cudaErrorInvalidValue;
  if (L.MApad * C::S >= (1ll << 31) || L.NBpad * C::S >= (1ll << 31) || L.nch > 65535) return cudaErrorInvalidValue;
  char* w = static_cast<char*>(work);
  auto* SA = reinterpret_cast<__nv_bfloat16*>(w);
  int* EA = reinterpret_cast<int*>(w + L.sa);
  auto* SB = reinterpret_cast<__nv_bfloat16*>(w + L.sa + L.ea);
  int* EB = reinterpret_cast<int*>(w + L.sa + L.ea + L.sb);
  float* part = L.nch > 1 ? reinterpret_cast<float*>(w + L.sa + L.ea + L.sb + L.eb) : nullptr;
  slice_launch<C::S, float>(s, m, k, A, lda, ta, L.MApad, L.Kpad, L.nch, SA, EA, nullptr);
  slice_launch<C::S, float>(s, n, k, B, ldb, !tb, L.NBpad, L.Kpad, L.nch, SB, EB, nullptr);
  note_launch(2);
  e = cudaGetLastError();
  CUtensorMap ma, mb;
  if (e == cudaSuccess && (!make_slice_map(&ma, SA, L.Kpad, C::S * L.MApad, OZ_BM) ||
                           !make_slice_map(&mb, SB, L.Kpad, C::S * L.NBpad, C::BN)))
    e = cudaErrorInvalidValue;
  if (e == cudaSuccess)
    e = per_device_once(g_oz32_attr, [] {
      return cudaFuncSetAttribute(gemm_oz32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    });
  if (e == cudaSuccess) {
    dim3 grid(static_cast<unsigned>(L.MApad / OZ_BM), static_cast<unsigned>(L.NBpad / C::BN),
              static_cast<unsigned>(L.nch));
    gemm_oz32_kernel<<<grid, OZ_NT, C::SMEM, s>>>(ma, mb, EA, EB, static_cast<int>(L.MApad), static_cast<int>(L.NBpad),
                                                  m, n, alpha, beta, D, ldd, part, err);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && part) {
    oz32_reduce_kernel<<<static_cast<unsigned>((m * n + 255) / 256), 256, 0, s>>>(m, n, L.nch, alpha, part, beta, D,
                                                                                 ldd);
    note_launch();
    e = cudaGetLastError();
  }
  prof_end(s, tok, 2.0 * m * n * k,
           4.0 * (m * k + k * n + m * n * (beta != 0.0f ? 2.0 : 1.0)) + 2.0 * static_cast<double>(L.sa + L.sb));
  return e;
}

}  // namespace

size_t gemm_oz_work_bytes(int64_t m, int64_t n, int64_t k) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  return ox_layout(m, n, k, 8, 8).total;
}

size_t gemm_oz_sketch_work_bytes(int64_t m, int64_t n, int64_t k) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  return ox_layout(m, n, k, 4, 5).total;
}

size_t gemm_oz_keep_bytes(int64_t m, int64_t n, int64_t k, bool sketch) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  const OxLayout L = ox_layout(m, n, k, sketch ? 4 : 8, sketch ? 5 : 8);
  return L.swap ? L.sb + L.eb : L.sa + L.ea;
}

cudaError_t gemm_oz_keep(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                         const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* D,
                         int64_t ldd, void* work, size_t work_bytes, int* err, OzKeep* keep) {
  return ozx_run(s, ta, tb, m, n, k, alpha, A, lda, false, 8, B, ldb, false, 8, beta, D, ldd, work, work_bytes, err,
                 keep);
}

size_t gemm_oz_head_bytes() { return al256(OX_HEAD); }

size_t gemm_oz32_work_bytes(int64_t m, int64_t n, int64_t k) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  return oz32_layout(m, n, k).total;
}

bool gemm_oz_supported() { return encode_fn() != nullptr; }

cudaError_t gemm_oz(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                    const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* D, int64_t ldd,
                    void* work, size_t work_bytes, int* err) {
  return ozx_run(s, ta, tb, m, n, k, alpha, A, lda, false, 8, B, ldb, false, 8, beta, D, ldd, work, work_bytes, err);
}

cudaError_t gemm_oz_sketch(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, const float* A,
                           int64_t lda, const double* B, int64_t ldb, double* D, int64_t ldd, void* work,
                           size_t work_bytes, int* err, OzKeep* keep) {
  return ozx_run(s, ta, tb, m, n, k, 1.0, A, lda, true, 4, B, ldb, false, 5, 0.0, D, ldd, work, work_bytes, err,
                 keep);
}

cudaError_t gemm_oz32(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, float alpha,
                      const float* A, int64_t lda, const float* B, int64_t ldb, float beta, float* D, int64_t ldd,
                      void* work, size_t work_bytes, int* err) {
  return oz32_run(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, D, ldd, work, work_bytes, err);
}

}  // namespace rutv

namespace {

// The ABI entry points: argument checks, scratch from cudaMallocAsync on the
// bound stream (the FP64 form's split-tile head cleared), synchronised.
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
  constexpr bool F64 = std::is_same<T, double>::value;
  cudaStream_t s = current_stream();
  const size_t wb = F64 ? gemm_oz_work_bytes(m, n, k) : gemm_oz32_work_bytes(m, n, k);
  void* ws = nullptr;
  int herr = 0;
  cudaError_t e = cudaMallocAsync(&ws, wb + 256, s);
  if (e != cudaSuccess) { cudaGetLastError(); return RANDUTV_ENOMEM; }
  int* err = reinterpret_cast<int*>(static_cast<char*>(ws) + wb);
  e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess && F64 && wb > 0) e = cudaMemsetAsync(ws, 0, gemm_oz_head_bytes(), s);
  if (e == cudaSuccess) {
    if constexpr (F64)
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
    char msg[192];
    snprintf(msg, sizeof(msg), "%s: %s", name, cudaGetErrorString(e));
    set_last_error(msg);
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

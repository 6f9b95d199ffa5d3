// FP64 GEMM from BF16 tensor-core products (the Ozaki scheme): D = alpha
// op(A) op(B) + beta D, column-major FP64, for the FP64 form's sketch
// products, block-reflector applications and rotations (Fig. 4).
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
#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace rutv {
namespace {

constexpr int OZ_S = 8;            // slices per operand, 7 bits each
constexpr int OZ_KC = 128;         // K chunk: exact FP32 group sums
constexpr int OZ_BM = 128, OZ_BN = 32;   // 128 x 32 tiles: two CTAs per SM
constexpr int OZ_KB = 64;          // K sub-block: 64 BF16 = 128 bytes = one swizzle row
constexpr int OZ_ASTAGES = 2;
constexpr int OZ_A_BYTES = OZ_BM * OZ_KB * 2;   // 16 KB: one A slice, one sub-block
constexpr int OZ_B_BYTES = OZ_BN * OZ_KB * 2;   // 4 KB: one B slice, one sub-block
constexpr int OZ_NT = 192;
constexpr int OZ_B_ALL = 2 * OZ_S * OZ_B_BYTES; // 64 KB
constexpr int OZ_SMEM = OZ_B_ALL + OZ_ASTAGES * OZ_A_BYTES + 1024 + 256;
constexpr uint32_t OZ_TMEM_COLS = OZ_S * OZ_BN; // 8 groups x 32 columns = 256 (half of an SM's)
static_assert(OZ_KC == 2 * OZ_KB, "two sub-blocks per chunk");
static_assert(OZ_S * OZ_KC * 127 * 127 < (1 << 24), "group sums exact in FP32");

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major,
// N = 64, M = 128.
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((OZ_BN >> 3) << 17) | ((OZ_BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(kIdescBf16), "r"(accumulate)
      : "memory");
}

// Slices of an R x K operand X (element (r, k) at X[r + k ldx], or at
// X[k + r ldx] when kcontig), per K chunk: S[(j Rpad + r) Kpad + k] (BF16,
// K contiguous) and e[c Rpad + r].  Rows r >= R and columns k >= K are zero.
// One CTA of 128 threads per 32 rows x one chunk, staged through shared
// memory so that both the FP64 reads and the BF16 writes are coalesced.
// Integer arithmetic only (FP64 is the slow pipe here): the scale e is the
// largest biased exponent of the row's chunk minus 1022 (so |x| < 2^e), and
// the slices are the 7-bit groups of the 56-bit fixed-point magnitude
// trunc(|x| 2^(56 - e)), each with the sign of x.
__global__ void __launch_bounds__(128)
oz_slice_kernel(int64_t R, int64_t K, const double* __restrict__ X, int64_t ldx, bool kcontig, int64_t Rpad,
                int64_t Kpad, __nv_bfloat16* __restrict__ S, int* __restrict__ E) {
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
    double v = 0.0;
    if (r < R && k < K) v = kcontig ? X[k + r * ldx] : X[r + k * ldx];
    tile[i][kk] = __double_as_longlong(v);
  }
  __syncthreads();
  for (int i = warp; i < 32; i += 4) {
    int be = 0;   // largest biased exponent of the row's chunk
    for (int kk = lane; kk < OZ_KC; kk += 32) be = max(be, static_cast<int>((tile[i][kk] >> 52) & 0x7ff));
    be = __reduce_max_sync(0xffffffffu, be);
    if (lane == 0) s_e[i] = (be == 0) ? 0 : be - 1022;   // zero (or subnormal-only) row: e = 0
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
      const long long bits = tile[i][lane * 4 + q];
      const int bexp = static_cast<int>((bits >> 52) & 0x7ff);
      neg[q] = bits < 0;
      const unsigned long long mant =
          (static_cast<unsigned long long>(bits) & 0xFFFFFFFFFFFFFull) | (bexp ? (1ull << 52) : 0ull);
      // |x| = mant 2^(max(bexp,1) - 1075); magnitude in units of 2^(e - 56)
      const int sh = max(bexp, 1) - 1019 - e;   // <= 3 because |x| < 2^e
      mag[q] = (sh >= 0) ? (mant << sh) : (sh > -64 ? (mant >> (-sh)) : 0ull);
    }
#pragma unroll
    for (int j = 0; j < OZ_S; ++j) {
      __nv_bfloat16 out[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int v = static_cast<int>((mag[q] >> (49 - 7 * j)) & 127ull);
        out[q] = __float2bfloat16_rn(static_cast<float>(neg[q] ? -v : v));   // exact: 7 bits
      }
      uint2 pk;
      pk.x = static_cast<uint32_t>(__bfloat16_as_ushort(out[0])) |
             (static_cast<uint32_t>(__bfloat16_as_ushort(out[1])) << 16);
      pk.y = static_cast<uint32_t>(__bfloat16_as_ushort(out[2])) |
             (static_cast<uint32_t>(__bfloat16_as_ushort(out[3])) << 16);
      *reinterpret_cast<uint2*>(S + (static_cast<int64_t>(j) * Rpad + r) * Kpad + k0 + lane * 4) = pk;
    }
  }
}

__global__ void __launch_bounds__(OZ_NT, 2)
gemm_oz_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
               const int* __restrict__ eA, const int* __restrict__ eB, int MApad, int NBpad, int64_t M, int64_t N,
               double alpha, double beta, double* __restrict__ D, int64_t ldd, double* __restrict__ part,
               int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char oz_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(oz_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  auto tileB = [&](int kb, int t) { return base + (kb * OZ_S + t) * OZ_B_BYTES; };
  auto tileA = [&](int st) { return base + OZ_B_ALL + st * OZ_A_BYTES; };
  uint64_t* bfull = reinterpret_cast<uint64_t*>(base + OZ_B_ALL + OZ_ASTAGES * OZ_A_BYTES);   // [2]
  uint64_t* afull = bfull + 2;                 // [OZ_ASTAGES]
  uint64_t* aempty = afull + OZ_ASTAGES;       // [OZ_ASTAGES]
  uint64_t* done = aempty + OZ_ASTAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int s_fail;
  __shared__ int s_eB[OZ_BN];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = static_cast<int>(blockIdx.x) * OZ_BM;
  const int n0 = static_cast<int>(blockIdx.y) * OZ_BN;
  const int z = static_cast<int>(blockIdx.z);
  constexpr int NA = 2 * OZ_S;   // A slice sub-blocks per CTA

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
  if (tid < OZ_BN) s_eB[tid] = eB[static_cast<int64_t>(z) * NBpad + n0 + tid];
  if (warp == 0) {   // all 512 columns: the 8 group accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(OZ_TMEM_COLS)
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
    // producer: B slices of a sub-block, then its 8 A slices through the ring
    for (int i = 0; i < NA; ++i) {
      const int kb = i / OZ_S, s = i % OZ_S, st = i % OZ_ASTAGES;
      if (s == 0) {
        mbar_expect_tx(&bfull[kb], OZ_S * OZ_B_BYTES);
        for (int t = 0; t < OZ_S; ++t) tma_load_2d(tileB(kb, t), &mapB, kx0 + kb * OZ_KB, t * NBpad + n0, &bfull[kb]);
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
      const int kb = i / OZ_S, s = i % OZ_S, st = i % OZ_ASTAGES;
      if (s == 0 && !mbar_wait(&bfull[kb], 0, t0)) { s_fail = 1; break; }
      if (!mbar_wait(&afull[st], (i / OZ_ASTAGES) & 1, t0)) { s_fail = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t da = kmajor_sw128_desc(smem_u32(tileA(st)));
      for (int t = 0; t + s < OZ_S; ++t) {
        const int g = s + t;
        const uint64_t db = kmajor_sw128_desc(smem_u32(tileB(kb, t)));
        const uint32_t dacc = tmem + static_cast<uint32_t>(g * OZ_BN);
#pragma unroll
        for (int kk = 0; kk < OZ_KB / 16; ++kk)   // K = 16 per instruction: 32 bytes (+2 in 16 B units)
          mma_bf16(dacc, da + 2ull * kk, db + 2ull * kk, (((inited >> g) & 1u) || kk > 0) ? 1u : 0u);
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
    for (int c0 = 0; c0 < OZ_BN; c0 += 8) {
      uint32_t r[OZ_S][8];
#pragma unroll
      for (int g = 0; g < OZ_S; ++g)
        tmem_ld8(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + static_cast<uint32_t>(g * OZ_BN + c0), r[g]);
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int64_t col = n0 + c0 + j;
          if (col >= N) break;
          long long gi[OZ_S];
#pragma unroll
          for (int g = 0; g < OZ_S; ++g) gi[g] = static_cast<long long>(__float2int_rn(__uint_as_float(r[g][j])));
          const long long H = (gi[0] << 14) + (gi[1] << 7) + gi[2];
          const long long L = (gi[3] << 28) + (gi[4] << 21) + (gi[5] << 14) + (gi[6] << 7) + gi[7];
          double v = fma(static_cast<double>(H), 0x1p35, static_cast<double>(L));   // one rounding
          const int sc = ea + s_eB[c0 + j] - 63;
          v = (sc > -1022 && sc < 1023) ? v * __longlong_as_double(static_cast<long long>(1023 + sc) << 52)
                                        : ldexp(v, sc);
          if (part) {
            part[static_cast<int64_t>(z) * M * N + row + col * M] = v;
          } else {
            double* dp = D + row + col * ldd;
            *dp = (beta == 0.0) ? alpha * v : fma(alpha, v, beta * *dp);
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
  }
}

// D = alpha sum_z part[z] + beta D (FP64, chunks in order).
__global__ void oz_reduce_kernel(int64_t M, int64_t N, int nch, double alpha, const double* __restrict__ part,
                                 double beta, double* __restrict__ D, int64_t ldd) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= M * N) return;
  double s = 0.0;
  for (int z = 0; z < nch; ++z) s += part[static_cast<int64_t>(z) * M * N + t];
  double* dp = D + (t % M) + (t / M) * ldd;
  *dp = (beta == 0.0) ? alpha * s : fma(alpha, s, beta * *dp);
}

__global__ void oz_scale_kernel(int64_t M, int64_t N, double beta, double* __restrict__ D, int64_t ldd) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= M * N) return;
  double* dp = D + (t % M) + (t / M) * ldd;
  *dp = (beta == 0.0) ? 0.0 : beta * *dp;
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

OzLayout oz_layout(int64_t m, int64_t n, int64_t k) {
  OzLayout L;
  L.nch = static_cast<int>((k + OZ_KC - 1) / OZ_KC);
  L.MApad = rup(m, OZ_BM);
  L.NBpad = rup(n, OZ_BN);
  L.Kpad = static_cast<int64_t>(L.nch) * OZ_KC;
  L.sa = al256(static_cast<size_t>(OZ_S) * L.MApad * L.Kpad * 2);
  L.ea = al256(static_cast<size_t>(L.nch) * L.MApad * 4);
  L.sb = al256(static_cast<size_t>(OZ_S) * L.NBpad * L.Kpad * 2);
  L.eb = al256(static_cast<size_t>(L.nch) * L.NBpad * 4);
  L.pt = L.nch > 1 ? al256(static_cast<size_t>(L.nch) * m * n * 8) : 0;
  L.total = L.sa + L.ea + L.sb + L.eb + L.pt;
  return L;
}

}  // namespace

size_t gemm_oz_work_bytes(int64_t m, int64_t n, int64_t k) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  return oz_layout(m, n, k).total;
}

bool gemm_oz_supported() { return encode_fn() != nullptr; }

// D (m x n) = alpha op(A) op(B) + beta D, FP64 column-major: op(A) = A^T with
// A k x m (ta) or A (m x k); op(B) = B (k x n, !tb) or B^T with B n x k.
// work: gemm_oz_work_bytes(m, n, k) bytes of device memory.
cudaError_t gemm_oz(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                    const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* D, int64_t ldd,
                    void* work, size_t work_bytes, int* err) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  const ProfToken tok = prof_begin(s, kProfGemmOz);
  cudaError_t e = cudaSuccess;
  if (k <= 0) {
    oz_scale_kernel<<<static_cast<unsigned>((m * n + 255) / 256), 256, 0, s>>>(m, n, beta, D, ldd);
    note_launch();
    e = cudaGetLastError();
    prof_end(s, tok, 0.0, 16.0 * m * n);
    return e;
  }
  const OzLayout L = oz_layout(m, n, k);
  if (work_bytes < L.total || !work) return cudaErrorInvalidValue;
  if (L.MApad * OZ_S >= (1ll << 31) || L.NBpad * OZ_S >= (1ll << 31) || L.nch > 65535) return cudaErrorInvalidValue;
  char* w = static_cast<char*>(work);
  auto* SA = reinterpret_cast<__nv_bfloat16*>(w);
  int* EA = reinterpret_cast<int*>(w + L.sa);
  auto* SB = reinterpret_cast<__nv_bfloat16*>(w + L.sa + L.ea);
  int* EB = reinterpret_cast<int*>(w + L.sa + L.ea + L.sb);
  double* part = L.nch > 1 ? reinterpret_cast<double*>(w + L.sa + L.ea + L.sb + L.eb) : nullptr;
  // op(A) rows = the m dimension, K contiguous when ta; op(B) columns = the n
  // dimension, K contiguous when !tb
  oz_slice_kernel<<<dim3(static_cast<unsigned>(L.MApad / 32), static_cast<unsigned>(L.nch)), 128, 0, s>>>(
      m, k, A, lda, ta, L.MApad, L.Kpad, SA, EA);
  oz_slice_kernel<<<dim3(static_cast<unsigned>(L.NBpad / 32), static_cast<unsigned>(L.nch)), 128, 0, s>>>(
      n, k, B, ldb, !tb, L.NBpad, L.Kpad, SB, EB);
  note_launch(2);
  e = cudaGetLastError();
  CUtensorMap ma, mb;
  if (e == cudaSuccess && (!make_slice_map(&ma, SA, L.Kpad, OZ_S * L.MApad, OZ_BM) ||
                           !make_slice_map(&mb, SB, L.Kpad, OZ_S * L.NBpad, OZ_BN)))
    e = cudaErrorInvalidValue;
  static bool attr = false;
  if (e == cudaSuccess && !attr) {
    e = cudaFuncSetAttribute(gemm_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
    if (e == cudaSuccess) attr = true;
  }
  if (e == cudaSuccess) {
    dim3 grid(static_cast<unsigned>(L.MApad / OZ_BM), static_cast<unsigned>(L.NBpad / OZ_BN),
              static_cast<unsigned>(L.nch));
    gemm_oz_kernel<<<grid, OZ_NT, OZ_SMEM, s>>>(ma, mb, EA, EB, static_cast<int>(L.MApad), static_cast<int>(L.NBpad),
                                                m, n, alpha, beta, D, ldd, part, err);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && part) {
    oz_reduce_kernel<<<static_cast<unsigned>((m * n + 255) / 256), 256, 0, s>>>(m, n, L.nch, alpha, part, beta, D,
                                                                               ldd);
    note_launch();
    e = cudaGetLastError();
  }
  // flops of the FP64 product it stands for; bytes: FP64 operands once, slices written and read
  prof_end(s, tok, 2.0 * m * n * k,
           8.0 * (m * k + k * n + m * n * (beta != 0.0 ? 2.0 : 1.0)) + 2.0 * static_cast<double>(L.sa + L.sb));
  return e;
}

}  // namespace rutv

extern "C" int randutv_dgemm_oz(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                                const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                                int64_t ldc) {
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
    set_last_error("randutv_dgemm_oz: cuTensorMapEncodeTiled is not available");
    return RANDUTV_EUNSUPPORTED;
  }
  cudaStream_t s = current_stream();
  const size_t wb = gemm_oz_work_bytes(m, n, k);
  void* ws = nullptr;
  int herr = 0;
  cudaError_t e = cudaMallocAsync(&ws, wb + 256, s);
  if (e != cudaSuccess) { cudaGetLastError(); return RANDUTV_ENOMEM; }
  int* err = reinterpret_cast<int*>(static_cast<char*>(ws) + wb);
  e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = gemm_oz(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, wb, err);
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

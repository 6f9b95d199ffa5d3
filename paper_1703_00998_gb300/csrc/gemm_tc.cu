// Tensor-core GEMM of the mixed-precision form (tcgen05, TF32 inputs, FP32
// accumulation in tensor memory): D = alpha op(A) op(B) + beta D, all
// column-major FP32, any transpose combination.  A transposed operand (A^T
// with A stored K x M, or B with B stored K x N) gives K-major tiles; the
// others give MN-major tiles.  Used for the sketch products Y = X^T G,
// Z = X Y, Y = X^T Z of Section 4.3 and for the short (inner dimension b)
// products of the block-reflector applications and rotations.
//
// One CTA computes a 128 x 128 tile of D over a K range (split-K partials
// are summed in FP64 by the FP32 GEMM's reduction kernel):
//   warp 0, one thread: TMA loads of 32-wide K slices of A and B (128B
//     swizzle) into a 4-stage shared-memory ring, mbarrier transaction counts;
//   warp 1, one thread: tcgen05.mma.kind::tf32 (M = N = 128, K = 8 per
//     instruction) into a 128-column FP32 accumulator in tensor memory, each
//     stage released by tcgen05.commit on its "empty" mbarrier;
//   all 4 warps: tcgen05.ld of their 32 lanes, alpha/beta, coalesced stores.
// Every mbarrier wait is bounded (~2 s of GPU time); on expiry the CTA sets
// the error word, waits (bounded) for its copies in flight, frees its tensor
// memory and returns.
#include <cuda.h>
#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace rutv {
namespace {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 32;   // BK = 32 fp32 = 128 bytes = one swizzle row
constexpr int TC_TILE_BYTES = TC_BM * TC_BK * 4;       // 16 KB per operand per stage

// Descriptor of an MN-major 32-bit tile.  For 32-bit elements an MN-major
// operand takes the "128B swizzle with 32-byte atoms" layout (type 1): rows
// of 128 bytes along M or N, whose four 32-byte granules are permuted across
// groups of 4 rows, written by TMA in its matching swizzle mode.  The tile
// is four 32-element (128-byte) chunks along M or N, each a TMA box of 32
// K-rows x 128 bytes (4096 bytes).  Leading byte offset = stride between
// those chunks (4096 bytes); stride byte offset = stride between 4-row
// groups along K (512 bytes: the rows are contiguous).
__device__ __forceinline__ uint64_t mnmajor_sw128a32_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(4096u >> 4) << 16;
  d |= static_cast<uint64_t>(512u >> 4) << 32;
  d |= static_cast<uint64_t>(1u) << 46;
  d |= static_cast<uint64_t>(1u) << 61;                 // 128B swizzle, 32-byte atoms
  return d;
}

// Instruction descriptor, kind::tf32: D FP32, A and B TF32, N = 128, M = 128;
// bit 15 / 16 set for an MN-major A / B.
template <bool AMN, bool BMN>
__host__ __device__ constexpr uint32_t idesc_tf32() {
  return (1u << 4)               // D format F32
         | (2u << 7)             // A format TF32
         | (2u << 10)            // B format TF32
         | ((AMN ? 1u : 0u) << 15)
         | ((BMN ? 1u : 0u) << 16)
         | ((TC_BN >> 3) << 17)
         | ((TC_BM >> 4) << 24);
}

template <bool AMN, bool BMN>
__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc_tf32<AMN, BMN>()), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

// Kernel configuration.  SPLIT = true is the 3xTF32 form: four more warps
// split each landed tile x into hi = rna_tf32(x) (in place) and
// lo = rna_tf32(x - hi), both exactly representable in TF32, and the MMA
// warp accumulates hi*hi + hi*lo + lo*hi (error ~2^-22 relative per product,
// FP32 level); the lo*lo term is dropped.
//
// Promotion (SPLIT): the tensor-core FP32 accumulator truncates at every
// MMA step, which costs about half an ulp of the running sum per K = 8, a
// bias that grows linearly with the reduction length (measured 6.5e-6
// relative at K = 910, 9.7e-7 at K = 146).  So the accumulation restarts
// every TC_CHUNK_KB k-blocks (K = 128) in the other of two tensor-memory
// accumulators, and the four splitter warps add each finished chunk into FP32
// registers (round to nearest) while the MMA warp fills the other one.
constexpr int TC_CHUNK_KB = 4;

template <bool SPLIT>
struct TcCfg {
  static constexpr int STAGES = SPLIT ? 3 : 4;
  static constexpr int TILES = SPLIT ? 4 : 2;               // tiles per stage: A, B (, A_lo, B_lo)
  static constexpr int NT = SPLIT ? 192 : 128;
  static constexpr int EPI_WARP0 = SPLIT ? 2 : 0;            // first of the 4 epilogue warps
  static constexpr uint32_t TMEM_COLS = SPLIT ? 2 * TC_BN : TC_BN;
  static constexpr int SMEM = STAGES * TILES * TC_TILE_BYTES + 1024 + 256;
};

template <bool SPLIT, bool AMN, bool BMN>
__global__ void __launch_bounds__(TcCfg<SPLIT>::NT, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int64_t M,
               int64_t N, int64_t K, float alpha, float beta, float* __restrict__ D, int64_t ldd,
               float* __restrict__ part, int64_t kchunk, int* __restrict__ err) {
  using C = TcCfg<SPLIT>;
  constexpr int S = C::STAGES;
  constexpr int CH = TC_CHUNK_KB;
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  // 1024-byte aligned tiles (the 128B swizzle pattern repeats every 1024 bytes)
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  auto tileA = [&](int st) { return base + st * C::TILES * TC_TILE_BYTES; };
  auto tileB = [&](int st) { return base + st * C::TILES * TC_TILE_BYTES + TC_TILE_BYTES; };
  auto tileAlo = [&](int st) { return base + st * C::TILES * TC_TILE_BYTES + 2 * TC_TILE_BYTES; };
  auto tileBlo = [&](int st) { return base + st * C::TILES * TC_TILE_BYTES + 3 * TC_TILE_BYTES; };
  uint64_t* full = reinterpret_cast<uint64_t*>(base + S * C::TILES * TC_TILE_BYTES);
  uint64_t* split = full + S;
  uint64_t* empty = split + S;
  uint64_t* done = empty + S;
  uint64_t* accf = done + 1;    // [2] accumulator buffer holds a finished chunk (SPLIT)
  uint64_t* acce = accf + 2;    // [2] accumulator buffer drained into registers (SPLIT)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = static_cast<int>(blockIdx.x) * TC_BM;
  const int n0 = static_cast<int>(blockIdx.y) * TC_BN;
  const int64_t kbeg = static_cast<int64_t>(blockIdx.z) * kchunk;
  const int64_t kend = (kbeg + kchunk < K) ? kbeg + kchunk : K;
  const int nkb = static_cast<int>((kend - kbeg + TC_BK - 1) / TC_BK);
  const int nch = (nkb + CH - 1) / CH;

  if (tid == 0) {
    s_fail = 0;
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&split[st], 128);
      mbar_init(&empty[st], 1);
    }
    mbar_init(done, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {   // allocate the FP32 accumulator(s) in tensor memory (128 lanes x 128 columns each)
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
  int issued = 0;   // TMA stages issued by the producer
  const int quarter = warp & 3;   // the 32 tensor-memory lanes this warp may read
  float racc[SPLIT ? TC_BN : 1];  // promoted sums of this thread's row (SPLIT)
#pragma unroll
  for (int j = 0; j < (SPLIT ? TC_BN : 1); ++j) racc[j] = 0.f;

  if (warp == 0 && lane == 0) {
    // producer
    for (int kb = 0; kb < nkb; ++kb) {
      const int st = kb % S;
      if (!mbar_wait(&empty[st], ((kb / S) & 1) ^ 1, t0)) { s_fail = 1; break; }
      mbar_expect_tx(&full[st], 2 * TC_TILE_BYTES);
      const int kx = static_cast<int>(kbeg + static_cast<int64_t>(kb) * TC_BK);
      if (AMN) {
        for (int j = 0; j < 4; ++j) tma_load_2d(tileA(st) + j * 4096, &mapA, m0 + 32 * j, kx, &full[st]);
      } else {
        tma_load_2d(tileA(st), &mapA, kx, m0, &full[st]);
      }
      if (BMN) {
        for (int j = 0; j < 4; ++j) tma_load_2d(tileB(st) + j * 4096, &mapB, n0 + 32 * j, kx, &full[st]);
      } else {
        tma_load_2d(tileB(st), &mapB, kx, n0, &full[st]);
      }
      ++issued;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    for (int kb = 0; kb < nkb; ++kb) {
      const int st = kb % S;
      const int c = kb / CH;
      const uint32_t buf = SPLIT ? static_cast<uint32_t>(c & 1) : 0u;
      const bool first = SPLIT ? (kb % CH == 0) : (kb == 0);
      // (SPLIT) this chunk's accumulator must have been drained two chunks ago
      if (SPLIT && first && c >= 2 && !mbar_wait(&acce[buf], ((c >> 1) - 1) & 1, t0)) { s_fail = 1; break; }
      if (!mbar_wait(SPLIT ? &split[st] : &full[st], (kb / S) & 1, t0)) { s_fail = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // K = 8 per instruction: a K-major tile advances 32 bytes (+2 in 16 B
      // units) along its rows, an MN-major tile one 1024-byte atom (+64)
      const uint64_t da = AMN ? mnmajor_sw128a32_desc(smem_u32(tileA(st))) : kmajor_sw128_desc(smem_u32(tileA(st)));
      const uint64_t db = BMN ? mnmajor_sw128a32_desc(smem_u32(tileB(st))) : kmajor_sw128_desc(smem_u32(tileB(st)));
      const uint64_t dal = AMN ? mnmajor_sw128a32_desc(smem_u32(tileAlo(st))) : kmajor_sw128_desc(smem_u32(tileAlo(st)));
      const uint64_t dbl = BMN ? mnmajor_sw128a32_desc(smem_u32(tileBlo(st))) : kmajor_sw128_desc(smem_u32(tileBlo(st)));
      constexpr uint64_t stepA = AMN ? 64ull : 2ull, stepB = BMN ? 64ull : 2ull;
      const uint32_t dacc = tmem + buf * static_cast<uint32_t>(TC_BN);
#pragma unroll
      for (int kk = 0; kk < TC_BK / 8; ++kk) {
        mma_tf32<AMN, BMN>(dacc, da + stepA * kk, db + stepB * kk, (!first || kk > 0) ? 1u : 0u);
        if (SPLIT) {
          mma_tf32<AMN, BMN>(dacc, da + stepA * kk, dbl + stepB * kk, 1u);
          mma_tf32<AMN, BMN>(dacc, dal + stepA * kk, db + stepB * kk, 1u);
        }
      }
      mma_commit(&empty[st]);
      if (SPLIT && (kb % CH == CH - 1 || kb == nkb - 1)) mma_commit(&accf[buf]);   // chunk c complete
    }
    if (!SPLIT) mma_commit(done);   // arrives once every issued MMA has completed
  } else if (SPLIT && warp >= 2) {
    // splitters: hi = rna_tf32(x) in place, lo = rna_tf32(x - hi); the A and B
    // tiles of a stage are adjacent (8192 floats), and so are their lo tiles.
    // After the last k-block of chunk c they promote chunk c - 1.
    const int w = tid - 64;
    bool failed = false;
    auto promote = [&](int c) {
      const uint32_t buf = static_cast<uint32_t>(c & 1);
      const bool waited = mbar_wait(&accf[buf], (c >> 1) & 1, t0);
      if (__all_sync(0xffffffffu, waited) == 0) { failed = true; return; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c0 = 0; c0 < TC_BN; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + buf * TC_BN + static_cast<uint32_t>(c0), r);
#pragma unroll
        for (int j = 0; j < 32; ++j) racc[c0 + j] += __uint_as_float(r[j]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&acce[buf]);
    };
    for (int kb = 0; kb < nkb && !failed; ++kb) {
      const int st = kb % S;
      if (!mbar_wait(&full[st], (kb / S) & 1, t0)) { failed = true; break; }
      float4* hi = reinterpret_cast<float4*>(tileA(st));
      float4* lo = reinterpret_cast<float4*>(tileAlo(st));
#pragma unroll 4
      for (int e = w; e < 2 * TC_TILE_BYTES / 16; e += 128) {
        const float4 x = hi[e];
        float4 h, l;
        h.x = tf32_rna(x.x); h.y = tf32_rna(x.y); h.z = tf32_rna(x.z); h.w = tf32_rna(x.w);
        l.x = tf32_rna(x.x - h.x); l.y = tf32_rna(x.y - h.y); l.z = tf32_rna(x.z - h.z); l.w = tf32_rna(x.w - h.w);
        hi[e] = h;
        lo[e] = l;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor-core reads
      mbar_arrive(&split[st]);
      if ((kb % CH == CH - 1 || kb == nkb - 1) && kb / CH >= 1) promote(kb / CH - 1);
    }
    if (!failed && nch > 0) promote(nch - 1);
    if (failed) s_fail = 1;
  }
  __syncwarp();
  const bool epi = warp >= C::EPI_WARP0 && warp < C::EPI_WARP0 + 4;
  if (!SPLIT) {
    // wait for the accumulator (the decision is made uniform across the
    // warp: tcgen05.ld below is a warp-collective instruction)
    const bool waited = epi ? mbar_wait(done, 0, t0) : true;
    const bool warp_ok = __all_sync(0xffffffffu, waited) != 0;
    if (!warp_ok && lane == 0) s_fail = 1;
  }
  __syncthreads();
  const bool ok = (s_fail == 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (epi && ok) {
    const int row = m0 + quarter * 32 + lane;
    auto put = [&](int64_t col, float v) {
      if (part) {
        part[static_cast<int64_t>(blockIdx.z) * M * N + row + col * M] = v;
      } else {
        float* dp = D + row + col * ldd;
        *dp = (beta == 0.f) ? alpha * v : fmaf(alpha, v, beta * *dp);
      }
    };
    if (SPLIT) {
      // racc holds the sum (zero for an empty K range)
      if (row < M) {
#pragma unroll
        for (int j = 0; j < (SPLIT ? TC_BN : 1); ++j) {
          const int64_t col = n0 + j;
          if (col < N) put(col, racc[j]);
        }
      }
    } else if (nkb > 0) {
      for (int c0 = 0; c0 < TC_BN; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + static_cast<uint32_t>(c0), r);
        if (row < M) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int64_t col = n0 + c0 + j;
            if (col < N) put(col, __uint_as_float(r[j]));
          }
        }
      }
    } else if (row < M) {
      for (int j = 0; j < TC_BN; ++j) {   // empty K range: D = beta D (or zero partials)
        const int64_t col = n0 + j;
        if (col >= N) break;
        put(col, 0.f);
      }
    }
  }
  if (!ok && tid == 0) atomicOr(err, kDevErrTimeout);
  // drain: the producer's copies in flight must land before the CTA exits
  if (!ok && warp == 0 && lane == 0) {
    for (int kb = 0; kb < issued; ++kb) mbar_wait(&full[kb % S], (kb / S) & 1, global_ns());
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
  }
}

// 2-D map of a column-major FP32 matrix with `rows` contiguous entries per
// column and `cols` columns, leading dimension ld, zero fill outside the
// matrix.  K-major operand (rows = K): box 32 (K) x 128, 128B swizzle;
// MN-major operand (rows = M or N): box 32 x 32 (K), four per tile, 128B
// swizzle with 32-byte atoms.
bool make_map(CUtensorMap* map, const float* ptr, int64_t rows, int64_t cols, int64_t ld, bool mn_major) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(rows), static_cast<cuuint64_t>(cols)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * sizeof(float)};
  cuuint32_t box[2] = {32u, mn_major ? 32u : static_cast<cuuint32_t>(TC_BM)};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, mn_major ? CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B : CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool gemm_tc_supported(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t m, int64_t n, int64_t k) {
  // TMA: 16-byte aligned bases and strides; sizes within the 32-bit coordinate range
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  return encode_fn() != nullptr && al16(A) && al16(B) && (lda % 4) == 0 && (ldb % 4) == 0 && m > 0 && n > 0 &&
         k > 0 && m < (1ll << 31) && n < (1ll << 31) && k < (1ll << 31);
}

template <bool SPLIT, bool AMN, bool BMN>
cudaError_t launch_tc(dim3 grid, cudaStream_t s, const CUtensorMap& ma, const CUtensorMap& mb, int64_t m, int64_t n,
                      int64_t k, float alpha, float beta, float* D, int64_t ldd, float* part, int64_t kc, int* err) {
  static PerDeviceOnce once;
  cudaError_t e = per_device_once(once, [] {
    return cudaFuncSetAttribute(gemm_tc_kernel<SPLIT, AMN, BMN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TcCfg<SPLIT>::SMEM);
  });
  if (e != cudaSuccess) return e;
  gemm_tc_kernel<SPLIT, AMN, BMN><<<grid, TcCfg<SPLIT>::NT, TcCfg<SPLIT>::SMEM, s>>>(ma, mb, m, n, k, alpha, beta, D,
                                                                                    ldd, part, kc, err);
  return cudaGetLastError();
}

// D (m x n) = alpha op(A) op(B) + beta D, column-major FP32: op(A) = A^T with
// A k x m (ta) or A with A m x k; op(B) = B with B k x n (!tb) or B^T with
// B n x k.  split = true runs the 3xTF32 form (FP32-level products).
cudaError_t gemm_tc(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, float alpha, const float* A,
                    int64_t lda, const float* B, int64_t ldb, float beta, float* D, int64_t ldd, float* work,
                    int64_t work_elems, int* err, bool split) {
  const bool amn = !ta, bmn = tb;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, amn ? m : k, amn ? k : m, lda, amn) || !make_map(&mb, B, bmn ? n : k, bmn ? k : n, ldb, bmn))
    return cudaErrorInvalidValue;
  const int64_t tiles = ((m + TC_BM - 1) / TC_BM) * ((n + TC_BN - 1) / TC_BN);
  // split K while the CTAs still fit one wave (each CTA takes one SM: >= 130 KB of shared memory)
  int splits = 1;
  while (tiles * (splits + 1) <= kNumSMs && (k / (splits + 1)) >= 4 * TC_BK && (splits + 1) * m * n <= work_elems)
    ++splits;
  int64_t kc = (k + splits - 1) / splits;
  kc = ((kc + TC_BK - 1) / TC_BK) * TC_BK;
  splits = static_cast<int>((k + kc - 1) / kc);
  float* part = splits > 1 ? work : nullptr;
  dim3 grid(static_cast<unsigned>((m + TC_BM - 1) / TC_BM), static_cast<unsigned>((n + TC_BN - 1) / TC_BN),
            static_cast<unsigned>(splits));
  const ProfToken tok = prof_begin(s, kProfGemmTc);
  cudaError_t e;
#define RUTV_TC(S_, A_, B_) e = launch_tc<S_, A_, B_>(grid, s, ma, mb, m, n, k, alpha, beta, D, ldd, part, kc, err)
  if (split) {
    if (!amn && !bmn) RUTV_TC(true, false, false);
    else if (amn && !bmn) RUTV_TC(true, true, false);
    else if (amn && bmn) RUTV_TC(true, true, true);
    else RUTV_TC(true, false, true);
  } else {
    if (!amn && !bmn) RUTV_TC(false, false, false);
    else if (amn && !bmn) RUTV_TC(false, true, false);
    else if (amn && bmn) RUTV_TC(false, true, true);
    else RUTV_TC(false, false, true);
  }
#undef RUTV_TC
  note_launch();
  if (e == cudaSuccess && splits > 1) e = gemm_f32_reduce(s, m, n, splits, alpha, part, beta, D, ldd);
  prof_end(s, tok, (split ? 3.0 : 1.0) * 2.0 * m * n * k, 4.0 * (m * k + k * n + m * n * (beta != 0.f ? 2.0 : 1.0)));
  return e;
}

cudaError_t gemm_tc_tn(cudaStream_t s, int64_t m, int64_t n, int64_t k, float alpha, const float* A, int64_t lda,
                       const float* B, int64_t ldb, float beta, float* D, int64_t ldd, float* work, int64_t work_elems,
                       int* err, bool split) {
  return gemm_tc(s, true, false, m, n, k, alpha, A, lda, B, ldb, beta, D, ldd, work, work_elems, err, split);
}

}  // namespace rutv

extern "C" int randutv_sgemm_tc(char transa, char transb, int64_t m, int64_t n, int64_t k, float alpha,
                                const float* A, int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                                int64_t ldc, int passes) {
  using namespace rutv;
  const bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
  if (!ta && transa != 'N' && transa != 'n') return -1;
  if (!tb && transb != 'N' && transb != 'n') return -2;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (k < 1) return -5;
  if (!A) return -7;
  if (lda < (ta ? k : m)) return -8;
  if (!B) return -9;
  if (ldb < (tb ? n : k)) return -10;
  if (!C) return -12;
  if (ldc < m) return -13;
  if (passes != 1 && passes != 3) return -14;
  if (!gemm_tc_supported(A, lda, B, ldb, m, n, k)) {
    set_last_error("randutv_sgemm_tc: operands do not meet the TMA alignment rules");
    return RANDUTV_EUNSUPPORTED;
  }
  cudaStream_t s = current_stream();
  const int64_t we = 16 * m * n;
  float* ws = nullptr;
  int* err = nullptr;
  int herr = 0;
  cudaError_t e = cudaMallocAsync(&ws, we * sizeof(float) + 256, s);
  if (e != cudaSuccess) { cudaGetLastError(); return RANDUTV_ENOMEM; }
  err = reinterpret_cast<int*>(reinterpret_cast<char*>(ws) + we * sizeof(float));
  e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = gemm_tc(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, we, err, passes == 3);
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

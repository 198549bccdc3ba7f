// Tensor-core GEMM of the propagation chain on sm_103a (tcgen05 + TMA).
//
// C[M, N] (fp32) = A[M, K] * B[N, K]^T with A and B K-major, the dense
// products of the chain: the backward step y = W^T nu (B = W^T stored
// [d_{i-1}, d_i]) and the reverse-mode step nubar = W a (B = W [d_i, d_{i-1}]).
//
//  * BF16 chain: tcgen05.mma kind::f16 with bf16 operands, fp32 accumulation.
//  * FP32 chain: kind::tf32 in three passes (A_hi B_hi + A_hi B_lo + A_lo B_hi
//    with x = x_hi + x_lo, x_hi = x rounded to tf32), which carries about 21
//    mantissa bits through the product: the split-operand scheme of Henry,
//    Tang and Heinecke for bfloat16, applied to tf32.
//
// One CTA computes a 128 x 128 tile; its fp32 accumulator lives in TMEM
// (128 lanes x 128 columns). Warp 0 (one lane) streams A/B tiles into shared
// memory with TMA (128-byte swizzle, the layout the MMA's descriptors name);
// warp 1 (one lane) issues the MMAs and commits each stage back to the
// producer through mbarriers; then all four warps read the accumulator with
// tcgen05.ld (thread = row) and store it. Every wait is bounded: on timeout the
// kernel records an error word, stops issuing work and frees its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "gcp_internal.cuh"

namespace gcp {

__device__ unsigned int g_tc_err;  // bit 0: pipeline wait timed out

namespace {

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int kRowBytes = 128;                 // K bytes per stage row (the swizzle span)
constexpr int kTileA = BM * kRowBytes;         // 16 KiB
constexpr int kTileB = BN * kRowBytes;         // 16 KiB
constexpr long long kWaitCycles = 2000000000;  // about one second at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity; false after about a second.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 1023u) == 1023u && clock64() - t0 > kWaitCycles) {
      atomicOr(&g_tc_err, 1u);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes in 8-row atoms of 1024 bytes (stride 1024 between atoms).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(16u >> 4) << 16;    // leading byte offset (unused for swizzled K-major)
  d |= static_cast<uint64_t>(1024u >> 4) << 32;  // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;           // descriptor version
  d |= static_cast<uint64_t>(2) << 61;           // 128-byte swizzle
  return d;
}

// Instruction descriptor: fp32 accumulator, K-major A and B, M x N shape.
__host__ __device__ constexpr uint32_t idesc(uint32_t ab_format, int M, int N) {
  return (1u << 4) | (ab_format << 7) | (ab_format << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id, uint32_t accumulate) {
  if constexpr (KIND == 0) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(tmem_d),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(tmem_d),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
  }
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int KIND>
struct TcCfg {
  static constexpr int kPasses = KIND == 0 ? 1 : 3;
  static constexpr int kTiles = KIND == 0 ? 2 : 4;  // A, B (+ A_lo, B_lo)
  static constexpr int kStageBytes = KIND == 0 ? kTileA + kTileB : 2 * kTileA + 2 * kTileB;
  static constexpr int kStages = KIND == 0 ? 4 : 3;
  static constexpr int kKElems = KIND == 0 ? 64 : 32;  // K elements per 128-byte row
  static constexpr uint32_t kFormat = KIND == 0 ? 1u : 2u;  // bf16 / tf32
  static constexpr int kSmem = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
};

template <int KIND>
__global__ void __launch_bounds__(128, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tAlo,
              const __grid_constant__ CUtensorMap tB, const __grid_constant__ CUtensorMap tBlo, int M, int N, int K,
              float* __restrict__ C) {
  using Cfg = TcCfg<KIND>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Cfg::kStages * Cfg::kStageBytes);
  uint64_t* empty = full + Cfg::kStages;
  uint64_t* done = empty + Cfg::kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int KT = (K + Cfg::kKElems - 1) / Cfg::kKElems;

  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: TMA loads of stage kt into slot kt % S
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % Cfg::kStages;
      const uint32_t ph = (kt / Cfg::kStages) & 1;
      if (!mbar_wait(&empty[s], ph ^ 1)) break;
      uint8_t* st = smem + s * Cfg::kStageBytes;
      mbar_expect_tx(&full[s], Cfg::kStageBytes);
      const int x = kt * Cfg::kKElems;
      tma_load_2d(st, &tA, &full[s], x, m0);
      tma_load_2d(st + kTileA, &tB, &full[s], x, n0);
      if constexpr (KIND == 1) {
        tma_load_2d(st + kTileA + kTileB, &tAlo, &full[s], x, m0);
        tma_load_2d(st + 2 * kTileA + kTileB, &tBlo, &full[s], x, n0);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: 4 K-steps of 32 bytes per stage, 1 or 3 passes each
    constexpr uint32_t id = idesc(Cfg::kFormat, BM, BN);
    bool ok = true;
    for (int kt = 0; kt < KT && ok; ++kt) {
      const int s = kt % Cfg::kStages;
      const uint32_t ph = (kt / Cfg::kStages) & 1;
      if (!mbar_wait(&full[s], ph)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a = smem_u32(smem + s * Cfg::kStageBytes);
      const uint32_t b = a + kTileA;
#pragma unroll
      for (int kk = 0; kk < kRowBytes / 32; ++kk) {
        const uint64_t da = sdesc(a + kk * 32), db = sdesc(b + kk * 32);
        umma<KIND>(tmem, da, db, id, (kt | kk) != 0);
        if constexpr (KIND == 1) {
          const uint64_t da_lo = sdesc(a + kTileA + kTileB + kk * 32), db_lo = sdesc(b + kTileA + kTileB + kk * 32);
          umma<KIND>(tmem, da, db_lo, id, 1);
          umma<KIND>(tmem, da_lo, db, id, 1);
        }
      }
      umma_commit(&empty[s]);  // slot free once these MMAs have read it
    }
    umma_commit(done);         // accumulator complete
  }
  __syncwarp();

  // epilogue: thread = row of the tile, 32 columns per TMEM load
  const bool ready = mbar_wait(done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ready) {
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c = 0; c < BN; c += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c, r);
      if (row < M) {
        float* dst = C + static_cast<int64_t>(row) * N + n0 + c;
        const int ncol = min(32, N - (n0 + c));
        if (ncol == 32 && (N & 3) == 0) {
#pragma unroll
          for (int q = 0; q < 32; q += 4)
            *reinterpret_cast<float4*>(dst + q) =
                make_float4(__uint_as_float(r[q]), __uint_as_float(r[q + 1]), __uint_as_float(r[q + 2]),
                            __uint_as_float(r[q + 3]));
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q)
            if (q < ncol) dst[q] = __uint_as_float(r[q]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
  }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_encode != nullptr;
}

// 2-D map of a row-major [rows, cols] matrix, box of box_rows x 128 bytes.
bool make_map(CUtensorMap* m, const void* base, bool bf16, int64_t rows, int64_t cols, int box_rows) {
  const int es = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(cols) * es};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kRowBytes / es), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  return g_encode(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KIND>
bool launch_tc(cudaStream_t st, int64_t M, int N, int K, const void* A, const void* Alo, const void* B,
               const void* Blo, float* C) {
  using Cfg = TcCfg<KIND>;
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(k_gemm_tc<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem);
  });
  const bool bf = KIND == 0;
  CUtensorMap ta{}, talo{}, tb{}, tblo{};
  if (!make_map(&ta, A, bf, M, K, BM) || !make_map(&tb, B, bf, N, K, BN)) return false;
  if (KIND == 1) {
    if (!make_map(&talo, Alo, bf, M, K, BM) || !make_map(&tblo, Blo, bf, N, K, BN)) return false;
  } else {
    talo = ta;
    tblo = tb;
  }
  dim3 grid((N + BN - 1) / BN, static_cast<unsigned>((M + BM - 1) / BM));
  k_gemm_tc<KIND><<<grid, 128, Cfg::kSmem, st>>>(ta, talo, tb, tblo, static_cast<int>(M), N, K, C);
  return true;
}

}  // namespace

bool tc_available(int K, bool bf16) {
  // TMA needs 16-byte row strides; the kernel tiles rows by 128.
  if (!encoder()) return false;
  return bf16 ? (K % 8 == 0) : (K % 4 == 0);
}

bool gemm_tc_bf16(cudaStream_t st, int64_t M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C) {
  if (M <= 0 || N <= 0) return true;
  if (!tc_available(K, true) || M > (int64_t)INT32_MAX) return false;
  if (!(reg_check(A, (double)M * K * 2, "tc A") & reg_check(B, (double)N * K * 2, "tc B") &
        reg_check(C, (double)M * N * 4, "tc C")))
    return true;  // reported by the caller's launch status
  int tk = prof_begin(st, "gemm_tc_bf16", 2.0 * M * N * K, ((double)M * K + (double)N * K) * 2 + (double)M * N * 4);
  const bool ok = launch_tc<0>(st, M, N, K, A, nullptr, B, nullptr, C);
  prof_end(st, tk);
  return ok;
}

bool gemm_tc_tf32x3(cudaStream_t st, int64_t M, int N, int K, const float* A, const float* Alo, const float* B,
                    const float* Blo, float* C) {
  if (M <= 0 || N <= 0) return true;
  if (!tc_available(K, false) || M > (int64_t)INT32_MAX) return false;
  if (!(reg_check(A, (double)M * K * 4, "tc A") & reg_check(Alo, (double)M * K * 4, "tc A lo") &
        reg_check(B, (double)N * K * 4, "tc B") & reg_check(Blo, (double)N * K * 4, "tc B lo") &
        reg_check(C, (double)M * N * 4, "tc C")))
    return true;
  int tk = prof_begin(st, "gemm_tc_tf32x3", 2.0 * M * N * K, ((double)M * K + (double)N * K) * 8 + (double)M * N * 4);
  const bool ok = launch_tc<1>(st, M, N, K, A, Alo, B, Blo, C);
  prof_end(st, tk);
  return ok;
}

std::string take_tc_error(cudaStream_t st) {
  unsigned int h = 0;
  if (cudaMemcpyFromSymbolAsync(&h, g_tc_err, sizeof h, 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess || h == 0)
    return std::string();
  const unsigned int z = 0;
  cudaMemcpyToSymbolAsync(g_tc_err, &z, sizeof z, 0, cudaMemcpyHostToDevice, st);
  cudaStreamSynchronize(st);
  return "tensor-core GEMM: a pipeline wait timed out";
}

}  // namespace gcp

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
//    Tang and Heinecke for bfloat16, applied to tf32. The weights are split
//    once at network load; A arrives as plain fp32, and warps 2-5 (thread =
//    tile row) split each staged A tile and store A_hi and A_lo into tensor
//    memory, where the MMAs read A from. Shared memory then only carries the
//    TMA traffic and the B operands: three passes reading A and B from shared
//    memory would move about 1.7x the bytes the tensor pipe needs per cycle.
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

#include <algorithm>
#include <cmath>
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

// The same with a suspend-time hint: each try may suspend the thread in
// hardware for up to a microsecond until the phase completes, instead of
// spinning and taking issue slots from the warps doing the work.
__device__ __forceinline__ bool mbar_wait_idle(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  for (uint32_t i = 0;; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
        : "memory");
    if (ok) return true;
    if ((i & 15u) == 15u && clock64() - t0 > kWaitCycles) {
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

// Bulk tensor store of a staged box (bulk-group completion).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(x), "r"(y)
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

// kind::tf32 with A in tensor memory (lane = row of A, one column per K element)
__device__ __forceinline__ void umma_tf32_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t id,
                                             uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::
          "r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(id), "r"(accumulate)
      : "memory");
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

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

// Stage layout: the A tile, then the B tile (KIND 1: and B_lo). KIND 1 keeps
// A_hi | A_lo of each stage in TMEM columns kAccCols + s * 64 (32 each).
template <int KIND, int BNT = BN>
struct TcCfg {
  static constexpr int kTileBt = BNT * kRowBytes;   // the B tile (BNT rows of 128 bytes)
  static constexpr int kStageBytes = KIND == 0 ? kTileA + kTileBt : kTileA + 2 * kTileBt;
  // three-pass tf32: three stages (144 KB) leave room beside a CTA for the
  // blocks of the next span kernel to start early (47.0 vs 47.4 ms per MLP
  // step); the bf16 kernel keeps four (three measured slower)
  static constexpr int kStages = KIND == 1 ? 3 : 4;
  static constexpr int kKElems = KIND == 0 ? 64 : 32;  // K elements per 128-byte row
  static constexpr uint32_t kFormat = KIND == 0 ? 1u : 2u;  // bf16 / tf32
  static constexpr int kAccCols = BNT;
  // KIND 1: A_hi | A_lo of stage s at TMEM columns kSplitCol + 64 s
  static constexpr int kSplitCol = BNT <= 128 ? 128 : 256;
  static constexpr int kTmemCols = KIND == 0 ? (BNT <= 128 ? 128 : 256) : 512;   // powers of two
  static constexpr int kSmem = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
};
static_assert(TcCfg<1>::kSplitCol + TcCfg<1>::kStages * 64 <= TcCfg<1>::kTmemCols, "TMEM columns");
static_assert(TcCfg<1, 224>::kSplitCol + TcCfg<1, 224>::kStages * 64 <= TcCfg<1, 224>::kTmemCols, "TMEM columns");
static_assert(TcCfg<1, 224>::kSmem <= 227 * 1024, "shared memory of the 224-column tiles");
static_assert(4 * 32 * BN * 4 <= TcCfg<0>::kStages * TcCfg<0>::kStageBytes, "epilogue staging fits the stages");
static_assert(4 * 32 * (224 + 4) * 4 <= TcCfg<1, 224>::kStages * TcCfg<1, 224>::kStageBytes, "epilogue staging");
static_assert(4 * 32 * (224 + 4) * 4 <= TcCfg<0, 224>::kStages * TcCfg<0, 224>::kStageBytes, "epilogue staging");
static_assert(TcCfg<0, 224>::kAccCols <= TcCfg<0, 224>::kTmemCols && TcCfg<0, 224>::kSmem <= 227 * 1024, "bf16 224");

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// threads: warp 0 producer lane, warp 1 MMA lane, warps 0-3 epilogue, and for
// the FP32 chain warps 2-5 the tf32 split of A
template <int KIND>
constexpr int tc_threads() { return KIND == 1 ? 192 : 128; }
constexpr int kSplitThreads = 128;

template <int KIND, int BNT = BN>
__global__ void __launch_bounds__(tc_threads<KIND>(), 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB,
              const __grid_constant__ CUtensorMap tBlo, const __grid_constant__ CUtensorMap tC, int c_tma, int M,
              int N, int K, float* __restrict__ C) {
  using Cfg = TcCfg<KIND, BNT>;
  constexpr int kTileB = Cfg::kTileBt;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Cfg::kStages * Cfg::kStageBytes);
  uint64_t* empty = full + Cfg::kStages;
  uint64_t* xfull = empty + Cfg::kStages;   // tf32 split of the stage's A tile done (KIND 1)
  uint64_t* done = xfull + Cfg::kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

  griddep_launch();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BNT;
  const int KT = (K + Cfg::kKElems - 1) / Cfg::kKElems;

  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&xfull[s], kSplitThreads);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    // the tensor maps are kernel parameters: fetch them while earlier kernels finish
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tB)) : "memory");
    if (KIND == 1) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tBlo)) : "memory");
    if (c_tma) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tC)) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(Cfg::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  // B (weights, or their exact slices) is never written by kernels that may
  // still be running: the first stages' B tiles load before the dependency
  // wait, under the previous kernel's tail; their stage barriers then wait
  // for A's bytes as well
  const int npre = KT < Cfg::kStages ? KT : Cfg::kStages;
  if (warp == 0 && lane == 0) {
    for (int kt = 0; kt < npre; ++kt) {
      uint8_t* st = smem + kt * Cfg::kStageBytes;
      mbar_expect_tx(&full[kt], Cfg::kStageBytes);
      tma_load_2d(st + kTileA, &tB, &full[kt], kt * Cfg::kKElems, n0);
      if constexpr (KIND == 1) tma_load_2d(st + kTileA + kTileB, &tBlo, &full[kt], kt * Cfg::kKElems, n0);
    }
  }
  griddep_wait();   // A (and C's previous readers) belong to earlier kernels

  if (warp == 0 && lane == 0) {
    // producer: TMA loads of stage kt into slot kt % S
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % Cfg::kStages;
      const uint32_t ph = (kt / Cfg::kStages) & 1;
      if (!mbar_wait_idle(&empty[s], ph ^ 1)) break;
      uint8_t* st = smem + s * Cfg::kStageBytes;
      const int x = kt * Cfg::kKElems;
      if (kt >= npre) {
        mbar_expect_tx(&full[s], Cfg::kStageBytes);
        tma_load_2d(st + kTileA, &tB, &full[s], x, n0);
        if constexpr (KIND == 1) tma_load_2d(st + kTileA + kTileB, &tBlo, &full[s], x, n0);
      }
      tma_load_2d(st, &tA, &full[s], x, m0);
    }
  } else if (KIND == 1 && warp >= 2) {
    // tf32 split of A into TMEM: x = hi + lo, hi = x rounded to tf32 (nearest,
    // ties away), lo exact. Thread = tile row; a warp may only reach the TMEM
    // lanes of its quadrant (warp % 4), so warps 2, 3, 4, 5 take rows 64-95,
    // 96-127, 0-31, 32-63. The staged row is 32 floats in 16-byte chunks,
    // chunk c at position c ^ (row % 8) (128-byte swizzle of a 1024-byte
    // aligned tile). full[s] completing implies the MMAs of the stage's
    // previous use have finished (the producer waited for them before the
    // TMA), so its TMEM columns are free.
    const int row = ((warp & 3) << 5) + lane;
    const uint32_t trow = tmem + (static_cast<uint32_t>((warp & 3) << 5) << 16) + Cfg::kSplitCol;
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % Cfg::kStages;
      const uint32_t ph = (kt / Cfg::kStages) & 1;
      if (!mbar_wait_idle(&full[s], ph)) break;
      const uint8_t* arow = smem + s * Cfg::kStageBytes + row * kRowBytes;
      uint32_t h[32], l[32];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float4 v = *reinterpret_cast<const float4*>(arow + ((c ^ (row & 7)) << 4));
        const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          uint32_t hb;
          asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(x[e]));
          h[4 * c + e] = hb;
          l[4 * c + e] = __float_as_uint(x[e] - __uint_as_float(hb));
        }
      }
      tmem_st32(trow + s * 64, h);
      tmem_st32(trow + s * 64 + 32, l);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&xfull[s]);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: 4 K-steps of 32 bytes per stage, 1 or 3 passes each
    constexpr uint32_t id = idesc(Cfg::kFormat, BM, BNT);
    bool ok = true;
    for (int kt = 0; kt < KT && ok; ++kt) {
      const int s = kt % Cfg::kStages;
      const uint32_t ph = (kt / Cfg::kStages) & 1;
      if (!mbar_wait_idle(KIND == 1 ? &xfull[s] : &full[s], ph)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a = smem_u32(smem + s * Cfg::kStageBytes);
      const uint32_t b = a + kTileA;
#pragma unroll
      for (int kk = 0; kk < kRowBytes / 32; ++kk) {
        const uint64_t db = sdesc(b + kk * 32);
        if constexpr (KIND == 1) {
          // A_hi, A_lo: 8 TMEM columns per K-step of 8 tf32 elements
          const uint32_t ta = tmem + Cfg::kSplitCol + s * 64 + kk * 8;
          const uint64_t db_lo = sdesc(b + kTileB + kk * 32);
          umma_tf32_ta(tmem, ta, db, id, (kt | kk) != 0);
          umma_tf32_ta(tmem, ta, db_lo, id, 1);
          umma_tf32_ta(tmem, ta + 32, db, id, 1);
        } else {
          umma<KIND>(tmem, sdesc(a + kk * 32), db, id, (kt | kk) != 0);
        }
      }
      umma_commit(&empty[s]);  // slot free once these MMAs have read it
    }
    umma_commit(done);         // accumulator complete
  }
  __syncwarp();

  // epilogue: warp w reads TMEM lanes 32w .. 32w+31 (thread = row, 32
  // columns per load) into the now idle stage memory. With a tensor map for C
  // (row stride a multiple of 16 bytes) the warp stages its 32 x 128 block as
  // four 32 x 32 boxes in the 128-byte swizzled layout (16-byte chunk q of row
  // i at position q ^ (i % 8): conflict-free stores) and one lane hands them
  // to bulk tensor stores, which clip the rows and columns beyond M and N.
  // Otherwise it stages a padded row-major tile and writes whole rows.
  const bool ready = warp < 4 && mbar_wait_idle(done, 0);   // warps 4-5 (split only) skip the epilogue
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ready && c_tma) {
    uint8_t* stg = smem + warp * (32 * BNT * 4);
#pragma unroll 1
    for (int c = 0; c < BNT; c += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c, r);
      uint8_t* row = stg + (c >> 5) * 4096 + lane * 128;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        *reinterpret_cast<uint4*>(row + ((q ^ (lane & 7)) << 4)) =
            make_uint4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) {
      const int y = m0 + warp * 32;
      for (int c = 0; c < BNT / 32; ++c)
        if (y < M && n0 + 32 * c < N) tma_store_2d(&tC, stg + c * 4096, n0 + 32 * c, y);
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");   // staging read before the CTA ends
    }
    __syncwarp();
  } else if (ready) {
    constexpr int kLd = BNT + 4;   // padded row stride (floats): conflict-free float4 stores
    float* ct = reinterpret_cast<float*>(smem) + warp * 32 * kLd;
#pragma unroll 1
    for (int c = 0; c < BNT; c += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c, r);
#pragma unroll
      for (int q = 0; q < 32; q += 4)
        *reinterpret_cast<float4*>(ct + lane * kLd + c + q) =
            make_float4(__uint_as_float(r[q]), __uint_as_float(r[q + 1]), __uint_as_float(r[q + 2]),
                        __uint_as_float(r[q + 3]));
    }
    __syncwarp();
    const int ncol = min(BNT, N - n0);
#pragma unroll 1
    for (int i = 0; i < 32; ++i) {
      const int row = m0 + warp * 32 + i;
      if (row >= M) break;
      float* dst = C + static_cast<int64_t>(row) * N + n0;
      const float* srcr = ct + i * kLd;
      for (int q = lane; q < ncol; q += 32) dst[q] = srcr[q];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::kTmemCols)
                 : "memory");
  }
}

// ------------------------------------------------------------------ implicit-GEMM convolution
// out = conv(src) (dir 0, the reverse-mode step through a convolution) or
// conv^T(src) (dir 1, the backward step y = W^T nu) for all rows as one GEMM
// on the tensor cores, bf16 operands and fp32 accumulation. The GEMM rows are
// the output pixels of all rows, phase by phase (ConvPlan): within phase f,
// row m = mbase_f + r * Hf * Wf + (i * Wf + j); the columns are output
// channels; the K index runs over the phase's taps and the source channels.
// A transposed convolution of stride s thus multiplies only the taps that
// reach each pixel (on average k*k / s^2 of them) instead of all k*k.
//
// A persistent CTA of 256 threads loops over 128-row tiles (a tile never
// crosses a phase). Per tile it stages the source-map rows its taps can reach
// in shared memory, channel innermost, then builds each 128 x 64 A block from
// them (two threads per row, four 16-byte chunks each) directly in the
// 128-byte-swizzled K-major layout the MMA descriptor names, double-buffered
// so building block j+1 overlaps the MMAs of block j. The packed weights
// [Np, Kp] stay in shared memory for the whole kernel; the accumulator
// (128 x Np fp32) lives in TMEM.
struct ConvTcArgs {
  ConvPlan c;
  int64_t R;
  int stg_rows;            // source-map rows the staging buffer holds
  int tmem_cols;
  int group;               // tiles per work unit: 1, or 2 = phases (ph, 0) and (ph, 1) together
  int units;
  int stg_bufs;            // staging buffers: 2 = the next unit's source rows load during this unit's A blocks
  const __nv_bfloat16* src;  // [R, Cs*Hs*Ws], channel-major (c, h, w)
  const __nv_bfloat16* Wp;   // [Np, Kp]
  float* out;                // [R, Co*Ho*Wo], channel-major
  // optional second weight operand: K-block kb's A block is also multiplied
  // by tile b2map[kb] (>= 0) of Wp2 [Np, 64 * nb2] and added (the low term of
  // the weights, which reuses the A block built for the high term)
  const __nv_bfloat16* Wp2;
  int nb2;
  int8_t b2map[kConvMaxKb];
};

// Roles of the 416 threads: warps 0-3 the epilogue (warp w reads TMEM lanes
// 32w .. 32w+31), warps 4-11 the producers (staging and A blocks), warp 12
// the MMA issuer (one lane).
constexpr int kConvEpiWarps = 4, kConvProdWarps = 8;
constexpr int kConvProdThreads = kConvProdWarps * 32;
constexpr int kConvThreads = (kConvEpiWarps + kConvProdWarps + 1) * 32;
constexpr int kConvStages = 4;   // A blocks in flight
struct ConvSmem {
  int b_off, stg_off, tab_off, bar_off, total;
};
__host__ __device__ inline ConvSmem conv_smem_layout(int Kp, int Np, int stg_rows, int Ws, int Csp, int bufs,
                                                     int nb2 = 0) {
  ConvSmem L;
  L.b_off = kConvStages * kTileA;                          // after the A stages
  L.stg_off = L.b_off + (Kp / 64 + nb2) * Np * kRowBytes;  // weights: Kp/64 (+ nb2) tiles of Np rows
  L.tab_off = (L.stg_off + bufs * stg_rows * Ws * Csp * 2 + 15) & ~15;
  L.bar_off = (L.tab_off + (Kp / 8) * 4 + 7) & ~7;         // chunk table: one word per 8 K columns
  // barriers: full/empty per A stage, full/empty per accumulator, abort flag, TMEM slot
  L.total = L.bar_off + (2 * kConvStages + 4) * 8 + 16 + 1024;
  return L;
}

// Named barrier 1 over the producer warps with an OR of v over them: every
// producer gets the same answer, so they leave their loop together.
__device__ __forceinline__ bool prod_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kConvProdThreads)
      : "memory");
  return r != 0;
}


// Tile geometry: phase, GEMM rows [m0, mend) of the phase (phase-local), batch
// rows r0 .. r0 + nrt - 1, and the source-map rows sh0 .. sh0 + nsh - 1 the
// tile reads (per batch row; the whole map when the tile spans several batch
// rows). 32-bit arithmetic: the launcher requires R * Ho * Wo < 2^31.
struct ConvTile {
  int f, nrt, sh0, nsh;
  int m0, mend, r0;
};
// Work unit u: one tile, or (group 2, a stride-2 transposed convolution)
// tile q of phases (ph, 0) and (ph, 1), which cover the same batch rows and
// phase-local pixels and read the same source rows. Their outputs interleave
// along w (columns 2j and 2j + 1), so the unit stages its source rows once and
// writes each output row segment whole: adjacent float pairs, full sectors.
__host__ __device__ inline int unit_tile(const ConvTcArgs& a, int u, int g) {
  if (a.group == 1) return u;
  const int p = u < a.c.f[0].ntiles ? 0 : 1;
  return a.c.f[2 * p + g].tile0 + (p ? u - a.c.f[0].ntiles : u);
}

__host__ __device__ inline ConvTile conv_tile(const ConvPlan& c, int R, int t) {
  ConvTile T{};
  int q = 0;
  while (q + 1 < c.nph && t >= c.f[q + 1].tile0) ++q;
  const ConvPhase& f = c.f[q];
  const int Pf = f.Hf * f.Wf;
  T.f = q;
  T.m0 = (t - f.tile0) * 128;
  T.mend = T.m0 + 128 < R * Pf ? T.m0 + 128 : R * Pf;
  T.r0 = f.dPf.div(T.m0);
  T.nrt = f.dPf.div(T.mend - 1) - T.r0 + 1;
  T.sh0 = 0;
  T.nsh = c.Hs;
  if (T.nrt == 1) {
    const int i_lo = f.dWf.div(T.m0 - T.r0 * Pf), i_hi = f.dWf.div(T.mend - 1 - T.r0 * Pf);
    const int s = c.dir == 0 ? 1 : c.stride;
    const int o_lo = f.ph + s * i_lo, o_hi = f.ph + s * i_hi;   // output rows
    int lo, hi;
    if (c.dir == 0) {
      lo = o_lo * c.stride - c.pad;
      hi = o_hi * c.stride + c.k - 1 - c.pad;
    } else {
      const int x = o_lo + c.pad - (f.rh + s * (f.nkh - 1));   // a multiple of s when >= 0
      lo = x > 0 ? c.dS.div(x) : 0;
      hi = c.dS.div(o_hi + c.pad - f.rh);
    }
    lo = lo < 0 ? 0 : lo;
    hi = hi > c.Hs - 1 ? c.Hs - 1 : hi;
    T.sh0 = lo;
    T.nsh = hi >= lo ? hi - lo + 1 : 0;
  }
  return T;
}
// Tile ranges of the phases for a batch of R rows; returns the tile count.
inline int conv_set_tiles(ConvPlan& c, int R) {
  int n = 0;
  c.dS = FastDiv(static_cast<uint32_t>(c.stride));
  for (int q = 0; q < c.nph; ++q) {
    c.f[q].dPf = FastDiv(static_cast<uint32_t>(std::max(1, c.f[q].Hf * c.f[q].Wf)));
    c.f[q].dWf = FastDiv(static_cast<uint32_t>(std::max(1, c.f[q].Wf)));
    c.f[q].tile0 = n;
    c.f[q].ntiles = (R * c.f[q].Hf * c.f[q].Wf + 127) / 128;
    n += c.f[q].ntiles;
  }
  return n;
}

// Staging of a unit's source rows in shared memory, channel innermost: one
// item = 8 channels of one pixel; consecutive producer threads take
// consecutive pixels of the same channel group, so each load reads a
// contiguous run of a channel's row. A thread's first kStageAhead items are
// loaded into registers one unit ahead (stage_load, issued before the current
// unit's A blocks are built) and written out at the start of their unit
// (stage_store), which also loads and writes any further items directly. The
// loads read a valid channel unconditionally (the last one for the padding
// channels) and the padding is zeroed at the store, so nothing consumes a
// loaded value before the store: the loads stay in flight. Chunk cg of pixel
// p sits at chunk position cg ^ (p & smask) of the pixel (smask = channel
// groups - 1 when that is a power of two), so that the 16-byte accesses of
// consecutive pixels, here and in the A-block build, fall in distinct banks.
constexpr int kStageAhead = 4;
struct StageAhead {
  uint32_t v[kStageAhead][8];
  int dst[kStageAhead];   // element offset in the staging buffer, -1 = none
  int nv[kStageAhead];    // real channels of the item (the rest is padding)
};
struct StageGeom {
  int npix, cgroups, nitems, smask;
};
__device__ __forceinline__ int stage_smask(const ConvPlan& c) {
  const int cg = c.Csp / 8;
  return (cg & (cg - 1)) == 0 ? cg - 1 : 0;
}
__device__ __forceinline__ StageGeom stage_geom(const ConvPlan& c, const ConvTile& T) {
  StageGeom G;
  G.npix = T.nsh * c.Ws;
  G.cgroups = c.Csp / 8;
  G.nitems = T.nrt * G.npix * G.cgroups;
  G.smask = stage_smask(c);
  return G;
}
// the item's position: pixel pw of the staged rows, channel group cg, batch row rr
__device__ __forceinline__ void stage_pos(const StageGeom& G, int item, int& pw, int& cg, int& rr) {
  pw = item % G.npix;
  cg = (item / G.npix) % G.cgroups;
  rr = item / (G.npix * G.cgroups);
}
__device__ __forceinline__ int stage_off(const ConvPlan& c, const StageGeom& G, int pw, int cg, int rr) {
  return (rr * G.npix + pw) * c.Csp + ((cg ^ (pw & G.smask)) << 3);
}
__device__ __forceinline__ void stage_item_load(const ConvTcArgs& a, const ConvTile& T, int pw, int cg, int rr,
                                                uint32_t (&v)[8]) {
  const ConvPlan& c = a.c;
  const int HW = c.Hs * c.Ws;
  const __nv_bfloat16* sp = a.src + (int64_t)(T.r0 + rr) * (c.Cs * HW) + (T.sh0 * c.Ws + pw);
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) v[cc] = __bfloat16_as_ushort(sp[min(cg * 8 + cc, c.Cs - 1) * HW]);
}
__device__ __forceinline__ void stage_item_store(__nv_bfloat16* dst, const uint32_t (&v)[8], int nv) {
  uint32_t w[8];
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) w[cc] = cc < nv ? v[cc] : 0u;
  *reinterpret_cast<uint4*>(dst) =
      make_uint4(w[0] | (w[1] << 16), w[2] | (w[3] << 16), w[4] | (w[5] << 16), w[6] | (w[7] << 16));
}
__device__ __forceinline__ void stage_load(const ConvTcArgs& a, const ConvTile& T, int ptid, StageAhead& sa) {
  const StageGeom G = stage_geom(a.c, T);
  int pw = 0, cg = 0, rr = 0;
  if (ptid < G.nitems) stage_pos(G, ptid, pw, cg, rr);   // later items by additions
#pragma unroll
  for (int q = 0; q < kStageAhead; ++q) {
    const int item = ptid + q * kConvProdThreads;
    sa.dst[q] = -1;
    if (item < G.nitems) {
      stage_item_load(a, T, pw, cg, rr, sa.v[q]);
      sa.dst[q] = stage_off(a.c, G, pw, cg, rr);
      sa.nv[q] = a.c.Cs - cg * 8;
      pw += kConvProdThreads;
      while (pw >= G.npix) {
        pw -= G.npix;
        if (++cg == G.cgroups) { cg = 0; ++rr; }
      }
    }
  }
}
__device__ __forceinline__ void stage_store(const ConvTcArgs& a, const ConvTile& T, int ptid, const StageAhead& sa,
                                            __nv_bfloat16* stg) {
#pragma unroll
  for (int q = 0; q < kStageAhead; ++q)
    if (sa.dst[q] >= 0) stage_item_store(stg + sa.dst[q], sa.v[q], sa.nv[q]);
  const StageGeom G = stage_geom(a.c, T);
  int item = ptid + kStageAhead * kConvProdThreads;
  if (item >= G.nitems) return;
  int pw, cg, rr;
  stage_pos(G, item, pw, cg, rr);
  for (; item < G.nitems; item += kConvProdThreads) {
    uint32_t v[8];
    stage_item_load(a, T, pw, cg, rr, v);
    stage_item_store(stg + stage_off(a.c, G, pw, cg, rr), v, a.c.Cs - cg * 8);
    pw += kConvProdThreads;   // the next item's position by additions
    while (pw >= G.npix) {
      pw -= G.npix;
      if (++cg == G.cgroups) { cg = 0; ++rr; }
    }
  }
}

__global__ void __launch_bounds__(kConvThreads, 1) k_conv_tc(const __grid_constant__ ConvTcArgs a) {
  const ConvPlan& c = a.c;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const ConvSmem lay = conv_smem_layout(c.Kp, c.Np, a.stg_rows, c.Ws, c.Csp, a.stg_bufs, a.nb2);
  uint8_t* As = smem;
  uint8_t* Bs = smem + lay.b_off;
  __nv_bfloat16* stg = reinterpret_cast<__nv_bfloat16*>(smem + lay.stg_off);
  uint32_t* tab = reinterpret_cast<uint32_t*>(smem + lay.tab_off);
  uint64_t* a_full = reinterpret_cast<uint64_t*>(smem + lay.bar_off);   // [kConvStages]
  uint64_t* a_empty = a_full + kConvStages;                              // [kConvStages]
  uint64_t* acc_full = a_empty + kConvStages;                            // [2]
  uint64_t* acc_empty = acc_full + 2;                                    // [2]
  volatile int* abort_flag = reinterpret_cast<volatile int*>(acc_empty + 2);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2) + 2;

  griddep_launch();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int q = 0; q < kConvStages; ++q) {
      mbar_init(&a_full[q], kConvProdThreads);
      mbar_init(&a_empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&acc_full[q], 1);
      mbar_init(&acc_empty[q], kConvEpiWarps * 32);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * a.group * a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // weights into shared memory, tile kb = K columns [64 kb, 64 kb + 64), swizzled rows
  {
    const int chunks = c.Kp / 8;   // 16-byte chunks per weight row
    for (int idx = tid; idx < c.Np * chunks; idx += kConvThreads) {
      const int n = idx / chunks, ch = idx - n * chunks;
      const int kb = ch >> 3, j = ch & 7;
      const uint4 v = *reinterpret_cast<const uint4*>(a.Wp + (int64_t)n * c.Kp + ch * 8);
      *reinterpret_cast<uint4*>(Bs + kb * c.Np * kRowBytes + n * kRowBytes + ((j ^ (n & 7)) << 4)) = v;
    }
    // the second weight operand's tiles after the first's
    const int chunks2 = a.nb2 * 8;
    for (int idx = tid; idx < c.Np * chunks2; idx += kConvThreads) {
      const int n = idx / chunks2, ch = idx - n * chunks2;
      const int kb = ch >> 3, j = ch & 7;
      const uint4 v = *reinterpret_cast<const uint4*>(a.Wp2 + (int64_t)n * chunks2 * 8 + ch * 8);
      *reinterpret_cast<uint4*>(Bs + (c.Kp / 64 + kb) * c.Np * kRowBytes + n * kRowBytes + ((j ^ (n & 7)) << 4)) = v;
    }
  }
  // chunk table: for the 8 K columns of chunk x (a phase's k-block kb, chunk
  // j): tap (a, b) of the phase and source channel c0, or 0 = no tap
  for (int q = 0; q < c.nph; ++q) {
    const ConvPhase& f = c.f[q];
    for (int x = tid; x < f.nkb * 8; x += kConvThreads) {
      const int kk = x * 8, tt = kk / c.Csp, c0 = kk - tt * c.Csp;
      uint32_t e = 0;
      if (tt < f.nkh * f.nkw) e = 1u | (uint32_t)(tt / f.nkw) << 1 | (uint32_t)(tt % f.nkw) << 9 | (uint32_t)c0 << 17;
      tab[f.kb0 * 8 + x] = e;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  griddep_wait();   // the source maps belong to earlier kernels

  const int HW = c.Hs * c.Ws, src_dim = c.Cs * HW, out_dim = c.Co * c.Ho * c.Wo;
  const int R = (int)a.R;
  const int s_out = c.dir == 0 ? 1 : c.stride;     // output-pixel step within a phase

  if (warp >= kConvEpiWarps && warp < kConvEpiWarps + kConvProdWarps) {
    // ---------------- producers: stage the reachable source rows, build A blocks
    const int ptid = tid - kConvEpiWarps * 32;
    const int row = ptid & (BM - 1), half = ptid >> 7;   // GEMM row; chunks 4*half .. 4*half+3
    const int smask = stage_smask(c);   // staging chunk swizzle
    const bool csp32 = (c.Csp & 31) == 0;    // a thread's four chunks of a block share one tap
    uint32_t g = 0;
    const int stg_elems = a.stg_rows * c.Ws * c.Csp;
    StageAhead sa;
    ConvTile Tn{};
    if (blockIdx.x < (unsigned)a.units) {
      Tn = conv_tile(c, R, unit_tile(a, blockIdx.x, 0));
      stage_load(a, Tn, ptid, sa);
    }
    int cur = 0;
    for (int u = blockIdx.x; u < a.units; u += gridDim.x) {
      // one staging buffer: wait until all producers finished the previous
      // unit's A blocks. Two: the buffer was last read two units ago, before
      // every producer passed the previous unit's staging barrier.
      if (a.stg_bufs == 1 && prod_sync_or(*abort_flag != 0)) break;
      const ConvTile T = Tn;
      __nv_bfloat16* sbuf = stg + cur * stg_elems;
      stage_store(a, T, ptid, sa, sbuf);
      if (prod_sync_or(*abort_flag != 0)) break;   // staging complete
      // the next unit's loads fly while this unit's A blocks are built
      const int un = u + (int)gridDim.x;
      if (un < a.units) {
        Tn = conv_tile(c, R, unit_tile(a, un, 0));
        stage_load(a, Tn, ptid, sa);
      }
      if (a.stg_bufs == 2) cur ^= 1;
      bool quit = false;
      for (int gs = 0; gs < a.group && !quit; ++gs) {
      // the unit's tiles share rows, pixels and staged source rows
      const ConvPhase& f = c.f[gs ? conv_tile(c, R, unit_tile(a, u, gs)).f : T.f];
      const int Pf = f.Hf * f.Wf;
      // this thread's GEMM row: batch row r, output pixel (oh, ow); its source
      // pixel for tap (a, b) is (bh + sg_tap * a, bw + sg_tap * b)
      const int m = T.m0 + row;
      const bool mv = m < T.mend;
      const int r = mv ? f.dPf.div(m) : 0;
      const int pos = mv ? m - r * Pf : 0;
      const int pi = f.dWf.div(pos);
      const int oh = f.ph + s_out * pi, ow = f.pw + s_out * (pos - pi * f.Wf), rl = r - T.r0;
      const int bh = c.dir == 0 ? oh * c.stride - c.pad : c.dS.div(oh + c.pad - f.rh);
      const int bw = c.dir == 0 ? ow * c.stride - c.pad : c.dS.div(ow + c.pad - f.rw);
      const int sg_tap = c.dir == 0 ? 1 : -1;
      const __nv_bfloat16* srow = sbuf + rl * T.nsh * c.Ws * c.Csp;
      for (int kb = 0; kb < f.nkb; ++kb, ++g) {
        const int sg = g % kConvStages;
        if (*abort_flag) { quit = true; break; }   // no barrier inside this loop: leaving alone is safe
        if (g >= kConvStages && !mbar_wait_idle(&a_empty[sg], ((g / kConvStages) - 1) & 1)) {
          *abort_flag = 1;
          quit = true;
          break;
        }
        uint8_t* At = As + sg * kTileA;
        if (csp32) {
          // four chunks of one tap (the tap's channels are a multiple of 32):
          // one table entry, one bounds check, one staged pixel
          const uint32_t e = tab[(f.kb0 + kb) * 8 + half * 4];
          uint4 v[4];
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) v[jj] = make_uint4(0u, 0u, 0u, 0u);
          if (mv && (e & 1u)) {
            const int sh = bh + sg_tap * (int)((e >> 1) & 0xFFu), sw = bw + sg_tap * (int)((e >> 9) & 0xFFu);
            if (sh >= T.sh0 && sh < T.sh0 + T.nsh && sh < c.Hs && sw >= 0 && sw < c.Ws) {
              const int pix = (sh - T.sh0) * c.Ws + sw;
              const __nv_bfloat16* sp = srow + pix * c.Csp;
              const int q0 = (int)(e >> 20), xm = pix & smask;
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) v[jj] = *reinterpret_cast<const uint4*>(sp + (((q0 + jj) ^ xm) << 3));
            }
          }
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int j = half * 4 + jj;
            *reinterpret_cast<uint4*>(At + row * kRowBytes + ((j ^ (row & 7)) << 4)) = v[jj];
          }
        } else {
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int j = half * 4 + jj;
            const uint32_t e = tab[(f.kb0 + kb) * 8 + j];
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (mv && (e & 1u)) {
              const int sh = bh + sg_tap * (int)((e >> 1) & 0xFFu), sw = bw + sg_tap * (int)((e >> 9) & 0xFFu);
              if (sh >= T.sh0 && sh < T.sh0 + T.nsh && sh < c.Hs && sw >= 0 && sw < c.Ws) {
                const int pix = (sh - T.sh0) * c.Ws + sw;
                v = *reinterpret_cast<const uint4*>(srow + pix * c.Csp + (((e >> 20) ^ (pix & smask)) << 3));
              }
            }
            *reinterpret_cast<uint4*>(At + row * kRowBytes + ((j ^ (row & 7)) << 4)) = v;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&a_full[sg]);
      }
      }
    }
  } else if (warp == kConvEpiWarps + kConvProdWarps) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t id = idesc(1u, BM, c.Np);
      uint32_t g = 0, it = 0;
      for (int u = blockIdx.x; u < a.units; u += gridDim.x, ++it) {
        if (*abort_flag) break;
        const uint32_t b = it & 1;
        if (it >= 2 && !mbar_wait_idle(&acc_empty[b], ((it >> 1) - 1) & 1)) { *abort_flag = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        bool ok = true;
        for (int gs = 0; gs < a.group && ok; ++gs) {
          const ConvPhase& f = c.f[conv_tile(c, R, unit_tile(a, u, gs)).f];
          const uint32_t acc = tmem + (b * a.group + gs) * a.tmem_cols;
          for (int kb = 0; kb < f.nkb; ++kb, ++g) {
            const int sg = g % kConvStages;
            if (!mbar_wait_idle(&a_full[sg], (g / kConvStages) & 1)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ab = smem_u32(As + sg * kTileA), bb = smem_u32(Bs + (f.kb0 + kb) * c.Np * kRowBytes);
#pragma unroll
            for (int k4 = 0; k4 < kRowBytes / 32; ++k4)
              umma<0>(acc, sdesc(ab + k4 * 32), sdesc(bb + k4 * 32), id, (kb | k4) != 0);
            const int t2 = a.nb2 > 0 ? a.b2map[f.kb0 + kb] : -1;
            if (t2 >= 0) {   // the same A block against the second weight operand
              const uint32_t bb2 = smem_u32(Bs + (c.Kp / 64 + t2) * c.Np * kRowBytes);
#pragma unroll
              for (int k4 = 0; k4 < kRowBytes / 32; ++k4) umma<0>(acc, sdesc(ab + k4 * 32), sdesc(bb2 + k4 * 32), id, 1);
            }
            umma_commit(&a_empty[sg]);   // the stage is free once these MMAs have read it
          }
        }
        if (!ok) { *abort_flag = 1; break; }
        umma_commit(&acc_full[b]);     // the unit's accumulators are complete
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: TMEM -> global, channel-major output
    uint32_t it = 0;
    for (int u = blockIdx.x; u < a.units; u += gridDim.x, ++it) {
      // decisions are warp-uniform: the TMEM loads below are warp-collective
      if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
      const ConvTile T = conv_tile(c, R, unit_tile(a, u, 0));
      const ConvPhase& f = c.f[T.f];
      const int Pf = f.Hf * f.Wf;
      const uint32_t b = it & 1;
      if (!__all_sync(0xffffffffu, mbar_wait_idle(&acc_full[b], (it >> 1) & 1))) { *abort_flag = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int erow = warp * 32 + lane;
      const int em = T.m0 + erow;
      const int er = f.dPf.div(em);
      const int epos = em - er * Pf;
      const int epi = f.dWf.div(epos);
      const int eoh = f.ph + s_out * epi, eow = f.pw + s_out * (epos - epi * f.Wf);
      float* dst = a.out + (int64_t)er * out_dim + (eoh * c.Wo + eow);
      const int64_t cstride = (int64_t)c.Ho * c.Wo;
      const uint32_t tl = tmem + b * a.group * a.tmem_cols + (static_cast<uint32_t>(warp * 32) << 16);
      if (a.group == 1) {
        for (int col = 0; col < c.Np; col += 32) {
          uint32_t v[32];
          tmem_ld32(tl + col, v);
          if (em < T.mend) {
#pragma unroll
            for (int t = 0; t < 32; ++t)
              if (col + t < c.Co) dst[(col + t) * cstride] = __uint_as_float(v[t]);
          }
        }
      } else {
        // phase (ph, 0) at column eow = 2j, phase (ph, 1) at 2j + 1: one
        // 8-byte store per channel (Wo and the row offsets are even)
        for (int col = 0; col < c.Np; col += 32) {
          uint32_t v0[32], v1[32];
          tmem_ld32(tl + col, v0);
          tmem_ld32(tl + a.tmem_cols + col, v1);
          if (em < T.mend) {
#pragma unroll
            for (int t = 0; t < 32; ++t)
              if (col + t < c.Co)
                *reinterpret_cast<float2*>(dst + (col + t) * cstride) =
                    make_float2(__uint_as_float(v0[t]), __uint_as_float(v1[t]));
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&acc_empty[b]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * a.group * a.tmem_cols)
                 : "memory");
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

// 2-D map of a row-major [rows, cols] matrix (row stride ld elements, 0: cols),
// box of box_rows x 128 bytes.
bool make_map(CUtensorMap* m, const void* base, bool bf16, int64_t rows, int64_t cols, int box_rows, int64_t ld = 0) {
  const int es = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld ? ld : cols) * es};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kRowBytes / es), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  return g_encode(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KIND, int BNT>
bool launch_tc_bn(cudaStream_t st, int64_t M, int N, int K, const void* A, const void* B, const void* Blo, float* C,
                  int64_t lda, int64_t ldb) {
  using Cfg = TcCfg<KIND, BNT>;
  smem_opt_in(reinterpret_cast<const void*>(k_gemm_tc<KIND, BNT>), Cfg::kSmem);
  const bool bf = KIND == 0;
  CUtensorMap ta{}, tb{}, tblo{}, tc{};
  if (!make_map(&ta, A, bf, M, K, BM, lda) || !make_map(&tb, B, bf, N, K, BNT, ldb)) return false;
  if (KIND == 1) {
    if (!make_map(&tblo, Blo, bf, N, K, BNT, ldb)) return false;
  } else {
    tblo = tb;
  }
  // C through bulk tensor stores: 16-byte aligned base and row stride
  const int c_tma = (reinterpret_cast<uintptr_t>(C) & 15) == 0 && (N & 3) == 0 && make_map(&tc, C, false, M, N, 32);
  dim3 grid((N + BNT - 1) / BNT, static_cast<unsigned>((M + BM - 1) / BM));
  launch_pdl(k_gemm_tc<KIND, BNT>, grid, dim3(tc_threads<KIND>()), Cfg::kSmem, st, ta, tb, tblo, tc, c_tma,
             static_cast<int>(M), N, K, C);
  return true;
}

// Tile width of the GEMMs: 128 columns, or 224 where the
// fewer waves of wider tiles take less time (a CTA's MMA time grows with its
// width): the 9216 x 784 product onto the MLP's input layer runs 288 CTAs in
// 1.9 waves instead of 504 in 3.3.
inline int tc_tile_cols(int64_t M, int N) {
  const int64_t rows = (M + BM - 1) / BM;
  auto cost = [&](int bn) { return ((rows * ((N + bn - 1) / bn) + 151) / 152) * bn; };
  return cost(224) < cost(128) ? 224 : 128;
}

template <int KIND>
bool launch_tc(cudaStream_t st, int64_t M, int N, int K, const void* A, const void* B, const void* Blo, float* C,
               int64_t lda = 0, int64_t ldb = 0) {
  if (tc_tile_cols(M, N) == 224) return launch_tc_bn<KIND, 224>(st, M, N, K, A, B, Blo, C, lda, ldb);
  return launch_tc_bn<KIND, BN>(st, M, N, K, A, B, Blo, C, lda, ldb);
}

}  // namespace

bool tc_available(int K, bool bf16) {
  // TMA needs 16-byte row strides; the kernel tiles rows by 128.
  if (!encoder()) return false;
  return bf16 ? (K % 8 == 0) : (K % 4 == 0);
}

bool gemm_tc_bf16(cudaStream_t st, int64_t M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C,
                  double flop_scale) {
  if (M <= 0 || N <= 0) return true;
  if (!tc_available(K, true) || M > (int64_t)INT32_MAX) return false;
  if (!(reg_check(A, (double)M * K * 2, "tc A") & reg_check(B, (double)N * K * 2, "tc B") &
        reg_check(C, (double)M * N * 4, "tc C")))
    return true;  // reported by the caller's launch status
  int tk = prof_begin(st, "gemm_tc_bf16", flop_scale * 2.0 * M * N * K,
                      ((double)M * K + (double)N * K) * 2 + (double)M * N * 4);
  bool ok = true;
  for (int rep = prof_repeats("gemm_tc_bf16"); rep > 0 && ok; --rep) ok = launch_tc<0>(st, M, N, K, A, B, nullptr, C);
  prof_end(st, tk);
  return ok;
}

bool gemm_tc_tf32x3(cudaStream_t st, int64_t M, int N, int K, const float* A, const float* B, const float* Blo,
                    float* C) {
  if (M <= 0 || N <= 0) return true;
  if (!tc_available(K, false) || M > (int64_t)INT32_MAX) return false;
  if (!(reg_check(A, (double)M * K * 4, "tc A") & reg_check(B, (double)N * K * 4, "tc B") &
        reg_check(Blo, (double)N * K * 4, "tc B lo") & reg_check(C, (double)M * N * 4, "tc C")))
    return true;
  int tk = prof_begin(st, "gemm_tc_tf32x3", 2.0 * M * N * K, (double)M * K * 4 + (double)N * K * 8 + (double)M * N * 4);
  bool ok = true;
  for (int rep = prof_repeats("gemm_tc_tf32x3"); rep > 0 && ok; --rep) ok = launch_tc<1>(st, M, N, K, A, B, Blo, C);
  prof_end(st, tk);
  return ok;
}

// ------------------------------------------------------------------ float64 by exact slices
namespace {
// Row exponent e with max |A[r, :]| < 2^e, from the bit pattern of the
// largest magnitude m (normal: m = 1.f 2^(E-1023) < 2^(E-1022)); 0 for m = 0.
__device__ __forceinline__ int exp_above(double m) {
  const long long bits = __double_as_longlong(m);
  const int E = static_cast<int>((bits >> 52) & 0x7ff);
  if (E != 0) return E - 1022;
  if (m == 0.0) return 0;
  const unsigned long long f = static_cast<unsigned long long>(bits) & ((1ull << 52) - 1);
  return -1074 + (64 - __clzll(static_cast<long long>(f)));   // subnormal: f 2^-1074 < 2^(bit length - 1074)
}

// One warp per row. x = A[r, k] 2^-e lies in (-1, 1); its first b * s bits
// after the binary point, X = trunc(|x| 2^(bs)), come from the mantissa by an
// integer shift, and slice i (1 = most significant) is bits
// b (s - i) .. b (s - i + 1) - 1 of X with the sign of x: the same integers as
// s rounds of x *= 2^b, a = trunc(x), x -= a. |a| < 2^b, exact in bf16. A
// row holding a non-finite value gets the exponent kSliceBadExp and zeros.
__global__ void k_slice_rows(int64_t M, int K, const double* __restrict__ A, int b, int s, int reverse,
                             __nv_bfloat16* __restrict__ planes, int32_t* __restrict__ exps) {
  const int64_t row = static_cast<int64_t>(blockIdx.x) * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= M) return;
  const double* a = A + row * K;
  double mx = 0.0;
  bool bad = false;
  for (int k = lane; k < K; k += 32) {
    const double v = a[k];
    bad |= !isfinite(v);
    mx = fmax(mx, fabs(v));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  bad = __any_sync(0xffffffffu, bad);
  const int e = bad ? 0 : exp_above(mx);
  if (lane == 0) exps[row] = bad ? kSliceBadExp : e;
  const int bs = b * s;   // <= 56
  const unsigned long long digit = (1ull << b) - 1;
  __nv_bfloat16* out = planes + row * static_cast<int64_t>(s) * K;
  for (int k = lane; k < K; k += 32) {
    const long long bits = bad ? 0 : __double_as_longlong(a[k]);
    const int E = static_cast<int>((bits >> 52) & 0x7ff);
    const unsigned long long m = (static_cast<unsigned long long>(bits) & ((1ull << 52) - 1)) | (E ? (1ull << 52) : 0);
    // |x| 2^bs = m 2^(max(E,1) - 1075 - e + bs)
    const int sh = (E ? E : 1) - 1075 - e + bs;
    const unsigned long long X = sh >= 0 ? (sh < 64 ? m << sh : 0) : (-sh < 64 ? m >> -sh : 0);
    const float sg = bits < 0 ? -1.f : 1.f;
    for (int i = 1; i <= s; ++i) {
      const float d = static_cast<float>((X >> (b * (s - i))) & digit);
      out[static_cast<int64_t>(reverse ? s - i : i - 1) * K + k] = __float2bfloat16_rn(sg * d);
    }
  }
}

// y[r, c] = sum over t = 2 .. s+1 of T_t[r, c] 2^(e_r + f_c - b t) (T_t the
// exact integer sums of the slice GEMMs, plane t - 2 of T), formed exactly as
// the 128-bit integer sum_t T_t 2^(b (s + 1 - t)) and rounded once to the
// nearest float64 (integer operations only: float64 arithmetic is scarce on
// this part); yabs[r, c] = 2^(e_r + f_c) K rounded up to float. Block = 8 rows
// of y, threads along c.
__device__ __forceinline__ double scale_pow2(double d, int k) {   // d * 2^k, d normal
  const int E = static_cast<int>((__double_as_longlong(d) >> 52) & 0x7ff);
  if (E + k >= 1 && E + k <= 2046)
    return __longlong_as_double(__double_as_longlong(d) + (static_cast<long long>(k) << 52));
  return ldexp(d, k);
}
__device__ __forceinline__ double i128_to_double_scaled(__int128 v, int k) {   // round(v) * 2^k
  if (v == 0) return 0.0;
  const bool neg = v < 0;
  const unsigned __int128 u = neg ? static_cast<unsigned __int128>(-v) : static_cast<unsigned __int128>(v);
  const unsigned long long hi = static_cast<unsigned long long>(u >> 64), lo = static_cast<unsigned long long>(u);
  const int nbits = hi ? 128 - __clzll(static_cast<long long>(hi)) : 64 - __clzll(static_cast<long long>(lo));
  int sh = nbits - 53;
  unsigned long long mant;
  if (sh > 0) {
    mant = static_cast<unsigned long long>(u >> sh);
    const unsigned __int128 rem = u & ((static_cast<unsigned __int128>(1) << sh) - 1);
    const unsigned __int128 half = static_cast<unsigned __int128>(1) << (sh - 1);
    if (rem > half || (rem == half && (mant & 1))) ++mant;   // to nearest, ties to even
    if (mant >> 53) {
      mant >>= 1;
      ++sh;
    }
  } else {
    mant = lo << -sh;
  }
  // value = mant 2^(sh + k), 2^52 <= mant < 2^53
  const int ef = 52 + sh + k + 1023;
  if (ef >= 1 && ef <= 2046)
    return __longlong_as_double((neg ? (1ll << 63) : 0ll) | (static_cast<long long>(ef) << 52) |
                                static_cast<long long>(mant & ((1ull << 52) - 1)));
  const double m = ldexp(static_cast<double>(mant), sh + k);   // outside the normal range (exact mant)
  return neg ? -m : m;
}
__global__ void k_slice_combine(int64_t M, int N, int b, int s, double kred, const float* __restrict__ T,
                                const int32_t* __restrict__ er, const int32_t* __restrict__ fc,
                                double* __restrict__ y, float* __restrict__ yabs) {
  const int64_t plane = M * N;
  const int64_t r1 = min(M, static_cast<int64_t>(blockIdx.x + 1) * 8);
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * 8; r < r1; ++r) {
    const int e = er[r];
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
      const int64_t i = r * N + c;
      const int f = __ldg(fc + c);
      if (e >= kSliceBadExp || f >= kSliceBadExp) {
        y[i] = __longlong_as_double(0x7ff8000000000000ll);
        yabs[i] = __int_as_float(0x7f800000);
        continue;
      }
      __int128 acc = 0;
      for (int t = 2; t <= s + 1; ++t)
        acc += static_cast<__int128>(__float2int_rz(__ldg(T + (t - 2) * plane + i))) *
               (static_cast<__int128>(1) << (b * (s + 1 - t)));
      y[i] = i128_to_double_scaled(acc, e + f - b * (s + 1));
      yabs[i] = __double2float_ru(scale_pow2(kred, e + f));
    }
  }
}
}  // namespace

bool slice_params(int K, int& b, int& s, double& cerr) {
  // at least 50 bits of each operand, and every partial sum of a slice GEMM
  // an integer below 2^22 (exact in the fp32 accumulator with room to spare)
  if (K <= 0 || K % 8 != 0) return false;
  for (b = 8; b >= 2; --b) {
    s = (50 + b - 1) / b;
    const double m = static_cast<double>((1 << b) - 1);
    if (static_cast<double>(s) * K * m * m < 4194304.0) break;
  }
  if (b < 2) return false;
  // truncation of both operands (2 + slop), the pairs i + j > s + 1 left out
  // ((s - 1) / (1 - 2^-b)), both relative to 2^-bs; the rounding of the sum
  // of the s terms to float64 (one rounding of the exact sum; bounded here as
  // gamma_(s-1) times the terms' magnitudes, <= 1 / (1 - 2^-b)^2); everything
  // in units of 2^(e_r + f_c) K
  const double u = std::ldexp(1.0, -53), r = 1.0 - std::ldexp(1.0, -b);
  const double gam = (s - 1) * u / (1.0 - (s - 1) * u);
  cerr = (std::ldexp(2.01 + (s - 1) / r, -b * s) + gam / (r * r)) * (1.0 + std::ldexp(1.0, -20));
  return true;
}

bool slice_rows(cudaStream_t st, int64_t M, int K, const double* A, int b, int s, bool reverse,
                __nv_bfloat16* planes, int32_t* exps) {
  if (M <= 0) return true;
  if (!(reg_check(A, (double)M * K * 8, "slice A") & reg_check(planes, (double)M * s * K * 2, "slice planes") &
        reg_check(exps, (double)M * 4, "slice exps")))
    return true;   // reported by the caller's launch status
  int tk = prof_begin(st, "slice_f64", 0.0, (double)M * K * (8.0 + 2.0 * s));
  k_slice_rows<<<static_cast<unsigned>((M + 7) / 8), 256, 0, st>>>(M, K, A, b, s, reverse ? 1 : 0, planes, exps);
  prof_end(st, tk);
  return true;
}

bool gemm_f64_slices(cudaStream_t st, int64_t M, int N, int K, const double* A, const SliceB& B,
                     __nv_bfloat16* ap, int32_t* ae, float* T, double* y, float* yabs) {
  if (M <= 0 || N <= 0) return true;
  const int s = B.s;
  if (!B.planes || s < 1 || !tc_available(K, true) || M > (int64_t)INT32_MAX) return false;
  if (!(reg_check(B.planes, (double)N * s * K * 2, "slice B") & reg_check(B.exps, (double)N * 4, "slice B exps") &
        reg_check(T, (double)s * M * N * 4, "slice sums") & reg_check(y, (double)M * N * 8, "slice y") &
        reg_check(yabs, (double)M * N * 4, "slice yabs")))
    return true;   // reported by the caller's launch status
  slice_rows(st, M, K, A, B.b, s, false, ap, ae);
  // T_t for t = 2 .. s+1: A's slices 1 .. t-1 (a prefix of each row) against
  // B's t-1 .. 1 (a suffix of B's reversed rows), K' = (t - 1) K. Each launch
  // is counted with the share (t - 1) / (s (s + 1) / 2) of the product's
  // algorithmic flops 2 M N K, and the slices it reads and the sums it writes.
  const double pairs = 0.5 * s * (s + 1);
  const int64_t plane = M * (int64_t)N;
  bool ok = true;
  for (int t = 2; t <= s + 1 && ok; ++t) {
    int tk = prof_begin(st, "gemm_tc_f64_slices", 2.0 * M * N * K * (t - 1) / pairs,
                        ((double)M + N) * K * 2.0 * (t - 1) + (double)plane * 4.0);
    ok = launch_tc<0>(st, M, N, (t - 1) * K, ap, B.planes + static_cast<int64_t>(s - t + 1) * K, nullptr,
                      T + (t - 2) * plane, static_cast<int64_t>(s) * K, static_cast<int64_t>(s) * K);
    prof_end(st, tk);
  }
  if (!ok) return false;
  int tk = prof_begin(st, "slice_combine_f64", 0.0, (double)plane * (4.0 * s + 12.0));
  k_slice_combine<<<static_cast<unsigned>((M + 7) / 8), 256, 0, st>>>(M, N, B.b, s, static_cast<double>(K), T, ae,
                                                                        B.exps, y, yabs);
  prof_end(st, tk);
  return true;
}

bool conv_tc_fits(const LayerGeom& g, int dir, int Kp, int Np, int nb2) {
  ConvPlan c;
  if (!conv_plan(g, dir, c) || c.Kp != Kp || c.Np != Np || Np > 256) return false;
  if (nb2 > 0 && Kp / 64 > kConvMaxKb) return false;
  // the staging window grows with the row count until a tile spans whole
  // rows of every phase; a large row count gives the largest
  const int R = 1 << 16;
  conv_set_tiles(c, R);
  int rows = 0;
  for (int q = 0; q < c.nph; ++q) {
    const int Pf = c.f[q].Hf * c.f[q].Wf;
    for (int t = 0; t < std::min(c.f[q].ntiles, Pf + 1); ++t) {
      const ConvTile T = conv_tile(c, R, c.f[q].tile0 + t);
      rows = std::max(rows, T.nrt == 1 ? T.nsh : T.nrt * c.Hs);
    }
  }
  int tc = 32;
  while (tc < Np) tc <<= 1;
  return conv_smem_layout(Kp, Np, std::max(rows, 1), c.Ws, c.Csp, 1, nb2).total <= 227 * 1024 && 2 * tc <= 512;
}

bool conv_tc_bf16(cudaStream_t st, int64_t R, const LayerGeom& g, int dir, const __nv_bfloat16* Wp, int Kp, int Np,
                  const __nv_bfloat16* src, float* out, double flop_scale, const ConvSecondB* b2) {
  if (R <= 0) return true;
  ConvTcArgs a{};
  ConvPlan& c = a.c;
  if (!Wp || !conv_plan(g, dir, c) || c.Kp != Kp || c.Np != Np || Np > 256) return false;
  if (R * (int64_t)c.Ho * c.Wo >= (int64_t)INT32_MAX - 128) return false;   // 32-bit tile arithmetic
  a.R = R;
  const int tiles = conv_set_tiles(c, (int)R);
  // staging rows: the largest window over the tiles (tile starts repeat with
  // period P_f within a phase, so the first P_f tiles of each phase cover all)
  int rows = 0;
  for (int q = 0; q < c.nph; ++q) {
    const int Pf = c.f[q].Hf * c.f[q].Wf;
    for (int t = 0; t < std::min(c.f[q].ntiles, Pf + 1); ++t) {
      const ConvTile T = conv_tile(c, (int)R, c.f[q].tile0 + t);
      rows = std::max(rows, T.nrt == 1 ? T.nsh : T.nrt * c.Hs);
    }
  }
  a.stg_rows = std::max(rows, 1);
  int tc = 32;
  while (tc < Np) tc <<= 1;
  a.tmem_cols = tc;
  // pair the phases (ph, 0), (ph, 1) of a stride-2 transposed convolution
  a.group = 1;
  if (dir == 1 && c.stride == 2 && c.nph == 4 && c.Wo % 2 == 0 && 4 * tc <= 512 &&
      (reinterpret_cast<uintptr_t>(out) & 7) == 0) {
    bool pairs = true;
    for (int p = 0; p < 2; ++p) {
      const ConvPhase &f0 = c.f[2 * p], &f1 = c.f[2 * p + 1];
      pairs = pairs && f0.ph == f1.ph && f0.pw == 0 && f1.pw == 1 && f0.Hf == f1.Hf && f0.Wf == f1.Wf &&
              f0.ntiles == f1.ntiles;
    }
    if (pairs) a.group = 2;
  }
  a.units = a.group == 2 ? c.f[0].ntiles + c.f[2].ntiles : tiles;
  a.stg_bufs = 2;
  if (b2 && b2->nb2 > 0) {
    if (Kp / 64 > kConvMaxKb || (int)b2->map.size() != Kp / 64 || !b2->W) return false;
    a.Wp2 = b2->W;
    a.nb2 = b2->nb2;
    for (int q = 0; q < Kp / 64; ++q) a.b2map[q] = b2->map[q];
  }
  ConvSmem L = conv_smem_layout(Kp, Np, a.stg_rows, c.Ws, c.Csp, 2, a.nb2);
  if (L.total > 227 * 1024) {
    a.stg_bufs = 1;
    L = conv_smem_layout(Kp, Np, a.stg_rows, c.Ws, c.Csp, 1, a.nb2);
  }
  if (L.total > 227 * 1024) return false;
  // opted in per device and size
  if (!smem_opt_in(reinterpret_cast<const void*>(k_conv_tc), (size_t)L.total)) return false;
  int n_sm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (n_sm <= 0) n_sm = 1;
  a.src = src;
  a.Wp = Wp;
  a.out = out;
  const int src_dim = c.Cs * c.Hs * c.Ws, out_dim = c.Co * c.Ho * c.Wo;
  if (!(reg_check(src, (double)R * src_dim * 2, "conv src") & reg_check(Wp, (double)Np * Kp * 2, "conv W") &
        reg_check(a.Wp2, a.nb2 ? (double)Np * 64 * a.nb2 * 2 : 0.0, "conv W2") &
        reg_check(out, (double)R * out_dim * 4, "conv out")))
    return true;  // reported by the caller's launch status
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv_tc, kConvThreads, L.total);
  if (2 * a.group * tc > 512) return false;
  // TMEM columns of the resident CTAs (two buffers of `group` accumulators each)
  per_sm = std::max(1, std::min(per_sm, 512 / (2 * a.group * tc)));
  const int grid = std::min(a.units, n_sm * per_sm);
  // algorithmic work: the convolution's multiply-adds (2 flops each); bytes:
  // source read and output written once
  const double macs = (double)R * g.c_out * g.h_out * g.w_out * g.c_in * g.k * g.k;
  int tk = prof_begin(st, dir == 0 ? "conv_tc_bf16_fwd" : "conv_tc_bf16_T", flop_scale * 2.0 * macs,
                      (double)R * src_dim * 2 + (double)R * out_dim * 4);
  launch_pdl(k_conv_tc, dim3(grid), dim3(kConvThreads), L.total, st, a);
  prof_end(st, tk);
  return true;
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

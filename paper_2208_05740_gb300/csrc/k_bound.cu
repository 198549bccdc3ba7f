// Per-neuron kernels of the GCP-CROWN chain (Theorem 3.1, Lemma A.1, App. A).
//
// Thread mapping: a warp owns one row and 32 consecutive neurons of one layer
// (lane = neuron), so every per-(row, neuron) array is read and written as
// whole 128-byte lines. Cut multipliers gamma [R, N], split multipliers
// beta [R, M] and cut-entry values E [R, nnz] are row-major, so the sparse
// gathers of a warp stay inside one row's vector. Per-row objective partials
// are reduced across the warp in a fixed shuffle order and written per neuron
// chunk, then summed in a fixed order (deterministic results).
#include <cstdio>
#include <type_traits>

#include <cstdlib>
#include <algorithm>

#include "gcp_internal.cuh"

namespace gcp {

// First data-dependent index that failed its check: {code, index, limit}; the
// access is skipped. Read and cleared by take_device_error().
__device__ unsigned long long g_dev_err[3];

namespace {

constexpr int kWarpsPerBlock = 8;
// Span kernels: small blocks (two warps) spread the subdomains' warps evenly
// over the SMs; a block of eight left some SMs with half the warps of others.
constexpr int kSpanWarps = 2;
// The relaxation is capped at 72 registers (kEvalMinBlocks blocks of two
// warps per SM; its shared memory allows 15), so a launch spreads each span's
// rows over up to kEvalWarpsPerSM warps per SM: on the MLP's 2,048-warp
// launches, two warps per span at 27 warps per SM instead of 13.5 measured
// 47.3 against 48.3 ms per step.
constexpr int kEvalMinBlocks = 14;
constexpr int64_t kEvalWarpsPerSM = 26;

__device__ __noinline__ void dev_error(unsigned long long code, long long idx, long long lim) {
  if (atomicCAS(&g_dev_err[0], 0ull, code) == 0ull) {
    g_dev_err[1] = (unsigned long long)idx;
    g_dev_err[2] = (unsigned long long)lim;
  }
}

// First failed index check of a thread, reported once when the kernel ends
// (keeps function calls out of the load sequences of the hot kernels).
struct DevErr {
  unsigned code = 0;
  long long idx = 0, lim = 0;
  __device__ __forceinline__ void set(unsigned c, long long i, long long l) {
    if (!code) { code = c; idx = i; lim = l; }
  }
  __device__ __forceinline__ void flush() const {
    if (code) dev_error(code, idx, lim);
  }
};

// split entries of subdomain s, checked against the entry count and slots
__device__ __forceinline__ void split_range(const SplitsDev& sp, int s, int M, int& q0, int& q1) {
  q0 = sp.ptr[s];
  q1 = sp.ptr[s + 1];
  if (q0 < 0 || q1 < q0 || (int64_t)q1 > sp.n || q1 - q0 > M) {
    dev_error(3, s, sp.n);
    q0 = q1 = 0;
  }
}

template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <typename T>
__device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }

template <typename Top, typename T>
__device__ __forceinline__ Top cvt_out(T v) { return static_cast<Top>(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_out<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }

// x = hi + lo with hi = x rounded to tf32 (nearest, ties away) and lo exact.
__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  return __uint_as_float(h);
}

// Store an operand of the next GEMM, split into tf32 high and low parts when
// the 3-pass tf32 GEMM consumes it.
template <typename Top, typename T>
__device__ __forceinline__ void put_operand(Top* hi, float* lo, int64_t i, T v) {
  if constexpr (std::is_same<Top, float>::value) {
    if (lo) {
      const float h = tf32_hi(v);
      hi[i] = h;
      lo[i] = v - h;
      return;
    }
  }
  hi[i] = cvt_out<Top>(v);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_rd(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __dadd_rd(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Warp coordinates: a warp owns one 32-neuron chunk c of a layer (lane =
// neuron j = 32c + lane) and one subdomain s, i.e. the K spec rows
// r = sK .. sK+K-1. Everything that does not depend on the row (bounds,
// split hits, the chunk's cut entries) is loaded once per warp; each row then
// costs one round of independent loads.
struct ChunkWarp {
  int s, c, lane, j;
  bool on;
};
__device__ __forceinline__ bool chunk_warp(int S, int d, ChunkWarp& w) {
  w.s = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  w.c = blockIdx.y;
  w.lane = threadIdx.x & 31;
  w.j = w.c * 32 + w.lane;
  w.on = w.j < d;
  return w.s < S;
}

// The split (if any) of subdomain s on neuron j of `layer`: slot and sign.
// Lane q of the warp inspects split q (and 32 + q) of the subdomain.
__device__ __forceinline__ int lane_split(const SplitsDev& sp, int s, int M, int layer, int c, int lane, int& sign) {
  int q0, q1;
  split_range(sp, s, M, q0, q1);
  int slot = -1;
  sign = 0;
  for (int base = 0; base < q1 - q0; base += 32) {
    const int q = q0 + base + lane;
    int lay = -1, idx = -1, sg = 0;
    if (q < q1) {
      lay = sp.layer[q];
      idx = sp.index[q];
      sg = sp.sign[q];
    }
    unsigned m = __ballot_sync(0xffffffffu, lay == layer && (idx >> 5) == c);
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      const int tj = __shfl_sync(0xffffffffu, idx, b) & 31;
      const int tsg = __shfl_sync(0xffffffffu, sg, b);
      if (tj == lane) { slot = base + b; sign = tsg; }
    }
  }
  return slot;
}

// Cut entries of the chunk: entries of its neurons are contiguous in CSC
// order. For one batch of up to 32 entries lane q holds entry cb + q; neuron
// lanes collect their own entries with shuffles.
template <typename T>
struct ChunkCuts {
  int e0, e1;       // this lane's neuron entries
  int cb, ce;       // the chunk's entries (warp-uniform)
  int cut, kind, nrn_lane;  // entry cb + lane of the first batch
  T coef;
};
template <typename T>
__device__ __forceinline__ void chunk_cuts(const CutCSC<T>& c, int N, int d, int ch, int lane, ChunkCuts<T>& cc) {
  const int j = ch * 32 + lane;
  const int jl = j < d ? j : d, jh = j + 1 < d ? j + 1 : d;
  cc.e0 = __ldg(c.ptr + jl);
  cc.e1 = __ldg(c.ptr + jh);
  cc.cb = __shfl_sync(0xffffffffu, cc.e0, 0);
  cc.ce = __shfl_sync(0xffffffffu, cc.e1, 31);
  const bool bad = cc.e0 < cc.cb || cc.e1 < cc.e0 || cc.e1 > cc.ce;
  if (__any_sync(0xffffffffu, bad) || cc.cb < 0 || cc.ce < cc.cb || (int64_t)cc.ce > c.n_total) {
    if (lane == 0) dev_error(1, ch, c.n_total);
    cc.e0 = cc.e1 = cc.cb = cc.ce = 0;
  }
  cc.cut = -1; cc.kind = -1; cc.nrn_lane = 0; cc.coef = T(0);
  const int e = cc.cb + lane;
  if (e < cc.ce && lane < 32) {
    cc.cut = __ldg(c.cut + e);
    cc.kind = __ldg(c.kind + e);
    cc.nrn_lane = (__ldg(c.nrn + e) - ch * 32) & 31;
    cc.coef = __ldg(c.coef + e);
    if (cc.cut < 0 || cc.cut >= N) { dev_error(2, e, N); cc.cut = -1; cc.kind = -1; }
  }
}

// Certification variant: round-to-nearest sums with their round-up absolute
// sums and term counts (for Higham's bound), per kind. A batch holds 32
// consecutive entries of the chunk, entry b0 + q on lane q; entries of one
// (kind, neuron) form a run of lanes, whose first lane adds the run's terms
// one by one to the warp's shared accumulator of that (kind, neuron), so each
// sum is the recursive sum of its terms in CSC order (Higham's bound holds for
// any order). acc: the warp's 3 * 32 sums, then 3 * 32 absolute sums, then
// 3 * 32 counts, all zero on entry and again on return.
constexpr int kCertAcc = 3 * 32 * 2 * 8 + 3 * 32 * 4;   // bytes per warp
template <typename Tg>
__device__ __forceinline__ void cut_sums_row_cert(const CutCSC<double>& c, const ChunkCuts<double>& cc,
                                                  const Tg* grow, int N, int lane, double (&sum)[3],
                                                  double (&abs_)[3], int (&cnt_)[3], unsigned char* acc) {
  double* as = reinterpret_cast<double*>(acc);
  double* aa = as + 96;
  int* an = reinterpret_cast<int*>(aa + 96);
#pragma unroll
  for (int q = 0; q < 3; ++q) { sum[q] = 0.0; abs_[q] = 0.0; cnt_[q] = 0; }
  if (cc.cb == cc.ce) return;
  for (int b0 = cc.cb; b0 < cc.ce; b0 += 32) {
    int kd = cc.kind, cut = cc.cut, nl = cc.nrn_lane;
    double cf = cc.coef;
    if (b0 != cc.cb) {
      const int e = b0 + lane;
      kd = -1; cut = -1; cf = 0.0; nl = 0;
      if (e < cc.ce) {
        cut = __ldg(c.cut + e);
        kd = __ldg(c.kind + e);
        cf = __ldg(c.coef + e);
        nl = (__ldg(c.nrn + e) & 31);
        if (cut < 0 || cut >= N || kd < 0 || kd > 2) { dev_error(2, e, N); cut = -1; kd = -1; }
      }
    }
    // the chunk's neurons are 32-aligned, so the neuron within the chunk is
    // its index mod 32; lanes without an entry form runs of their own
    const bool has = cut >= 0 && kd >= 0 && kd <= 2;
    const int dest = has ? kd * 32 + nl : -1 - lane;   // in [0, 96) for an entry
    double val = 0.0, av = 0.0;
    if (has) {
      const double gv = (double)grow[cut];
      val = cf * gv;
      av = __dmul_ru(fabs(cf), fabs(gv));
    }
    const int prev = __shfl_up_sync(0xffffffffu, dest, 1);
    const bool cont = lane > 0 && prev == dest;
    const unsigned cm = __ballot_sync(0xffffffffu, cont);
    int len = 1;
    if (lane < 31) {
      const unsigned after = cm >> (lane + 1), all = 0xffffffffu >> (lane + 1);
      len += after == all ? 31 - lane : __ffs(~after) - 1;
    }
    const int run = cont ? 0 : len;
    const int maxrun = __reduce_max_sync(0xffffffffu, run);
    const bool head = run > 0 && has;
    if (head) {
      val = as[dest] + val;
      av = __dadd_ru(aa[dest], av);
    }
    for (int q = 1; q < maxrun; ++q) {
      const double u = __shfl_down_sync(0xffffffffu, val, q);
      const double ua = __shfl_down_sync(0xffffffffu, av, q);
      if (q < run) {
        val += u;
        av = __dadd_ru(av, ua);
      }
    }
    if (head) {
      as[dest] = val;
      aa[dest] = av;
      an[dest] += run;
    }
    __syncwarp();
  }
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    sum[t] = as[t * 32 + lane];
    abs_[t] = aa[t * 32 + lane];
    cnt_[t] = an[t * 32 + lane];
    as[t * 32 + lane] = 0.0;
    aa[t * 32 + lane] = 0.0;
    an[t * 32 + lane] = 0;
  }
  __syncwarp();
}

// zero a warp's certification accumulator
__device__ __forceinline__ void cert_acc_zero(unsigned char* acc, int lane) {
  double* as = reinterpret_cast<double*>(acc);
  int* an = reinterpret_cast<int*>(as + 192);
#pragma unroll
  for (int t = 0; t < 6; ++t) as[t * 32 + lane] = 0.0;
#pragma unroll
  for (int t = 0; t < 3; ++t) an[t * 32 + lane] = 0;
  __syncwarp();
}

// One ascent step on x. Adam (Kingma & Ba): bias-corrected moments m, v are
// read and updated in place (values, loaded by the caller ahead of time); the
// float chain uses the approximate square root and reciprocal divide (a step
// size, not a bound).
template <typename T>
__device__ __forceinline__ T step_apply(const StepArgs<T>& st, T x, T grad, T lr, T& m, T& v) {
  if (st.mode == 1) return x + lr * grad;
  m = st.b1 * m + (T(1) - st.b1) * grad;
  v = st.b2 * v + (T(1) - st.b2) * grad * grad;
  if constexpr (std::is_same<T, float>::value) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v * st.ic2));   // a step size, not a bound
    return x + lr * __fdividef(m * st.ic1, r + st.eps);
  } else {
    return x + lr * (m / st.c1) / (sqrt(v / st.c2) + st.eps);
  }
}

// ------------------------------------------------------------------ span kernels
// The per-neuron kernels of the chain (relaxation, adjoint, concretization)
// give each warp a span of 32*V consecutive neurons of one layer and one
// subdomain, i.e. its K spec rows: lane l holds neurons base + lV .. base +
// lV + V - 1, read and written as 16-byte vectors when V = 4 (float chains on
// layers whose width is a multiple of 4). Row-independent data (bounds, split
// hits, the span's cut entries) is set up once per warp.
template <int V>
struct SpanWarp {
  int s, c, lane, base, j0;
  bool on;              // the lane's V neurons exist (d is a multiple of V)
};
template <int V>
__device__ __forceinline__ bool span_warp(int S, int d, SpanWarp<V>& w) {
  w.s = blockIdx.x * kSpanWarps + (threadIdx.x >> 5);
  w.c = blockIdx.y;
  w.lane = threadIdx.x & 31;
  w.base = w.c * 32 * V;
  w.j0 = w.base + w.lane * V;
  w.on = w.j0 < d;
  return w.s < S;
}

template <int V, typename T>
__device__ __forceinline__ void ldv(const T* p, T (&o)[V]) {      // read-only during the kernel
  if constexpr (V == 4 && sizeof(T) == 4) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
  } else if constexpr (V == 2 && sizeof(T) == 4) {
    const float2 q = __ldg(reinterpret_cast<const float2*>(p));
    o[0] = q.x; o[1] = q.y;
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) o[v] = __ldg(p + v);
  }
}
template <int V, typename T>
__device__ __forceinline__ void ldv_rw(const T* p, T (&o)[V]) {   // also written by the kernel
  if constexpr (V == 4 && sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
  } else if constexpr (V == 2 && sizeof(T) == 4) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    o[0] = q.x; o[1] = q.y;
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) o[v] = p[v];
  }
}
template <int V, typename T>
__device__ __forceinline__ void stv(T* p, const T (&o)[V]) {
  if constexpr (V == 4 && sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  } else if constexpr (V == 2 && sizeof(T) == 4) {
    *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) p[v] = o[v];
  }
}

// Operand of the next GEMM for V neurons: tf32 high/low parts for the 3-pass
// tf32 GEMM, bf16 for the bf16 GEMM, or the value itself.
template <int V, typename Top, typename T>
__device__ __forceinline__ void put_operand_v(Top* hi, float* lo, int64_t i, const T (&x)[V]) {
  if constexpr (std::is_same<Top, float>::value && std::is_same<T, float>::value) {
    if (lo) {
      float h[V], l[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        h[v] = tf32_hi(x[v]);
        l[v] = x[v] - h[v];
      }
      stv<V>(hi + i, h);
      stv<V>(lo + i, l);
    } else {
      stv<V>(hi + i, x);
    }
  } else if constexpr (std::is_same<Top, __nv_bfloat16>::value && V == 4) {
    const __nv_bfloat162 p0 = __floats2bfloat162_rn(x[0], x[1]), p1 = __floats2bfloat162_rn(x[2], x[3]);
    uint2 u;
    u.x = *reinterpret_cast<const uint32_t*>(&p0);
    u.y = *reinterpret_cast<const uint32_t*>(&p1);
    *reinterpret_cast<uint2*>(hi + i) = u;
  } else if constexpr (std::is_same<Top, __nv_bfloat16>::value && V == 2) {
    const __nv_bfloat162 p0 = __floats2bfloat162_rn(x[0], x[1]);
    *reinterpret_cast<uint32_t*>(hi + i) = *reinterpret_cast<const uint32_t*>(&p0);
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) hi[i + v] = cvt_out<Top>(x[v]);
  }
}

// Multi-term bf16 operand of the mixed-precision chain: hi = bf16(x) at p[i]
// (and at p[i + 2d] for three terms), lo = bf16(x - hi) at p[i + d] (hi + lo
// carries about 16 significant bits).
template <int V, typename Top, typename T>
__device__ __forceinline__ void put_split_v(Top* p, int64_t i, int d, const T (&x)[V], int terms) {
  if constexpr (std::is_same<Top, __nv_bfloat16>::value && std::is_same<T, float>::value) {
    float lo[V];
    __nv_bfloat16 h[V], l[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      h[v] = __float2bfloat16_rn(x[v]);
      lo[v] = x[v] - __bfloat162float(h[v]);
      l[v] = __float2bfloat16_rn(lo[v]);
    }
    if constexpr (V == 4) {
      const __nv_bfloat162 h0 = __halves2bfloat162(h[0], h[1]), h1 = __halves2bfloat162(h[2], h[3]);
      const __nv_bfloat162 l0 = __halves2bfloat162(l[0], l[1]), l1 = __halves2bfloat162(l[2], l[3]);
      uint2 uh, ul;
      uh.x = *reinterpret_cast<const uint32_t*>(&h0);
      uh.y = *reinterpret_cast<const uint32_t*>(&h1);
      ul.x = *reinterpret_cast<const uint32_t*>(&l0);
      ul.y = *reinterpret_cast<const uint32_t*>(&l1);
      *reinterpret_cast<uint2*>(p + i) = uh;
      *reinterpret_cast<uint2*>(p + i + d) = ul;
      if (terms == 3) *reinterpret_cast<uint2*>(p + i + 2 * d) = uh;
    } else if constexpr (V == 2) {
      const __nv_bfloat162 h0 = __halves2bfloat162(h[0], h[1]), l0 = __halves2bfloat162(l[0], l[1]);
      const uint32_t uh = *reinterpret_cast<const uint32_t*>(&h0), ul = *reinterpret_cast<const uint32_t*>(&l0);
      *reinterpret_cast<uint32_t*>(p + i) = uh;
      *reinterpret_cast<uint32_t*>(p + i + d) = ul;
      if (terms == 3) *reinterpret_cast<uint32_t*>(p + i + 2 * d) = uh;
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        p[i + v] = h[v];
        p[i + d + v] = l[v];
        if (terms == 3) p[i + 2 * d + v] = h[v];
      }
    }
  }
}

// Bounds, class and split of the lane's V neurons.
template <typename T, int V>
struct SpanNeurons {
  T lo[V], hi[V], bj[V], iv[V];
  int cls[V];           // 0 inactive, 1 active, 2 unstable
  int slot[V], sign[V]; // split slot of the row's subdomain on the neuron (-1 none)
  bool unstable;        // any of the V neurons unstable
  bool split;           // any of the V neurons split
};
template <typename T, int V>
__device__ __forceinline__ void span_neurons(const SpanWarp<V>& w, const T* lo_, const T* hi_, const T* bias,
                                             const T* inv_ul, const SplitsDev& sp, int M, int layer,
                                             SpanNeurons<T, V>& n) {
#pragma unroll
  for (int v = 0; v < V; ++v) {
    n.lo[v] = n.hi[v] = n.bj[v] = n.iv[v] = T(0);
    n.slot[v] = -1;
    n.sign[v] = 0;
  }
  if (w.on) {
    ldv<V>(lo_ + w.j0, n.lo);
    ldv<V>(hi_ + w.j0, n.hi);
    ldv<V>(bias + w.j0, n.bj);
    if (inv_ul) {
      ldv<V>(inv_ul + w.j0, n.iv);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) n.iv[v] = n.hi[v] > n.lo[v] ? T(1) / (n.hi[v] - n.lo[v]) : T(0);
    }
  }
  // splits of the subdomain: lane q inspects slot q (and 32 + q) of its row
  // of the split table
  for (int b0 = 0; b0 < M; b0 += 32) {
    const int q = b0 + w.lane;
    const int code = q < M ? __ldg(sp.tab + (int64_t)w.s * M + q) : -1;
    const int lay = code >= 0 ? (code >> 24) : -1, idx = code & 0x7fffff, sg = (code >> 23) & 1 ? 1 : -1;
    unsigned m = __ballot_sync(0xffffffffu, lay == layer && idx >= w.base && idx < w.base + 32 * V);
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      const int tj = __shfl_sync(0xffffffffu, idx, b) - w.base;
      const int tsg = __shfl_sync(0xffffffffu, sg, b);
      // selects, not an indexed store: the neuron arrays stay in registers
      const int tv = tj - w.lane * V;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        n.slot[v] = tv == v ? b0 + b : n.slot[v];
        n.sign[v] = tv == v ? tsg : n.sign[v];
      }
    }
  }
  n.unstable = false;
  n.split = false;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    if (n.slot[v] >= 0) {
      n.split = true;
      if (n.sign[v] > 0) n.lo[v] = tmax(n.lo[v], T(0)); else n.hi[v] = tmin(n.hi[v], T(0));
    }
    n.cls[v] = n.hi[v] <= T(0) ? 0 : (n.lo[v] >= T(0) ? 1 : 2);
    n.unstable |= w.on && n.cls[v] == 2;
  }
}

// Cut entries of a span: contiguous in CSC order, sorted by (neuron, kind).
// A batch is 32 consecutive entries, entry b0 + lane on lane `lane`; entries
// of one (kind, neuron) form a run of lanes, and the run's first lane adds
// the run's values (in lane order) to the per-warp shared accumulator of that
// (kind, neuron). The first kSpanBatches batches stay in registers.
constexpr int kSpanBatches = 3;
template <typename T>
struct SpanEntry {
  int cut;      // cut id, -1 for no entry
  int dest;     // kind * 32V + neuron - base
  int run;      // length of the run this lane starts, 0 inside a run
  int maxrun;   // longest run of the batch (warp-uniform)
  T coef;
};
// Runs of a batch: lanes whose entries share a destination form a run of
// consecutive lanes; the first lane of each run gets its length.
template <typename T>
__device__ __forceinline__ void entry_runs(SpanEntry<T>& en, int lane) {
  const int prev = __shfl_up_sync(0xffffffffu, en.dest, 1);
  const bool cont = lane > 0 && prev == en.dest;
  const unsigned cm = __ballot_sync(0xffffffffu, cont);
  // run length: this lane plus the continuation lanes right after it
  int len = 1;
  if (lane < 31) {
    const unsigned after = cm >> (lane + 1), all = 0xffffffffu >> (lane + 1);
    len += after == all ? 31 - lane : __ffs(~after) - 1;
  }
  en.run = cont ? 0 : len;
  en.maxrun = __reduce_max_sync(0xffffffffu, en.run);
}
template <typename T, int V>
__device__ __forceinline__ void span_entry(const CutCSC<T>& c, int N, int base, int b0, int ce, int lane,
                                           SpanEntry<T>& en, DevErr& er) {
  const int e = b0 + lane;
  en.cut = -1;
  en.coef = T(0);
  en.dest = -1 - lane;   // lanes without an entry form runs of their own
  if (e < ce) {
    const int cut = __ldg(c.cut + e);
    const int kind = __ldg(c.kind + e);
    const int nl = __ldg(c.nrn + e) - base;
    if (cut < 0 || cut >= N || kind < 0 || kind > 2 || nl < 0 || nl >= 32 * V) {
      er.set(2, e, N);
    } else {
      en.cut = cut;
      en.coef = __ldg(c.coef + e);
      en.dest = kind * 32 * V + nl;
    }
  }
  entry_runs(en, lane);
}
template <typename T>
struct SpanCuts {
  int cb, ce;                       // the span's entries (warp-uniform)
  SpanEntry<T> b[kSpanBatches];
};
template <typename T, int V>
__device__ __forceinline__ void span_cuts(const CutCSC<T>& c, int N, int d, const SpanWarp<V>& w, SpanCuts<T>& sc,
                                          DevErr& er) {
  const int jb = min(w.base, d), je = min(w.base + 32 * V, d);
  sc.cb = __ldg(c.ptr + jb);
  sc.ce = __ldg(c.ptr + je);
  if (sc.cb < 0 || sc.ce < sc.cb || (int64_t)sc.ce > c.n_total) {
    er.set(1, w.c, c.n_total);
    sc.cb = sc.ce = 0;
  }
#pragma unroll
  for (int q = 0; q < kSpanBatches; ++q) span_entry<T, V>(c, N, w.base, sc.cb + 32 * q, sc.ce, w.lane, sc.b[q], er);
}

// acc[kind * 32V + neuron] += gamma-weighted entries of one batch; gv is
// gamma[row, cut] of the lane's entry.
// The first lane of a run starts from the destination's sum so far and the
// run's later lanes are added one by one, so every destination adds its
// entries in CSC order starting from 0, however they fall into batches: the
// sums do not depend on the span width or on which entries share a batch.
template <typename T>
__device__ __forceinline__ void span_batch_sum(const SpanEntry<T>& en, T gv, T* acc) {
  const bool head = en.run > 0 && en.cut >= 0;
  T v = en.cut >= 0 ? en.coef * gv : T(0);
  if (head) v = acc[en.dest] + v;
  for (int q = 1; q < en.maxrun; ++q) {
    const T u = __shfl_down_sync(0xffffffffu, v, q);
    if (q < en.run) v += u;
  }
  if (head) acc[en.dest] = v;
  __syncwarp();
}

// Per-neuron cut sums of one row: t (x entries), g (xhat), s (z) of the
// lane's V neurons. gam[32q + lane] holds gamma[row, cut] of the lane's entry
// in cached batch q (staged ahead); later batches read the row grow. acc is
// the warp's zeroed accumulator (3 * 32V), zeroed again on return.
template <typename T, int V>
__device__ __forceinline__ void span_cut_sums(const CutCSC<T>& c, const SpanCuts<T>& sc, int N,
                                              const SpanWarp<V>& w, const T* gam, const T* grow, T* acc, T (&t)[V],
                                              T (&g)[V], T (&s)[V], DevErr& er) {
#pragma unroll
  for (int v = 0; v < V; ++v) t[v] = g[v] = s[v] = T(0);
  if (sc.cb == sc.ce) return;
#pragma unroll
  for (int q = 0; q < kSpanBatches; ++q)
    if (sc.cb + 32 * q < sc.ce) span_batch_sum(sc.b[q], gam[32 * q + w.lane], acc);
  for (int b0 = sc.cb + 32 * kSpanBatches; b0 < sc.ce; b0 += 32) {
    SpanEntry<T> en;
    span_entry<T, V>(c, N, w.base, b0, sc.ce, w.lane, en, er);
    span_batch_sum(en, en.cut >= 0 ? (T)grow[en.cut] : T(0), acc);
  }
  T* a0 = acc + w.lane * V;
  ldv_rw<V>(a0, t);
  ldv_rw<V>(a0 + 32 * V, g);
  ldv_rw<V>(a0 + 64 * V, s);
  T z[V];
#pragma unroll
  for (int v = 0; v < V; ++v) z[v] = T(0);
  stv<V>(a0, z);
  stv<V>(a0 + 32 * V, z);
  stv<V>(a0 + 64 * V, z);
  __syncwarp();
}

template <typename T, int V>
__device__ __forceinline__ void span_zero(T* buf, int lane) {
  T z[V];
#pragma unroll
  for (int v = 0; v < V; ++v) z[v] = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) stv<V>(buf + k * 32 * V + lane * V, z);
  __syncwarp();
}

// The adjoint needs only the z sums s of its neurons (the x and xhat sums
// enter through nuhat, which the relaxation stored). When the span's entries
// are all cached (at most kSpanBatches batches) and at most kZBatches * 32 of
// them are z entries, those are compacted, in their CSC order, into kZBatches
// batches of their own: a row then stages and sums only them. Runs stay
// contiguous, so each (z, neuron) sum still adds its entries in CSC order.
constexpr int kZBatches = 2;
template <typename T>
struct SpanZ {
  bool ok;                  // compacted (warp-uniform); else the full sums
  int nb;                   // batches in use (warp-uniform)
  SpanEntry<T> b[kZBatches];
};
// scratch: the warp's zeroed accumulator (3 * 32V elements of T), zeroed
// again on return.
template <typename T, int V>
__device__ __forceinline__ void span_zcuts(const SpanCuts<T>& sc, const SpanWarp<V>& w, T* scratch, SpanZ<T>& z) {
  constexpr int cap = (32 * V < 32 * kZBatches) ? 32 * V : 32 * kZBatches;   // 3 arrays of cap in 3 * 32V
  int nz = 0;
  unsigned mk[kSpanBatches];
  int base[kSpanBatches];
#pragma unroll
  for (int q = 0; q < kSpanBatches; ++q) {
    const SpanEntry<T>& en = sc.b[q];
    const bool isz = sc.cb + 32 * q < sc.ce && en.cut >= 0 && en.dest >= 2 * 32 * V;
    mk[q] = __ballot_sync(0xffffffffu, isz);
    base[q] = nz;
    nz += __popc(mk[q]);
  }
  z.ok = sc.ce - sc.cb <= 32 * kSpanBatches && nz <= cap;
  z.nb = (nz + 31) / 32;
#pragma unroll
  for (int q = 0; q < kZBatches; ++q) {
    z.b[q].cut = -1;
    z.b[q].coef = T(0);
    z.b[q].dest = -1 - w.lane;
    z.b[q].run = 1;
    z.b[q].maxrun = 1;
  }
  if (!z.ok) return;
  int* zcut = reinterpret_cast<int*>(scratch);
  int* zdst = zcut + cap;
  T* zcoef = scratch + 2 * cap * sizeof(int) / sizeof(T);
#pragma unroll
  for (int q = 0; q < kSpanBatches; ++q) {
    if ((mk[q] >> w.lane) & 1u) {
      const int p = base[q] + __popc(mk[q] & ((1u << w.lane) - 1u));
      zcut[p] = sc.b[q].cut;
      zdst[p] = sc.b[q].dest;
      zcoef[p] = sc.b[q].coef;
    }
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < kZBatches; ++q) {
    const int p = 32 * q + w.lane;
    if (p < nz) {
      z.b[q].cut = zcut[p];
      z.b[q].dest = zdst[p];
      z.b[q].coef = zcoef[p];
    }
    entry_runs(z.b[q], w.lane);
  }
  __syncwarp();
  span_zero<T, V>(scratch, w.lane);
}

// s of the lane's V neurons from the compacted z entries; gam[32q + lane]
// holds gamma[row, cut] of the lane's entry in z batch q.
template <typename T, int V>
__device__ __forceinline__ void span_z_sums(const SpanZ<T>& z, const SpanWarp<V>& w, const T* gam, T* acc,
                                            T (&s)[V]) {
#pragma unroll
  for (int v = 0; v < V; ++v) s[v] = T(0);
  if (z.nb == 0) return;
#pragma unroll
  for (int q = 0; q < kZBatches; ++q)
    if (q < z.nb) span_batch_sum(z.b[q], gam[32 * q + w.lane], acc);
  T* a2 = acc + 64 * V + w.lane * V;
  ldv_rw<V>(a2, s);
  T zr[V];
#pragma unroll
  for (int v = 0; v < V; ++v) zr[v] = T(0);
  stv<V>(a2, zr);
  __syncwarp();
}

// E[r, e] = coef_e * value of the entry's (kind, neuron): x -> vx, xhat -> vh,
// z -> vz, e the entry's CSC position (a span's entries are contiguous, so a
// batch is one coalesced store). ev is the warp's staging buffer (3 * 32V).
template <typename T, int V>
__device__ __forceinline__ void span_cut_writes(const CutCSC<T>& c, const SpanCuts<T>& sc, int N,
                                                const SpanWarp<V>& w, const T (&vx)[V], const T (&vh)[V],
                                                const T (&vz)[V], T* ev, T* Erow, DevErr& er) {
  if (sc.cb == sc.ce) return;
  T* a0 = ev + w.lane * V;
  stv<V>(a0, vx);
  stv<V>(a0 + 32 * V, vh);
  stv<V>(a0 + 64 * V, vz);
  __syncwarp();
#pragma unroll
  for (int q = 0; q < kSpanBatches; ++q) {
    const SpanEntry<T>& en = sc.b[q];
    if (en.cut >= 0) Erow[sc.cb + 32 * q + w.lane] = en.coef * ev[en.dest];
  }
  for (int b0 = sc.cb + 32 * kSpanBatches; b0 < sc.ce; b0 += 32) {
    SpanEntry<T> en;
    span_entry<T, V>(c, N, w.base, b0, sc.ce, w.lane, en, er);
    if (en.cut >= 0) Erow[b0 + w.lane] = en.coef * ev[en.dest];
  }
  __syncwarp();
}


// Objective partial of the row: the span covers the 32-neuron partial slots
// V*c .. V*c + V - 1 of its layer; the first gets the sum, the others 0.
template <typename T, int V>
__device__ __forceinline__ void span_partial(T* obj_part, int64_t R, int64_t r, int c, int d, int lane, T term) {
  term = warp_sum(term);
  const int slot = c * V + lane;
  if (lane < V && slot < (d + 31) / 32) obj_part[(int64_t)slot * R + r] = lane == 0 ? term : T(0);
}

// ------------------------------------------------------------------ staging
// The per-neuron kernels stream their rows through a kStages-deep pipeline of
// asynchronous copies (cp.async) into the warp's shared memory: the dense
// per-row operands of the lane's V neurons and the row's scattered values
// (gamma of the cached cut batches, beta of the split slots). Each lane copies
// and later reads only its own slots, so a lane waits only for its own copies.
constexpr int kStages = 3;

template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool pred) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = pred ? BYTES : 0;   // 0: no read, the slot is zero-filled
  if constexpr (BYTES == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(BYTES), "r"(n)
                 : "memory");
  }
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Shared-memory layout of one warp (in elements of T): fixed buffers, then
// NS stages of ND dense rows of 32V, kSpanBatches x 32 gamma values and
// NB x 32 beta values.
template <int V, int ND, int NB, int NFIX, int NS = kStages>
struct StageLayout {
  static constexpr int SPAN = 32 * V;
  static constexpr int STAGE = ND * SPAN + kSpanBatches * 32 + NB * 32;
  static constexpr int WARP = NFIX * SPAN + NS * STAGE;
};

// ------------------------------------------------------------------ eval
// PI: the unstable neurons' pi is theta * [nuhat]_+ with theta a dual of its
// own (App. A's closing remark), read from a.theta, or written there from
// Lemma A.1's closed form when a.theta_init is set.
template <typename T, typename Top, int V, bool PI>
__global__ void __launch_bounds__(kSpanWarps * 32, kEvalMinBlocks) k_relax_eval(RelaxArgs<T, Top> a) {
  using Lay = StageLayout<V, 2, V, 3>;   // dense: y, alpha; fixed: acc
  constexpr int SPAN = Lay::SPAN, NS = kStages;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* wb = reinterpret_cast<T*>(smem_raw) + (threadIdx.x >> 5) * Lay::WARP;
  T* acc = wb;
  griddep_launch();
  SpanWarp<V> w;
  if (!span_warp<V>((int)(a.R / a.K), a.d, w)) return;
  const int KR = (a.K + (int)gridDim.z - 1) / (int)gridDim.z;   // rows of this warp: [kb, ke)
  const int kb = (int)blockIdx.z * KR, ke = min(a.K, kb + KR);
  const T* dummy = a.y;
  auto stage = [&](int st) { return wb + 3 * SPAN + st * Lay::STAGE; };
  auto dense = [&](int k, int st) {
    T* sb = stage(st) + w.lane * V;
    const bool ok = k < ke && w.on;
    const int64_t r = (int64_t)w.s * a.K + k;
    cp_async<V * sizeof(T)>(sb, ok ? a.y + (a.y_per_spec ? (int64_t)k : r) * a.d + w.j0 : dummy, ok);
    cp_async<V * sizeof(T)>(sb + SPAN, ok ? a.alpha + r * a.d + w.j0 : dummy, ok);
  };
  SpanNeurons<T, V> n;
  DevErr er;
  SpanCuts<T> sc;
  bool wsplit = false;   // some lane of the warp has a split neuron (warp-uniform)
  auto scattered = [&](int k, int st) {
    T* sb = stage(st) + 2 * SPAN;
    const int64_t r = (int64_t)w.s * a.K + k;
#pragma unroll
    for (int q = 0; q < kSpanBatches; ++q) {
      const bool ok = k < ke && sc.b[q].cut >= 0 && sc.cb + 32 * q < sc.ce;
      cp_async<sizeof(T)>(sb + 32 * q + w.lane, ok ? a.gamma + r * a.N + sc.b[q].cut : dummy, ok);
    }
    if (wsplit) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const bool ok = k < ke && w.on && n.slot[v] >= 0;
        cp_async<sizeof(T)>(sb + kSpanBatches * 32 + 32 * v + w.lane, ok ? a.beta + r * a.M + n.slot[v] : dummy,
                            ok);
      }
    }
  };
  span_zero<T, V>(acc, w.lane);
  span_neurons<T, V>(w, a.lo, a.hi, a.bias, a.inv_ul, a.sp, a.M, a.layer, n);
  wsplit = __any_sync(0xffffffffu, w.on && n.split);
  span_cuts<T, V>(a.csc, a.N, a.d, w, sc, er);
  const bool obj = a.obj_part != nullptr;   // ascent steps leave the objective out
  // everything above reads static data only; the rows come from earlier kernels
  griddep_wait();
#pragma unroll
  for (int st = 0; st < NS; ++st) {
    dense(kb + st, st);
    scattered(kb + st, st);
  }
  cp_commit();
  // rows in groups of NS: the stage of each row is a compile-time index
  for (int k0 = kb; k0 < ke; k0 += NS) {
#pragma unroll
    for (int st = 0; st < NS; ++st) {
      const int k = k0 + st;
      if (k >= ke) break;
      // the prologue is one group (rows kb .. kb+NS-1); row k >= kb+NS is the
      // group committed NS-1 groups ago
      if (k == kb) cp_wait<0>();
      else cp_wait<NS - 1>();
      const T* sb = stage(st);
      const int64_t r = (int64_t)w.s * a.K + k;
      const int64_t ij = r * a.d + w.j0;
      T t[V], gg[V], sq[V];
      span_cut_sums<T, V>(a.csc, sc, a.N, w, sb + 2 * SPAN, a.gamma + r * a.N, acc, t, gg, sq, er);
      T term = T(0);
      if (w.on) {
        T yv[V], al[V], nu[V], nh[V], th[V];
        ldv_rw<V>(sb + w.lane * V, yv);
        ldv_rw<V>(sb + SPAN + w.lane * V, al);
        if constexpr (PI) {
          if (!a.theta_init) ldv_rw<V>(a.theta + ij, th);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
          if (n.slot[v] >= 0) {        // split row -x <= 0 (x >= 0) or x <= 0
            const T b = sb[2 * SPAN + kSpanBatches * 32 + 32 * v + w.lane];
            t[v] += n.sign[v] > 0 ? -b : b;
          }
          nh[v] = yv[v] - gg[v];
          // unstable: Lemma A.1 with q = -s
          const T C = tmax(nh[v], T(0));
          T pi = tmin(tmax((n.hi[v] * C - sq[v]) * n.iv[v], T(0)), C);
          if constexpr (PI) {
            if (a.theta_init) th[v] = C > T(0) ? tmin(pi / C, T(1)) : n.hi[v] * n.iv[v];
            else pi = tmin(tmax(th[v], T(0)), T(1)) * C;
          }
          const T hu = n.lo[v] * pi - tmax(T(0), n.hi[v] * (C - pi) + n.lo[v] * pi - sq[v]);
          const T nuu = pi - al[v] * tmax(-nh[v], T(0)) - t[v];
          const int cl = n.cls[v];
          nu[v] = cl == 2 ? nuu : (cl == 1 ? nh[v] - t[v] : -t[v]);   // active: xhat = x, z = 1
          if (obj) term += (cl == 2 ? hu : (cl == 1 ? sq[v] : T(0))) - nu[v] * n.bj[v];
        }
        if (a.nu_out) put_operand_v<V, Top>(a.nu_out, a.nu_lo, ij, nu);
        if (a.nu_split) put_split_v<V, Top>(a.nu_split, r * a.split_terms * a.d + w.j0, a.d, nu, a.split_terms);
        if (a.nu_full) stv<V>(a.nu_full + ij, nu);
        stv<V>(a.nuhat_out + ij, nh);
        if constexpr (PI) {
          if (a.theta_init) stv<V>(a.theta + ij, th);
        }
      }
      if (obj) span_partial<T, V>(a.obj_part, a.R, r, w.c, a.d, w.lane, term);
      dense(k + NS, st);
      scattered(k + NS, st);
      cp_commit();
    }
  }
  cp_wait<0>();
  er.flush();
}

// ------------------------------------------------------------------ adjoint
// Writes dg/dbeta of every split slot whose neuron is in this layer into
// g_beta (the gradient output, or the input of the beta step in the gather).
template <typename T, typename Top, int V, bool PI>
__global__ void __launch_bounds__(kSpanWarps * 32) k_relax_adj(AdjArgs<T, Top> a) {
  using Lay = StageLayout<V, 5, 0, 6>;   // dense: nubar, nuhat, alpha, m, v; fixed: acc, ev
  constexpr int SPAN = Lay::SPAN, NS = kStages;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* wb = reinterpret_cast<T*>(smem_raw) + (threadIdx.x >> 5) * Lay::WARP;
  T* acc = wb;
  T* ev = wb + 3 * SPAN;
  griddep_launch();
  SpanWarp<V> w;
  if (!span_warp<V>((int)(a.R / a.K), a.d, w)) return;
  const int KR = (a.K + (int)gridDim.z - 1) / (int)gridDim.z;   // rows of this warp: [kb, ke)
  const int kb = (int)blockIdx.z * KR, ke = min(a.K, kb + KR);
  const int mode = a.st.mode;
  const T* dummy = a.nubar;
  auto stage = [&](int st) { return wb + 6 * SPAN + st * Lay::STAGE; };
  auto dense = [&](int k, int st) {
    T* sb = stage(st) + w.lane * V;
    const bool ok = k < ke && w.on;
    const bool okm = ok && mode == 2;
    const int64_t ij = ((int64_t)w.s * a.K + k) * a.d + w.j0;
    cp_async<V * sizeof(T)>(sb, ok ? a.nubar + ij : dummy, ok);
    cp_async<V * sizeof(T)>(sb + SPAN, ok ? a.nuhat + ij : dummy, ok);
    cp_async<V * sizeof(T)>(sb + 2 * SPAN, ok ? a.alpha + ij : dummy, ok);
    cp_async<V * sizeof(T)>(sb + 3 * SPAN, okm ? a.m_alpha + ij : dummy, okm);
    cp_async<V * sizeof(T)>(sb + 4 * SPAN, okm ? a.v_alpha + ij : dummy, okm);
  };
  SpanNeurons<T, V> n;
  DevErr er;
  SpanCuts<T> sc;
  SpanZ<T> zc;
  auto scattered = [&](int k, int st) {
    T* sb = stage(st) + 5 * SPAN;
    const int64_t r = (int64_t)w.s * a.K + k;
    if (zc.ok) {
#pragma unroll
      for (int q = 0; q < kZBatches; ++q) {
        if (q >= zc.nb) break;
        const bool ok = k < ke && zc.b[q].cut >= 0;
        cp_async<sizeof(T)>(sb + 32 * q + w.lane, ok ? a.gamma + r * a.N + zc.b[q].cut : dummy, ok);
      }
      return;
    }
#pragma unroll
    for (int q = 0; q < kSpanBatches; ++q) {
      const bool ok = k < ke && sc.b[q].cut >= 0 && sc.cb + 32 * q < sc.ce;
      cp_async<sizeof(T)>(sb + 32 * q + w.lane, ok ? a.gamma + r * a.N + sc.b[q].cut : dummy, ok);
    }
  };
  span_zero<T, V>(acc, w.lane);
  span_neurons<T, V>(w, a.lo, a.hi, a.bias, a.inv_ul, a.sp, a.M, a.layer, n);
  span_cuts<T, V>(a.csc, a.N, a.d, w, sc, er);
  span_zcuts<T, V>(sc, w, acc, zc);
  // everything above reads static data only; the rows come from earlier kernels
  griddep_wait();
#pragma unroll
  for (int st = 0; st < NS; ++st) {
    dense(kb + st, st);
    scattered(kb + st, st);
  }
  cp_commit();
  // rows in groups of NS: the stage of each row is a compile-time index
  for (int k0 = kb; k0 < ke; k0 += NS) {
#pragma unroll
    for (int st = 0; st < NS; ++st) {
      const int k = k0 + st;
      if (k >= ke) break;
      // the prologue is one group (rows kb .. kb+NS-1); row k >= kb+NS is the
      // group committed NS-1 groups ago
      if (k == kb) cp_wait<0>();
      else cp_wait<NS - 1>();
      const T* sb = stage(st);
      const int64_t r = (int64_t)w.s * a.K + k;
      const int64_t ij = r * a.d + w.j0;
      const T wr = a.seed ? __ldg(a.seed + r) : T(1);
      T sq[V];
      if (zc.ok) {
        span_z_sums<T, V>(zc, w, sb + 5 * SPAN, acc, sq);
      } else {
        T t[V], gg[V];
        span_cut_sums<T, V>(a.csc, sc, a.N, w, sb + 5 * SPAN, a.gamma + r * a.N, acc, t, gg, sq, er);
      }
      T nbv[V], nh[V], al[V], ma[V], va[V];
      ldv_rw<V>(sb + w.lane * V, nbv);
      ldv_rw<V>(sb + SPAN + w.lane * V, nh);
      ldv_rw<V>(sb + 2 * SPAN + w.lane * V, al);
      ldv_rw<V>(sb + 3 * SPAN + w.lane * V, ma);
      ldv_rw<V>(sb + 4 * SPAN + w.lane * V, va);
      T dt[V], dnh[V], dnhn[V], ds[V], ga[V];
      T th[V], gt[V], mt[V], vt[V];     // pi = theta * [nuhat]_+ (PI)
#pragma unroll
      for (int v = 0; v < V; ++v) th[v] = gt[v] = mt[v] = vt[v] = T(0);
      if constexpr (PI) {
        if (w.on) {
          ldv_rw<V>(a.theta + ij, th);
          if (mode == 2) {
            ldv_rw<V>(a.m_theta + ij, mt);
            ldv_rw<V>(a.v_theta + ij, vt);
          }
        }
      }
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const T nb = nbv[v] - wr * n.bj[v];   // dg/dnu^(i)
        const T h = nh[v], hi = n.hi[v], lo = n.lo[v], iv = n.iv[v];
        // local derivatives of nu and of the objective term h by case
        const bool act1 = n.cls[v] == 1;           // active: nu = nuhat - t, h = s
        T dnu_dnh = act1 ? T(1) : T(0), dh_dnh = T(0), dnu_ds = T(0), dh_ds = act1 ? wr : T(0);
        if (PI && n.cls[v] == 2) {
          // pi = th C, q = u (C - pi) + l pi - s, h = l pi - max(q, 0), nu = pi - tau - t
          const T tc = tmin(tmax(th[v], T(0)), T(1));
          const bool pos = h > T(0);
          const T C = pos ? h : T(0);
          const bool act = hi * (C - tc * C) + lo * tc * C - sq[v] > T(0);
          dnu_dnh = pos ? tc : (h < T(0) ? al[v] : T(0));
          dh_dnh = pos ? wr * (lo * tc - (act ? hi * (T(1) - tc) + lo * tc : T(0))) : T(0);
          dh_ds = act ? wr : T(0);
          gt[v] = C * (nb + wr * (lo + (act ? hi - lo : T(0))));
        }
        if constexpr (!PI) {
          // unstable: the closed-form pi of Lemma A.1, computed for every
          // neuron and selected by class (no divergent branches)
          const T p0 = (hi * h - sq[v]) * iv;
          const bool pos = h > T(0);
          const bool mid = pos && p0 > T(0) && p0 < h;          // pi* = p0
          const bool top = pos && !(p0 < h);                    // pi* = C; h = s when l C - s > 0
          const bool un = n.cls[v] == 2;
          const T hiv = hi * iv;
          dnu_dnh = un ? (mid ? hiv : (top ? T(1) : (h < T(0) ? al[v] : T(0)))) : dnu_dnh;
          dh_dnh = un && mid ? wr * lo * hiv : dh_dnh;
          dnu_ds = un && mid ? -iv : dnu_ds;
          const T zs = top ? (lo * h - sq[v] > T(0) ? wr : T(0)) : (pos ? T(0) : (sq[v] < T(0) ? wr : T(0)));
          dh_ds = un ? (mid ? -wr * lo * iv : zs) : dh_ds;
        }
        ga[v] = n.cls[v] == 2 ? nb * (-tmax(-h, T(0))) : T(0);
        dnh[v] = nb * dnu_dnh + dh_dnh;
        dnhn[v] = -dnh[v];
        ds[v] = nb * dnu_ds + dh_ds;
        dt[v] = -nb;
      }
      if (w.on) {
        if (mode == 0) {
          stv<V>(a.g_alpha + ij, ga);
        } else if (n.unstable) {
#pragma unroll
          for (int v = 0; v < V; ++v) {
            // every neuron's step, kept for the unstable ones (no divergence)
            T mv = ma[v], vv = va[v];
            const T na = step_apply(a.st, al[v], ga[v], a.st.lr_a, mv, vv);
            const bool un = n.cls[v] == 2;
            al[v] = un ? tmin(tmax(na, T(0)), T(1)) : al[v];
            ma[v] = un ? mv : ma[v];
            va[v] = un ? vv : va[v];
          }
          stv<V>(a.alpha + ij, al);
          if (mode == 2) {
            stv<V>(a.m_alpha + ij, ma);
            stv<V>(a.v_alpha + ij, va);
          }
        }
        if constexpr (PI) {
          if (mode == 0) {
            if (a.g_theta) stv<V>(a.g_theta + ij, gt);
          } else if (n.unstable) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
              if (n.cls[v] == 2) {
                const T nt = step_apply(a.st, th[v], gt[v], a.st.lr_a, mt[v], vt[v]);
                th[v] = tmin(tmax(nt, T(0)), T(1));
              }
            }
            stv<V>(a.theta + ij, th);
            if (mode == 2) {
              stv<V>(a.m_theta + ij, mt);
              stv<V>(a.v_theta + ij, vt);
            }
          }
        }
        if (a.a_out) put_operand_v<V, Top>(a.a_out, a.a_lo, ij, dnh);
        if (n.split) {
#pragma unroll
          for (int v = 0; v < V; ++v)
            if (n.slot[v] >= 0) a.g_beta[r * a.M + n.slot[v]] = (n.sign[v] > 0 ? T(-1) : T(1)) * dt[v];
        }
      }
      if (a.E) span_cut_writes<T, V>(a.csc, sc, a.N, w, dt, dnhn, ds, ev, a.E + r * a.csc.n_total, er);
      dense(k + NS, st);
      scattered(k + NS, st);
      cp_commit();
    }
  }
  cp_wait<0>();
  er.flush();
}

// ------------------------------------------------------------------ concretization
template <typename T, typename Top, int V>
__global__ void __launch_bounds__(kSpanWarps * 32) k_concretize(ConcArgs<T, Top> a) {
  using Lay = StageLayout<V, 1, 0, 6>;   // dense: y0; fixed: acc, ev
  constexpr int SPAN = Lay::SPAN, NS = kStages;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* wb = reinterpret_cast<T*>(smem_raw) + (threadIdx.x >> 5) * Lay::WARP;
  T* acc = wb;
  T* ev = wb + 3 * SPAN;
  griddep_launch();
  SpanWarp<V> w;
  if (!span_warp<V>((int)(a.R / a.K), a.d0, w)) return;
  const int KR = (a.K + (int)gridDim.z - 1) / (int)gridDim.z;   // rows of this warp: [kb, ke)
  const int kb = (int)blockIdx.z * KR, ke = min(a.K, kb + KR);
  const T* dummy = a.y0;
  auto stage = [&](int st) { return wb + 6 * SPAN + st * Lay::STAGE; };
  auto dense = [&](int k, int st) {
    const bool ok = k < ke && w.on;
    const int64_t ij = ((int64_t)w.s * a.K + k) * a.d0 + w.j0;
    cp_async<V * sizeof(T)>(stage(st) + w.lane * V, ok ? a.y0 + ij : dummy, ok);
  };
  DevErr er;
  SpanCuts<T> sc;
  auto scattered = [&](int k, int st) {
    T* sb = stage(st) + SPAN;
    const int64_t r = (int64_t)w.s * a.K + k;
#pragma unroll
    for (int q = 0; q < kSpanBatches; ++q) {
      const bool ok = k < ke && sc.b[q].cut >= 0 && sc.cb + 32 * q < sc.ce;
      cp_async<sizeof(T)>(sb + 32 * q + w.lane, ok ? a.gamma + r * a.N + sc.b[q].cut : dummy, ok);
    }
  };
  span_zero<T, V>(acc, w.lane);
  T xl[V], xh[V];
#pragma unroll
  for (int v = 0; v < V; ++v) xl[v] = xh[v] = T(0);
  if (w.on) {
    ldv<V>(a.x_lo + w.j0, xl);
    ldv<V>(a.x_hi + w.j0, xh);
  }
  span_cuts<T, V>(a.csc, a.N, a.d0, w, sc, er);
  // everything above reads static data only; the rows come from earlier kernels
  griddep_wait();
#pragma unroll
  for (int st = 0; st < NS; ++st) {
    dense(kb + st, st);
    scattered(kb + st, st);
  }
  cp_commit();
  // rows in groups of NS: the stage of each row is a compile-time index
  for (int k0 = kb; k0 < ke; k0 += NS) {
#pragma unroll
    for (int st = 0; st < NS; ++st) {
      const int k = k0 + st;
      if (k >= ke) break;
      // the prologue is one group (rows kb .. kb+NS-1); row k >= kb+NS is the
      // group committed NS-1 groups ago
      if (k == kb) cp_wait<0>();
      else cp_wait<NS - 1>();
      const T* sb = stage(st);
      const int64_t r = (int64_t)w.s * a.K + k;
      const int64_t ij = r * a.d0 + w.j0;
      const T wr = a.seed ? __ldg(a.seed + r) : T(1);
      T h0[V], ug[V], us[V];
      span_cut_sums<T, V>(a.csc, sc, a.N, w, sb + SPAN, a.gamma + r * a.N, acc, h0, ug, us, er);   // layer 0: kind x
      T yv[V];
      ldv_rw<V>(sb + w.lane * V, yv);
      T term = T(0), xs[V], a0[V], zero[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const T c0 = -yv[v] + h0[v];
        const T x = c0 > T(0) ? xl[v] : (c0 < T(0) ? xh[v] : T(0.5) * (xl[v] + xh[v]));
        xs[v] = wr * x;
        a0[v] = -wr * x;
        zero[v] = T(0);
        if (w.on) term += tmin(c0 * xl[v], c0 * xh[v]);
      }
      if (a.E) span_cut_writes<T, V>(a.csc, sc, a.N, w, xs, zero, zero, ev, a.E + r * a.csc.n_total, er);
      if (w.on && a.a0_out) put_operand_v<V, Top>(a.a0_out, a.a0_lo, ij, a0);
      if (a.obj_part) span_partial<T, V>(a.obj_part, a.R, r, w.c, a.d0, w.lane, term);
      dense(k + NS, st);
      scattered(k + NS, st);
      cp_commit();
    }
  }
  cp_wait<0>();
  er.flush();
}

// dynamic shared memory of one block of the span kernels
template <typename T, int V, int ND, int NB, int NFIX, int NS = kStages>
constexpr size_t span_smem() {
  return (size_t)kSpanWarps * StageLayout<V, ND, NB, NFIX, NS>::WARP * sizeof(T);
}

// g[r] = c_k^T b^(L) - gamma_r^T d + sum of the partials. A warp takes 32
// consecutive rows: lane i sums the partials of row r0 + i in slot order
// (reads coalesced over rows), and the warp forms each row's gamma_r^T d.
template <typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_finalize(FinalArgs<T> a) {
  const int64_t r0 = ((int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)) * 32;
  if (r0 >= a.R) return;
  const int lane = threadIdx.x & 31;
  const int nr = (int)(a.R - r0 < 32 ? a.R - r0 : 32);
  T gd = T(0);
  if (a.N > 0) {
    for (int i = 0; i < nr; ++i) {
      T p = T(0);
      for (int n = lane; n < a.N; n += 32) p += a.gamma[(r0 + i) * a.N + n] * a.d[n];
      p = warp_sum(p);
      if (lane == i) gd = p;
    }
  }
  if (lane >= nr) return;
  const int64_t r = r0 + lane;
  T g = T(0);
  for (int q = 0; q < a.P; ++q) g += a.obj_part[(int64_t)q * a.R + r];
  a.g[r] = g - gd + a.cb[(int)(r % a.K)];
}

// dg/dgamma_k = -d_k + sum of the cut's entry values (violation of cut k at the
// primal point implied by the duals), then the projected step on gamma. One
// thread per (row, cut); the cut's entry positions in the row of E, then
// their values, are read kGatherUnroll at a time.
constexpr int kGatherUnroll = 8;
template <typename T>
__global__ void k_gather(GatherArgs<T> a) {
  griddep_launch();
  griddep_wait();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.R * a.N) {
    // threads past the cuts: the projected step on beta from dg/dbeta
    // written by the adjoint (slots holding a split only). The launch covers
    // these threads only when it steps (modes 1 and 2); in mode 0 they are
    // the tail of the last block and must leave beta alone.
    if (a.st.mode == 0) return;
    i -= a.R * a.N;
    if (i >= a.R * a.M) return;
    const int64_t r = i / a.M;
    const int q = (int)(i - r * a.M);
    if (__ldg(a.sp_tab + (r / a.K) * a.M + q) < 0) return;
    T m = T(0), v = T(0);
    if (a.st.mode == 2) { m = a.m_beta[i]; v = a.v_beta[i]; }
    const T x = step_apply(a.st, a.beta[i], a.g_beta[i], a.st.lr_b, m, v);
    a.beta[i] = tmax(x, T(0));
    if (a.st.mode == 2) { a.m_beta[i] = m; a.v_beta[i] = v; }
    return;
  }
  const int64_t r = i / a.N;
  const int n = (int)(i - r * a.N);
  if (a.cut_lo) {
    // a cut of another query batched alongside: its multiplier stays 0
    const int64_t s = r / a.K;
    if (n < a.cut_lo[s] || n >= a.cut_hi[s]) {
      if (a.st.mode == 0) a.g_gamma[i] = T(0);
      return;
    }
  }
  T x = T(0), m = T(0), v = T(0);
  if (a.st.mode != 0) x = a.gamma[i];
  if (a.st.mode == 2) { m = a.m_gamma[i]; v = a.v_gamma[i]; }
  const T w = a.seed ? a.seed[r] : T(1);
  int e0 = __ldg(a.cut_ptr + n), e1 = __ldg(a.cut_ptr + n + 1);
  if (e0 < 0 || e1 < e0 || (int64_t)e1 > a.nnz) { dev_error(5, n, a.nnz); e0 = e1 = 0; }
  const T* Er = a.E + r * a.nnz;
  T grad = -w * __ldg(a.d + n);
  for (int e = e0; e < e1; e += kGatherUnroll) {
    int q_[kGatherUnroll];
#pragma unroll
    for (int q = 0; q < kGatherUnroll; ++q) {
      q_[q] = e + q < e1 ? __ldg(a.pos + e + q) : -1;
      if (q_[q] >= 0 && (int64_t)q_[q] >= a.nnz) { dev_error(5, e + q, a.nnz); q_[q] = -1; }
    }
    T ev[kGatherUnroll];
#pragma unroll
    for (int q = 0; q < kGatherUnroll; ++q) ev[q] = q_[q] >= 0 ? Er[q_[q]] : T(0);
#pragma unroll
    for (int q = 0; q < kGatherUnroll; ++q) grad += ev[q];
  }
  if (a.st.mode == 0) {
    a.g_gamma[i] = grad;
  } else {
    x = step_apply(a.st, x, grad, a.st.lr_g, m, v);
    a.gamma[i] = tmax(x, T(0));
    if (a.st.mode == 2) { a.m_gamma[i] = m; a.v_gamma[i] = v; }
  }
}

// ------------------------------------------------------------------ certification
// Lower bound of k*x over k in [klo,khi], x in [xlo,xhi] (corners, rounded down).
__device__ __forceinline__ double box_min_rd(double klo, double khi, double xlo, double xhi) {
  return fmin(fmin(__dmul_rd(klo, xlo), __dmul_rd(klo, xhi)), fmin(__dmul_rd(khi, xlo), __dmul_rd(khi, xhi)));
}

// Higham's gamma_n = n u / (1 - n u), u = 2^-53, rounded up.
__device__ __forceinline__ double gamma_of(int n) {
  const double nu = __dmul_ru((double)n, 1.1102230246251565e-16);
  return __ddiv_ru(nu, __dsub_rd(1.0, nu));
}

template <typename Td>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_certify_relax(CertArgs<Td> a) {
  ChunkWarp w;
  if (!chunk_warp((int)(a.R / a.K), a.d, w)) return;
  const int j = w.j;
  int sign = 0;
  const int slot = lane_split(a.sp, w.s, a.M, a.layer, w.c, w.lane, sign);
  ChunkCuts<double> cc;
  chunk_cuts(a.csc, a.N, a.d, w.c, w.lane, cc);
  __shared__ __align__(16) unsigned char cacc_all[kWarpsPerBlock * kCertAcc];
  unsigned char* cacc = cacc_all + (threadIdx.x >> 5) * kCertAcc;
  cert_acc_zero(cacc, w.lane);
  // row-independent: the neuron's bounds after its split, 1/(u - l) (pi only
  // has to lie in [0, C] for the certificate to hold), and Higham's factors
  // for the sparse sums (the entry counts per kind do not depend on the row)
  double lo0 = 0.0, hi0 = 0.0;
  if (w.on) {
    lo0 = a.lo[j];
    hi0 = a.hi[j];
    if (slot >= 0) {
      if (sign > 0) lo0 = fmax(lo0, 0.0); else hi0 = fmin(hi0, 0.0);
    }
  }
  const double inv_ul = hi0 > lo0 ? 1.0 / (hi0 - lo0) : 0.0;
  // whether the warp's neurons fall in more than one class (inactive,
  // active, unstable): row-independent, warp-uniform
  const unsigned cls_bits = w.on ? (hi0 <= 0.0 ? 1u : (lo0 >= 0.0 ? 2u : 4u)) : 0u;
  const unsigned present = __reduce_or_sync(0xffffffffu, cls_bits);
  const bool mixed = (present & (present - 1u)) != 0u;
  double gt = 0.0, gg_n = 0.0, gs_n = 0.0;
  for (int k = 0; k < a.K; ++k) {
    const int64_t r = (int64_t)w.s * a.K + k;
    double sum[3], abs_[3];
    int cnt_[3];
    cut_sums_row_cert(a.csc, cc, a.gamma + r * a.N, a.N, w.lane, sum, abs_, cnt_, cacc);
    double part = 0.0;
    if (w.on) {
    // sparse sums in round-to-nearest with their Higham error bounds
    double t = sum[GCP_VAR_X], gg = sum[GCP_VAR_XHAT], sq = sum[GCP_VAR_Z];
    double ta = abs_[GCP_VAR_X];
    const double lo = lo0, hi = hi0;
    if (slot >= 0) {
      const double bv = (double)a.beta[r * a.M + slot];
      if (sign > 0) t -= bv; else t += bv;
      ta = __dadd_ru(ta, fabs(bv));
    }
    if (k == 0) {
      gt = gamma_of(cnt_[GCP_VAR_X] + (slot >= 0 ? 1 : 0));
      gg_n = gamma_of(cnt_[GCP_VAR_XHAT]);
      gs_n = gamma_of(cnt_[GCP_VAR_Z]);
    }
    const double et = __dmul_ru(gt, ta);
    const double eg = __dmul_ru(gg_n, abs_[GCP_VAR_XHAT]);
    const double es = __dmul_ru(gs_n, abs_[GCP_VAR_Z]);
    const int64_t yi = (a.y_per_spec ? (int64_t)k : r) * a.d + j;
    const double y = a.y[yi];
    const double ey = __dmul_ru(a.gamma_n, (double)a.yabs[yi]);
    const double nh = y - gg;
    // enclosures of the exact t, y, g, s
    const double t_lo = __dsub_rd(t, et), t_hi = __dadd_ru(t, et);
    const double y_lo = __dsub_rd(y, ey), y_hi = __dadd_ru(y, ey);
    const double g_lo = __dsub_rd(gg, eg), g_hi = __dadd_ru(gg, eg);
    const double s_lo = __dsub_rd(sq, es);
    double nu;
    if (mixed) {
      // One formula for the three classes, the class choosing its terms by
      // selects: a warp's lanes usually mix classes, and FP64 instructions,
      // not memory, set this pass's time. Per class the result is the same
      // number as the case-by-case form: the terms a class does not have are
      // exact zeros added with directed rounding.
      //   inactive (xhat = z = 0): (nu + t) x over x in [lo, hi], nu = -t;
      //   active (xhat = x, z = 1): (nu + t - y + g) x plus s, nu = nuhat - t;
      //   unstable: explicit duals pi, gamma_r = C - pi, tau, mu = M - tau (all
      //   >= 0), nu = pi - tau - t; x: (nu + t + tau - pi) x over [lo, hi];
      //   xhat: (-y + g - mu - tau + gamma_r + pi) xhat over [0, hi];
      //   z: (-hi gamma_r - lo pi + s) z over [0, 1]; plus pi lo.
      const bool inact = hi <= 0.0, act = !inact && lo >= 0.0, unst = !inact && !act;
      const double C = fmax(nh, 0.0), Mm = fmax(-nh, 0.0);
      const double p0 = (hi * C - sq) * inv_ul;
      // Lemma A.1's pi, or theta * C for directly optimised duals; either is
      // in [0, C] (theta <= 1 and rounding is monotone), so gr >= 0
      const double pi = a.theta ? fmin(fmax((double)a.theta[r * a.d + j], 0.0), 1.0) * C : fmin(fmax(p0, 0.0), C);
      const double gr = C - pi;
      const double al = fmin(fmax((double)a.alpha[r * a.d + j], 0.0), 1.0);
      const double tau = al * Mm;
      const double mu = Mm - tau;
      nu = inact ? -t : (act ? nh : pi - tau) - t;
      // x's coefficient (nu + t) + A + B, rounded down and up
      const double A_lo = act ? -y_hi : (unst ? tau : 0.0), A_hi = act ? -y_lo : (unst ? tau : 0.0);
      const double B_lo = act ? g_lo : (unst ? -pi : 0.0), B_hi = act ? g_hi : (unst ? -pi : 0.0);
      const double k_lo = __dadd_rd(__dadd_rd(__dadd_rd(nu, t_lo), A_lo), B_lo);
      const double k_hi = __dadd_ru(__dadd_ru(__dadd_ru(nu, t_hi), A_hi), B_hi);
      double kh_lo = __dadd_rd(-y_hi, g_lo);
      kh_lo = __dadd_rd(__dsub_rd(__dsub_rd(kh_lo, mu), tau), __dadd_rd(gr, pi));
      const double kz_lo = __dadd_rd(__dadd_rd(-__dmul_ru(hi, gr), -__dmul_ru(lo, pi)), s_lo);
      part = box_min_rd(k_lo, k_hi, lo, hi);
      part = __dadd_rd(part, act ? s_lo : (unst ? fmin(0.0, __dmul_rd(kh_lo, hi)) : 0.0));
      part = __dadd_rd(part, unst ? fmin(0.0, kz_lo) : 0.0);
      part = __dadd_rd(part, unst ? __dmul_rd(pi, lo) : 0.0);
    } else {
      // every lane of the warp in one class: that class's terms only
      if (hi <= 0.0) {
        // inactive: xhat = z = 0; Lagrangian term (nu + t) x over x in [lo, hi]
        nu = -t;
        part = box_min_rd(__dadd_rd(nu, t_lo), __dadd_ru(nu, t_hi), lo, hi);
      } else if (lo >= 0.0) {
        // active: xhat = x, z = 1; term (nu + t - y + g) x plus s
        nu = nh - t;
        const double klo = __dadd_rd(__dadd_rd(__dadd_rd(nu, t_lo), -y_hi), g_lo);
        const double khi = __dadd_ru(__dadd_ru(__dadd_ru(nu, t_hi), -y_lo), g_hi);
        part = __dadd_rd(box_min_rd(klo, khi, lo, hi), s_lo);
      } else {
        // unstable: explicit duals pi, gamma_r = C - pi, tau, mu = M - tau (all >= 0)
        const double C = fmax(nh, 0.0), Mm = fmax(-nh, 0.0);
        const double p0 = (hi * C - sq) * inv_ul;
        // Lemma A.1's pi, or theta * C for directly optimised duals; either is
        // in [0, C] (theta <= 1 and rounding is monotone), so gr >= 0
        const double pi = a.theta ? fmin(fmax((double)a.theta[r * a.d + j], 0.0), 1.0) * C : fmin(fmax(p0, 0.0), C);
        const double gr = C - pi;
        const double al = fmin(fmax((double)a.alpha[r * a.d + j], 0.0), 1.0);
        const double tau = al * Mm;
        const double mu = Mm - tau;
        nu = (pi - tau) - t;
        // x: (nu + t + tau - pi) x over [lo, hi]
        const double kx_lo = __dsub_rd(__dadd_rd(__dadd_rd(nu, t_lo), tau), pi);
        const double kx_hi = __dsub_ru(__dadd_ru(__dadd_ru(nu, t_hi), tau), pi);
        // xhat: (-y + g - mu - tau + gr + pi) xhat over [0, hi]
        double kh_lo = __dadd_rd(-y_hi, g_lo);
        kh_lo = __dadd_rd(__dsub_rd(__dsub_rd(kh_lo, mu), tau), __dadd_rd(gr, pi));
        // z: (-hi gr - lo pi + s) z over [0, 1]
        const double kz_lo = __dadd_rd(__dadd_rd(-__dmul_ru(hi, gr), -__dmul_ru(lo, pi)), s_lo);
        part = box_min_rd(kx_lo, kx_hi, lo, hi);
        part = __dadd_rd(part, fmin(0.0, __dmul_rd(kh_lo, hi)));
        part = __dadd_rd(part, fmin(0.0, kz_lo));
        part = __dadd_rd(part, __dmul_rd(pi, lo));
      }
    }
    part = __dadd_rd(part, __dmul_rd(-nu, a.bias[j]));
    a.nu_out[r * a.d + j] = nu;
    if (a.nuabs_out) a.nuabs_out[r * a.d + j] = __double2float_ru(fabs(nu));
    }
    part = warp_sum_rd(part);
    if (w.lane == 0) a.obj_part[(int64_t)w.c * a.R + r] = part;
  }
}

template <typename Td>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_certify_conc(int64_t R, int K, int N, int d0,
                                                                       const double* y0, const float* y0abs,
                                                                       double gamma_n, const double* x_lo,
                                                                       const double* x_hi, const Td* gamma,
                                                                       CutCSC<double> csc, double* obj_part) {
  ChunkWarp w;
  if (!chunk_warp((int)(R / K), d0, w)) return;
  const int j = w.j;
  ChunkCuts<double> cc;
  chunk_cuts(csc, N, d0, w.c, w.lane, cc);
  __shared__ __align__(16) unsigned char cacc_all[kWarpsPerBlock * kCertAcc];
  unsigned char* cacc = cacc_all + (threadIdx.x >> 5) * kCertAcc;
  cert_acc_zero(cacc, w.lane);
  double gh = 0.0;   // Higham's factor of the input neuron's cut sum (the same for every row)
  for (int k = 0; k < K; ++k) {
    const int64_t r = (int64_t)w.s * K + k;
    double sum[3], abs_[3];
    int cnt_[3];
    cut_sums_row_cert(csc, cc, gamma + r * N, N, w.lane, sum, abs_, cnt_, cacc);
    double part = 0.0;
    if (w.on) {
      const double h = sum[GCP_VAR_X];
      if (k == 0) gh = gamma_of(cnt_[GCP_VAR_X]);
      const double eh = __dmul_ru(gh, abs_[GCP_VAR_X]);
      const double y = y0[r * d0 + j];
      const double ey = __dmul_ru(gamma_n, (double)y0abs[r * d0 + j]);
      const double c_lo = __dadd_rd(__dsub_rd(-y, ey), __dsub_rd(h, eh));
      const double c_hi = __dadd_ru(__dadd_ru(-y, ey), __dadd_ru(h, eh));
      part = box_min_rd(c_lo, c_hi, x_lo[j], x_hi[j]);
    }
    part = warp_sum_rd(part);
    if (w.lane == 0) obj_part[(int64_t)w.c * R + r] = part;
  }
}

template <typename Td>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_certify_final(int64_t R, int K, int N, int P, const double* C,
                                                                       const double* bL, int dL, const double* d,
                                                                       const Td* gamma, const double* obj_part,
                                                                       double* out) {
  const int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (r >= R) return;
  const int lane = threadIdx.x & 31;
  const int k = (int)(r % K);
  double g = 0.0;
  for (int q = lane; q < dL; q += 32) g = __dadd_rd(g, __dmul_rd(C[(int64_t)k * dL + q], bL[q]));  // -nu^(L)^T b^(L)
  for (int n = lane; n < N; n += 32) g = __dadd_rd(g, __dmul_rd(-(double)gamma[r * N + n], d[n]));
  for (int q = lane; q < P; q += 32) g = __dadd_rd(g, obj_part[(int64_t)q * R + r]);
  g = warp_sum_rd(g);
  if (lane == 0) out[r] = g;
}

// ------------------------------------------------------------------ layout helpers
template <typename Ts, typename Td>
__global__ void k_transpose_cast(int64_t rows, int64_t cols, const Ts* __restrict__ src, Td* __restrict__ dst) {
  __shared__ Ts tile[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t rr = r0 + i, cc = c0 + threadIdx.x;
    if (rr < rows && cc < cols) tile[i][threadIdx.x] = src[rr * cols + cc];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t cc = c0 + i, rr = r0 + threadIdx.x;
    if (rr < rows && cc < cols) dst[cc * rows + rr] = static_cast<Td>(tile[threadIdx.x][i]);
  }
}

template <typename Ts, typename Td>
__global__ void k_cast(int64_t n, const Ts* __restrict__ src, Td* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = static_cast<Td>(src[i]);
}

template <typename T>
__global__ void k_default_alpha(int64_t R, int K, int d, int layer, const T* lo, const T* hi, SplitsDev sp,
                                T* alpha) {
  const int64_t n = R * (int64_t)d;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / d;
    const int j = (int)(i - r * d);
    const int s = (int)(r / K);
    T l = lo[j], u = hi[j];
    int q0, q1;
    split_range(sp, s, kMaxSplits, q0, q1);
    for (int q = q0; q < q1; ++q)
      if (sp.layer[q] == layer && sp.index[q] == j) {
        if (sp.sign[q] > 0) l = tmax(l, T(0)); else u = tmin(u, T(0));
      }
    alpha[i] = (u >= -l) ? T(1) : T(0);
  }
}

// one warp per (subdomain, 32-neuron chunk)
inline dim3 chunk_blocks(int64_t R, int K, int d) {
  const int64_t S = R / K;
  return dim3((unsigned)((S + kWarpsPerBlock - 1) / kWarpsPerBlock), (unsigned)((d + 31) / 32));
}
inline unsigned row_blocks(int64_t R) { return (unsigned)((R + kWarpsPerBlock - 1) / kWarpsPerBlock); }
inline int flat_grid(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

template <typename T>
const char* tsfx() { return sizeof(T) == 8 ? "f64" : "f32"; }

// Neurons per lane of the span kernels: 4 (16-byte vectors) for float chains
// on layers whose width is a multiple of 4, unless a 128-neuron span of the
// layer has more cut entries than the kSpanBatches batches a warp keeps in
// registers (later batches reread their entries from memory every row): then
// 2 (8-byte vectors, 64-neuron spans) when the width is even; else 1. The cut
// sums add each destination's entries in CSC order whatever the span width,
// so the choice changes no dual, gradient or certified bound; only the float
// chain's own objective partials (one per span, summed over its lanes) are
// added in a tree that follows the span width.
template <typename T>
inline bool span_v4(int d) { return sizeof(T) == 4 && d % 4 == 0; }
template <typename T>
inline int span_vec(int d, int max_span4, bool al16_all, bool al8_all) {
  if (sizeof(T) != 4) return 1;
  const bool ok4 = d % 4 == 0 && al16_all, ok2 = d % 2 == 0 && al8_all;
  if (ok4 && !(ok2 && max_span4 > 32 * kSpanBatches)) return 4;
  return ok2 ? 2 : 1;
}
// A warp takes all K rows of its subdomain span, its setup (bounds, split
// hits, cut entries) shared by the rows; a launch that would then leave the
// GPU mostly idle (a small batch, where one warp's K rows in sequence are the
// kernel's latency) spreads each span's rows over gridDim.z warps instead,
// enough to bring the launch near 8 warps per SM.
inline int row_split(int64_t S, int K, int spans, int64_t target = 152 * 8) {
  const int64_t warps = S * spans;
  if (warps >= target || K <= 1) return 1;
  return (int)std::min<int64_t>(K, (target + warps - 1) / warps);
}
inline bool al16(const void* p) { return ((uintptr_t)p & 15) == 0; }
inline bool al8(const void* p) { return ((uintptr_t)p & 7) == 0; }

// Launch a span kernel with its dynamic shared memory (opted in above 48 KB).
template <typename Kern, typename Args>
void launch_span(Kern kern, size_t smem, dim3 grid, cudaStream_t st, const Args& a) {
  smem_opt_in(reinterpret_cast<const void*>(kern), smem);
  launch_pdl(kern, grid, dim3(kSpanWarps * 32), smem, st, a);
}
inline dim3 span_blocks(int64_t R, int K, int d, int V, int64_t target = 152 * 8) {
  const int64_t S = R / K;
  const int spans = (d + 32 * V - 1) / (32 * V);
  return dim3((unsigned)((S + kSpanWarps - 1) / kSpanWarps), (unsigned)spans,
              (unsigned)row_split(S, K, spans, target));
}

// host-side extent checks shared by the launchers
inline bool chk_splits(const SplitsDev& sp, int64_t R, int K, int M = 0) {
  const double S = K > 0 ? (double)(R / K) : 0.0;
  return reg_check(sp.ptr, (S + 1) * 4.0, "split ptr") & reg_check(sp.layer, sp.n * 2.0, "split layer") &
         reg_check(sp.index, sp.n * 4.0, "split index") & reg_check(sp.sign, (double)sp.n, "split sign") &
         reg_check(sp.tab, M > 0 ? S * M * 4.0 : 0.0, "split table");
}
template <typename T>
inline bool chk_csc(const CutCSC<T>& c, int d) {
  return reg_check(c.ptr, (d + 1) * 4.0, "csc ptr") & reg_check(c.cut, c.n_total * 4.0, "csc cut") &
         reg_check(c.kind, (double)c.n_total, "csc kind") & reg_check(c.coef, c.n_total * (double)sizeof(T), "csc coef") &
         reg_check(c.nrn, c.n_total * 4.0, "csc nrn");
}

template <int V, typename T, typename Top>
void launch_eval(cudaStream_t st, const RelaxArgs<T, Top>& a) {
  const dim3 g = span_blocks(a.R, a.K, a.d, V, 152 * kEvalWarpsPerSM);
  if (a.theta)
    launch_span(k_relax_eval<T, Top, V, true>, span_smem<T, V, 2, V, 3>(), g, st, a);
  else
    launch_span(k_relax_eval<T, Top, V, false>, span_smem<T, V, 2, V, 3>(), g, st, a);
}
template <int V, typename T, typename Top>
void launch_adj(cudaStream_t st, const AdjArgs<T, Top>& a) {
  const dim3 g = span_blocks(a.R, a.K, a.d, V);
  if (a.theta)
    launch_span(k_relax_adj<T, Top, V, true>, span_smem<T, V, 5, 0, 6>(), g, st, a);
  else
    launch_span(k_relax_adj<T, Top, V, false>, span_smem<T, V, 5, 0, 6>(), g, st, a);
}

// Algorithmic bytes per launch: every per-(row, neuron) array read or written
// once, one gamma read (and E write) per cut entry and row, partial sums.
template <typename T, typename Top>
void relax_eval(cudaStream_t st, const RelaxArgs<T, Top>& a) {
  if (a.R <= 0 || a.d <= 0) return;
  if (a.nu_split && a.split_terms != 2 && a.split_terms != 3)
    return (void)reg_check(nullptr, 1.0, "relax: split operand of 2 or 3 terms");
  char nm[48];
  snprintf(nm, sizeof nm, "relax_eval_%s%s", tsfx<T>(), sizeof(Top) == 2 ? "_bf16" : "");
  const double bytes = (double)a.R * a.d * (3.0 * sizeof(T) + (a.nu_out ? sizeof(Top) : 0) +
                                            (a.nu_split ? a.split_terms * sizeof(Top) : 0.0) + (a.nu_full ? sizeof(T) : 0)) +
                       (double)a.R * (a.csc.n_entries + (a.d + 31) / 32) * sizeof(T);
  const double Rd = (double)a.R * a.d, tb = sizeof(T);
  if (!(reg_check(a.y, (a.y_per_spec ? (double)a.K : (double)a.R) * a.d * tb, "relax y") &
        reg_check(a.lo, a.d * tb, "lo") & reg_check(a.hi, a.d * tb, "hi") & reg_check(a.bias, a.d * tb, "bias") &
        reg_check(a.inv_ul, a.inv_ul ? a.d * tb : 0.0, "inv_ul") &
        reg_check(a.alpha, Rd * tb, "alpha") & reg_check(a.beta, (double)a.M * a.R * tb, "beta") &
        reg_check(a.gamma, (a.csc.n_total ? (double)a.N * a.R : 0.0) * tb, "gamma") & chk_splits(a.sp, a.R, a.K, a.M) &
        chk_csc(a.csc, a.d) & reg_check(a.nu_out, a.nu_out ? Rd * sizeof(Top) : 0.0, "nu out") &
        reg_check(a.nu_split, a.nu_split ? a.split_terms * Rd * sizeof(Top) : 0.0, "nu split") &
        reg_check(a.nu_lo, a.nu_lo ? Rd * 4.0 : 0.0, "nu lo") &
        reg_check(a.nuhat_out, Rd * tb, "nuhat out") & reg_check(a.theta, a.theta ? Rd * tb : 0.0, "theta") &
        reg_check(a.nu_full, a.nu_full ? Rd * tb : 0.0, "nu full") &
        (!a.obj_part || reg_check(a.obj_part, ((a.d + 31) / 32) * (double)a.R * tb, "obj part"))))
    return;
  int tk = prof_begin(st, nm, 0.0, bytes);
  const bool a16 = al16(a.y) && al16(a.alpha) && al16(a.lo) && al16(a.hi) && al16(a.bias) && al16(a.inv_ul) &&
                   al16(a.nu_out) && al16(a.nu_lo) && al16(a.nuhat_out) && al16(a.theta) && al16(a.nu_full) &&
                   (reinterpret_cast<uintptr_t>(a.nu_split) & 7) == 0;
  const bool a8 = al8(a.y) && al8(a.alpha) && al8(a.lo) && al8(a.hi) && al8(a.bias) && al8(a.inv_ul) &&
                  al8(a.nu_out) && al8(a.nu_lo) && al8(a.nuhat_out) && al8(a.theta) && al8(a.nu_full) &&
                  (reinterpret_cast<uintptr_t>(a.nu_split) & 3) == 0;
  const int V = span_vec<T>(a.d, a.csc.max_span4, a16, a8);
  if constexpr (sizeof(T) == 4) {
    if (V == 4) launch_eval<4>(st, a);
    else if (V == 2) launch_eval<2>(st, a);
    else launch_eval<1>(st, a);
  } else {
    launch_eval<1>(st, a);
  }
  prof_end(st, tk);
}
template <typename T, typename Top>
void relax_adjoint(cudaStream_t st, const AdjArgs<T, Top>& a) {
  if (a.R <= 0 || a.d <= 0) return;
  char nm[48];
  snprintf(nm, sizeof nm, "relax_adj_%s%s", tsfx<T>(), sizeof(Top) == 2 ? "_bf16" : "");
  // per (row, neuron): nubar and nuhat read; alpha read and either its
  // gradient written (mode 0) or alpha written back (PGA) together with both
  // Adam moments read and written; a written for the next GEMM. Per cut entry
  // and row: gamma read, E written.
  const double per_elem = a.st.mode == 0 ? 4.0 : (a.st.mode == 1 ? 4.0 : 8.0);
  const double bytes = (double)a.R * a.d * (per_elem * sizeof(T) + (a.a_out ? sizeof(Top) : 0)) +
                       (double)a.R * a.csc.n_entries * 2.0 * sizeof(T);
  const double Rd = (double)a.R * a.d, tb = sizeof(T);
  const bool m0 = a.st.mode == 0, m2 = a.st.mode == 2;
  if (!(reg_check(a.nubar, Rd * tb, "nubar") & reg_check(a.seed, a.seed ? a.R * tb : 0.0, "seed") &
        reg_check(a.lo, a.d * tb, "lo") & reg_check(a.hi, a.d * tb, "hi") & reg_check(a.bias, a.d * tb, "bias") &
        reg_check(a.inv_ul, a.inv_ul ? a.d * tb : 0.0, "inv_ul") &
        reg_check(a.alpha, Rd * tb, "alpha") &
        reg_check(a.gamma, (a.csc.n_total ? (double)a.N * a.R : 0.0) * tb, "gamma") &
        reg_check(a.nuhat, Rd * tb, "nuhat") & chk_splits(a.sp, a.R, a.K, a.M) & chk_csc(a.csc, a.d) &
        reg_check(a.a_out, a.a_out ? Rd * sizeof(Top) : 0.0, "a out") &
        reg_check(a.a_lo, (a.a_out && a.a_lo) ? Rd * 4.0 : 0.0, "a lo") &
        reg_check(a.E, a.csc.n_entries ? (double)a.csc.n_total * a.R * tb : 0.0, "E") &
        reg_check(a.g_alpha, m0 ? Rd * tb : 0.0, "g_alpha") &
        reg_check(a.g_beta, a.M > 0 ? (double)a.M * a.R * tb : 0.0, "g_beta") &
        reg_check(a.m_alpha, m2 ? Rd * tb : 0.0, "m_alpha") & reg_check(a.v_alpha, m2 ? Rd * tb : 0.0, "v_alpha") &
        reg_check(a.theta, a.theta ? Rd * tb : 0.0, "theta") &
        reg_check(a.g_theta, (a.theta && m0 && a.g_theta) ? Rd * tb : 0.0, "g_theta") &
        reg_check(a.m_theta, (a.theta && m2) ? Rd * tb : 0.0, "m_theta") &
        reg_check(a.v_theta, (a.theta && m2) ? Rd * tb : 0.0, "v_theta")))
    return;
  int tk = prof_begin(st, nm, 0.0, bytes);
  const bool a16 = al16(a.nubar) && al16(a.nuhat) && al16(a.alpha) && al16(a.m_alpha) && al16(a.v_alpha) &&
                   al16(a.g_alpha) && al16(a.lo) && al16(a.hi) && al16(a.bias) && al16(a.inv_ul) && al16(a.a_out) &&
                   al16(a.a_lo) && al16(a.theta) && al16(a.g_theta) && al16(a.m_theta) && al16(a.v_theta);
  const bool a8 = al8(a.nubar) && al8(a.nuhat) && al8(a.alpha) && al8(a.m_alpha) && al8(a.v_alpha) &&
                  al8(a.g_alpha) && al8(a.lo) && al8(a.hi) && al8(a.bias) && al8(a.inv_ul) && al8(a.a_out) &&
                  al8(a.a_lo) && al8(a.theta) && al8(a.g_theta) && al8(a.m_theta) && al8(a.v_theta);
  const int V = span_vec<T>(a.d, a.csc.max_span4, a16, a8);
  if constexpr (sizeof(T) == 4) {
    if (V == 4) launch_adj<4>(st, a);
    else if (V == 2) launch_adj<2>(st, a);
    else launch_adj<1>(st, a);
  } else {
    launch_adj<1>(st, a);
  }
  prof_end(st, tk);
}
template <typename T, typename Top>
void concretize(cudaStream_t st, const ConcArgs<T, Top>& a) {
  if (a.R <= 0 || a.d0 <= 0) return;
  char nm[48];
  snprintf(nm, sizeof nm, "concretize_%s", tsfx<T>());
  const double bytes = (double)a.R * a.d0 * (sizeof(T) + (a.a0_out ? sizeof(Top) : 0)) +
                       (double)a.R * (a.csc.n_entries * (a.E ? 2.0 : 1.0) + (a.d0 + 31) / 32) * sizeof(T);
  const double Rd = (double)a.R * a.d0, tb = sizeof(T);
  if (!(reg_check(a.y0, Rd * tb, "y0") & reg_check(a.x_lo, a.d0 * tb, "x_lo") & reg_check(a.x_hi, a.d0 * tb, "x_hi") &
        reg_check(a.gamma, (a.csc.n_total ? (double)a.N * a.R : 0.0) * tb, "gamma") &
        reg_check(a.seed, a.seed ? a.R * tb : 0.0, "seed") & chk_csc(a.csc, a.d0) &
        reg_check(a.a0_out, a.a0_out ? Rd * sizeof(Top) : 0.0, "a0 out") &
        reg_check(a.a0_lo, (a.a0_out && a.a0_lo) ? Rd * 4.0 : 0.0, "a0 lo") &
        reg_check(a.E, (a.E && a.csc.n_entries) ? (double)a.csc.n_total * a.R * tb : 0.0, "E") &
        (!a.obj_part || reg_check(a.obj_part, ((a.d0 + 31) / 32) * (double)a.R * tb, "obj part"))))
    return;
  int tk = prof_begin(st, nm, 0.0, bytes);
  if constexpr (sizeof(T) == 4) {
    if (span_v4<T>(a.d0) && al16(a.y0) && al16(a.x_lo) && al16(a.x_hi) && al16(a.a0_out) && al16(a.a0_lo)) {
      launch_span(k_concretize<T, Top, 4>, span_smem<T, 4, 1, 0, 6>(), span_blocks(a.R, a.K, a.d0, 4), st, a);
      prof_end(st, tk);
      return;
    }
  }
  launch_span(k_concretize<T, Top, 1>, span_smem<T, 1, 1, 0, 6>(), span_blocks(a.R, a.K, a.d0, 1), st, a);
  prof_end(st, tk);
}
template <typename T>
void finalize_bound(cudaStream_t st, const FinalArgs<T>& a) {
  if (a.R <= 0) return;
  const double tb = sizeof(T);
  if (!(reg_check(a.cb, a.K * tb, "cb") & reg_check(a.d, a.N * tb, "d") &
        reg_check(a.gamma, (double)a.N * a.R * tb, "gamma") & reg_check(a.obj_part, (double)a.P * a.R * tb, "obj part") &
        reg_check(a.g, a.R * tb, "g")))
    return;
  int tk = prof_begin(st, sizeof(T) == 8 ? "finalize_f64" : "finalize_f32", 0.0,
                      (double)a.R * (a.N + a.P + 1) * sizeof(T));
  k_finalize<T><<<row_blocks((a.R + 31) / 32), kWarpsPerBlock * 32, 0, st>>>(a);
  prof_end(st, tk);
}
template <typename T>
void gather_gamma(cudaStream_t st, const GatherArgs<T>& a) {
  const int64_t nb = a.st.mode != 0 ? a.R * a.M : 0;   // beta steps (modes 1 and 2)
  if (a.R <= 0 || (a.N <= 0 && nb == 0)) return;
  const double tb = sizeof(T), NR = (double)a.N * a.R, MR = (double)nb;
  const bool m0 = a.st.mode == 0, m2 = a.st.mode == 2;
  if (!(reg_check(a.cut_ptr, a.N > 0 ? (a.N + 1) * 4.0 : 0.0, "cut ptr") & reg_check(a.pos, a.nnz * 4.0, "cut pos") & 
        reg_check(a.E, (double)a.nnz * a.R * tb, "E") &
        reg_check(a.d, a.N * tb, "d") & reg_check(a.seed, a.seed ? a.R * tb : 0.0, "seed") &
        reg_check(a.gamma, NR * tb, "gamma") & reg_check(a.g_gamma, m0 ? NR * tb : 0.0, "g_gamma") &
        reg_check(a.m_gamma, m2 ? NR * tb : 0.0, "m_gamma") & reg_check(a.v_gamma, m2 ? NR * tb : 0.0, "v_gamma") &
        reg_check(a.cut_lo, a.cut_lo ? (double)(a.R / a.K) * 4.0 : 0.0, "cut lo") &
        reg_check(a.cut_hi, a.cut_hi ? (double)(a.R / a.K) * 4.0 : 0.0, "cut hi") &
        reg_check(a.sp_tab, MR * 4.0 / a.K, "split table") & reg_check(a.beta, MR * tb, "beta") &
        reg_check(a.g_beta, MR * tb, "g_beta") & reg_check(a.m_beta, m2 ? MR * tb : 0.0, "m_beta") &
        reg_check(a.v_beta, m2 ? MR * tb : 0.0, "v_beta")))
    return;
  // E read; gamma read and written (and both Adam moments read and written);
  // the same for beta
  int tk = prof_begin(st, sizeof(T) == 8 ? "gather_gamma_f64" : "gather_gamma_f32", 0.0,
                      ((double)a.R * a.nnz + (m2 ? 6.0 : 2.0) * (NR + MR)) * sizeof(T));
  const int64_t n = a.R * a.N + nb;
  launch_pdl(k_gather<T>, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st, a);
  prof_end(st, tk);
}
template <typename Td>
void certify_relax(cudaStream_t st, const CertArgs<Td>& a) {
  if (a.R <= 0 || a.d <= 0) return;
  const double bytes = (double)a.R * a.d * (8.0 + 4.0 + 8.0 + sizeof(Td)) +
                       (double)a.R * (a.csc.n_entries * sizeof(Td) + ((a.d + 31) / 32) * 8.0);
  const double Rd = (double)a.R * a.d, yr = (a.y_per_spec ? (double)a.K : (double)a.R) * a.d, tb = sizeof(Td);
  if (!(reg_check(a.y, yr * 8.0, "cert y") & reg_check(a.yabs, yr * 4.0, "cert yabs") &
        reg_check(a.lo, a.d * 8.0, "lo") & reg_check(a.hi, a.d * 8.0, "hi") & reg_check(a.bias, a.d * 8.0, "bias") &
        reg_check(a.alpha, Rd * tb, "alpha") & reg_check(a.beta, (double)a.M * a.R * tb, "beta") &
        reg_check(a.gamma, (a.csc.n_total ? (double)a.N * a.R : 0.0) * tb, "gamma") & chk_splits(a.sp, a.R, a.K, a.M) &
        chk_csc(a.csc, a.d) & reg_check(a.nu_out, Rd * 8.0, "cert nu") &
        reg_check(a.nuabs_out, a.nuabs_out ? Rd * 4.0 : 0.0, "cert |nu|") &
        reg_check(a.theta, a.theta ? Rd * tb : 0.0, "cert theta") &
        reg_check(a.obj_part, ((a.d + 31) / 32) * (double)a.R * 8.0, "cert part")))
    return;
  int tk = prof_begin(st, "certify_relax_f64", 0.0, bytes);
  k_certify_relax<Td><<<chunk_blocks(a.R, a.K, a.d), kWarpsPerBlock * 32, 0, st>>>(a);
  prof_end(st, tk);
}
template <typename Td>
void certify_concretize(cudaStream_t st, int64_t R, int K, int N, int d0, const double* y0, const float* y0abs,
                        double gamma_n, const double* x_lo, const double* x_hi, const Td* gamma,
                        CutCSC<double> csc, double* obj_part) {
  if (R <= 0 || d0 <= 0) return;
  if (!(reg_check(y0, (double)R * d0 * 8.0, "cert y0") & reg_check(y0abs, (double)R * d0 * 4.0, "cert y0abs") &
        reg_check(x_lo, d0 * 8.0, "x_lo") & reg_check(x_hi, d0 * 8.0, "x_hi") & chk_csc(csc, d0) &
        reg_check(obj_part, ((d0 + 31) / 32) * (double)R * 8.0, "cert part")))
    return;
  int tk = prof_begin(st, "certify_conc_f64", 0.0, (double)R * d0 * 12.0);
  k_certify_conc<Td><<<chunk_blocks(R, K, d0), kWarpsPerBlock * 32, 0, st>>>(R, K, N, d0, y0, y0abs, gamma_n, x_lo, x_hi,
                                                                    gamma, csc, obj_part);
  prof_end(st, tk);
}
template <typename Td>
void certify_finalize(cudaStream_t st, int64_t R, int K, int N, int P, const double* C, const double* bL, int dL,
                      const double* d, const Td* gamma, const double* obj_part, double* out) {
  if (R <= 0) return;
  if (!(reg_check(C, (double)K * dL * 8.0, "spec C") & reg_check(bL, dL * 8.0, "bL") & reg_check(d, N * 8.0, "d") &
        reg_check(gamma, (double)N * R * sizeof(Td), "gamma") & reg_check(obj_part, (double)P * R * 8.0, "part") &
        reg_check(out, R * 8.0, "cert out")))
    return;
  int tk = prof_begin(st, "certify_final_f64", 0.0, (double)R * (N * sizeof(Td) + P * 8.0 + 8.0));
  k_certify_final<Td><<<row_blocks(R), kWarpsPerBlock * 32, 0, st>>>(R, K, N, P, C, bL, dL, d, gamma, obj_part, out);
  prof_end(st, tk);
}
template <typename Ts, typename Td>
void transpose_cast(cudaStream_t st, int64_t rows, int64_t cols, const Ts* src, Td* dst) {
  if (rows <= 0 || cols <= 0) return;
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  if (!(reg_check(src, (double)rows * cols * sizeof(Ts), "transpose src") &
        reg_check(dst, (double)rows * cols * sizeof(Td), "transpose dst")))
    return;
  int tk = prof_begin(st, "transpose", 0.0, (double)rows * cols * (sizeof(Ts) + sizeof(Td)));
  k_transpose_cast<Ts, Td><<<grid, dim3(32, 8), 0, st>>>(rows, cols, src, dst);
  prof_end(st, tk);
}
template <typename Ts, typename Td>
void cast_copy(cudaStream_t st, int64_t n, const Ts* src, Td* dst) {
  if (n <= 0) return;
  if (!(reg_check(src, (double)n * sizeof(Ts), "cast src") & reg_check(dst, (double)n * sizeof(Td), "cast dst")))
    return;
  int tk = prof_begin(st, "cast", 0.0, (double)n * (sizeof(Ts) + sizeof(Td)));
  k_cast<Ts, Td><<<flat_grid(n), 256, 0, st>>>(n, src, dst);
  prof_end(st, tk);
}
template <typename T>
void default_alpha(cudaStream_t st, int64_t R, int K, int d, int layer, const T* lo, const T* hi, SplitsDev sp,
                   T* alpha) {
  if (R <= 0 || d <= 0) return;
  if (!(reg_check(lo, d * (double)sizeof(T), "lo") & reg_check(hi, d * (double)sizeof(T), "hi") &
        chk_splits(sp, R, K) & reg_check(alpha, (double)R * d * sizeof(T), "alpha")))
    return;
  int tk = prof_begin(st, "default_alpha", 0.0, (double)R * d * sizeof(T));
  k_default_alpha<T><<<flat_grid(R * d), 256, 0, st>>>(R, K, d, layer, lo, hi, sp, alpha);
  prof_end(st, tk);
}

std::string take_device_error(cudaStream_t st) {
  unsigned long long h[3] = {0, 0, 0};
  if (cudaMemcpyFromSymbolAsync(h, g_dev_err, sizeof h, 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return std::string();
  if (h[0] == 0) return std::string();
  const unsigned long long z[3] = {0, 0, 0};
  cudaMemcpyToSymbolAsync(g_dev_err, z, sizeof z, 0, cudaMemcpyHostToDevice, st);
  cudaStreamSynchronize(st);
  static const char* what[] = {"", "cut entry range of a neuron", "cut index", "split range of a subdomain",
                               "cut entry row", "cut entry range of a cut"};
  char buf[192];
  snprintf(buf, sizeof buf, "kernel index check: %s out of range (index %lld, limit %lld)",
           h[0] < 6 ? what[h[0]] : "?", (long long)h[1], (long long)h[2]);
  return buf;
}

#define GCP_INST_CHAIN(T, Top)                                                    \
  template void relax_eval<T, Top>(cudaStream_t, const RelaxArgs<T, Top>&);       \
  template void relax_adjoint<T, Top>(cudaStream_t, const AdjArgs<T, Top>&);      \
  template void concretize<T, Top>(cudaStream_t, const ConcArgs<T, Top>&);
GCP_INST_CHAIN(double, double)
GCP_INST_CHAIN(float, float)
GCP_INST_CHAIN(float, __nv_bfloat16)
template void finalize_bound<double>(cudaStream_t, const FinalArgs<double>&);
template void finalize_bound<float>(cudaStream_t, const FinalArgs<float>&);
template void gather_gamma<double>(cudaStream_t, const GatherArgs<double>&);
template void gather_gamma<float>(cudaStream_t, const GatherArgs<float>&);
template void certify_relax<double>(cudaStream_t, const CertArgs<double>&);
template void certify_relax<float>(cudaStream_t, const CertArgs<float>&);
template void certify_concretize<double>(cudaStream_t, int64_t, int, int, int, const double*, const float*, double,
                                         const double*, const double*, const double*, CutCSC<double>, double*);
template void certify_concretize<float>(cudaStream_t, int64_t, int, int, int, const double*, const float*, double,
                                        const double*, const double*, const float*, CutCSC<double>, double*);
template void certify_finalize<double>(cudaStream_t, int64_t, int, int, int, const double*, const double*, int,
                                       const double*, const double*, const double*, double*);
template void certify_finalize<float>(cudaStream_t, int64_t, int, int, int, const double*, const double*, int,
                                      const double*, const float*, const double*, double*);
template void transpose_cast<double, double>(cudaStream_t, int64_t, int64_t, const double*, double*);
template void transpose_cast<double, float>(cudaStream_t, int64_t, int64_t, const double*, float*);
template void transpose_cast<float, double>(cudaStream_t, int64_t, int64_t, const float*, double*);
template void transpose_cast<float, float>(cudaStream_t, int64_t, int64_t, const float*, float*);
template void cast_copy<double, float>(cudaStream_t, int64_t, const double*, float*);
template void cast_copy<float, double>(cudaStream_t, int64_t, const float*, double*);
template void cast_copy<double, double>(cudaStream_t, int64_t, const double*, double*);
template void cast_copy<float, float>(cudaStream_t, int64_t, const float*, float*);
template void cast_copy<float, __nv_bfloat16>(cudaStream_t, int64_t, const float*, __nv_bfloat16*);
template void default_alpha<double>(cudaStream_t, int64_t, int, int, int, const double*, const double*, SplitsDev,
                                    double*);
template void default_alpha<float>(cudaStream_t, int64_t, int, int, int, const float*, const float*, SplitsDev,
                                   float*);

}  // namespace gcp

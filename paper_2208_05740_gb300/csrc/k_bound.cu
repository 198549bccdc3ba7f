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

#include "gcp_internal.cuh"

namespace gcp {

// First data-dependent index that failed its check: {code, index, limit}; the
// access is skipped. Read and cleared by take_device_error().
__device__ unsigned long long g_dev_err[3];

namespace {

constexpr int kWarpsPerBlock = 8;

__device__ __noinline__ void dev_error(unsigned long long code, long long idx, long long lim) {
  if (atomicCAS(&g_dev_err[0], 0ull, code) == 0ull) {
    g_dev_err[1] = (unsigned long long)idx;
    g_dev_err[2] = (unsigned long long)lim;
  }
}

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

// Entry values coef * gamma[cut] of one batch for row grow, summed per
// neuron lane into t (x), g (xhat), s (z). Batches past the first reload
// their entries (chunks with more than 32 entries).
template <typename T, typename Tg>
__device__ __forceinline__ void cut_sums_row(const CutCSC<T>& c, const ChunkCuts<T>& cc, const Tg* grow, int N,
                                             int ch, int lane, T& t, T& g, T& s) {
  t = T(0); g = T(0); s = T(0);
  for (int b0 = cc.cb; b0 < cc.ce; b0 += 32) {
    int kd = cc.kind, cut = cc.cut;
    T cf = cc.coef;
    if (b0 != cc.cb) {
      const int e = b0 + lane;
      kd = -1; cut = -1; cf = T(0);
      if (e < cc.ce) {
        cut = __ldg(c.cut + e);
        kd = __ldg(c.kind + e);
        cf = __ldg(c.coef + e);
        if (cut < 0 || cut >= N) { dev_error(2, e, N); cut = -1; kd = -1; }
      }
    }
    const T val = cut >= 0 ? cf * (T)grow[cut] : T(0);
    const int lo_e = max(cc.e0, b0), cnt = max(0, min(cc.e1, b0 + 32) - lo_e);
    const int mx = __reduce_max_sync(0xffffffffu, cnt);
    for (int q = 0; q < mx; ++q) {
      const int src = (lo_e + q - b0) & 31;
      const T v = __shfl_sync(0xffffffffu, val, src);
      const int kq = __shfl_sync(0xffffffffu, kd, src);
      if (q < cnt) {
        if (kq == GCP_VAR_X) t += v;
        else if (kq == GCP_VAR_XHAT) g += v;
        else if (kq == GCP_VAR_Z) s += v;
      }
    }
  }
}

// E[r, e] = coef * (x: dt, xhat: -dnh, z: ds) of the entry's neuron, e the
// entry's CSC position (the chunk's entries are contiguous: whole lines).
template <typename T>
__device__ __forceinline__ void cut_writes_row(const CutCSC<T>& c, const ChunkCuts<T>& cc, int ch, int lane, T dt,
                                               T dnh, T ds, T* Erow) {
  for (int b0 = cc.cb; b0 < cc.ce; b0 += 32) {
    int kd = cc.kind, src = cc.nrn_lane;
    T cf = cc.coef;
    const int e = b0 + lane;
    if (b0 != cc.cb) {
      kd = -1; src = 0; cf = T(0);
      if (e < cc.ce) {
        kd = __ldg(c.kind + e);
        src = (__ldg(c.nrn + e) - ch * 32) & 31;
        cf = __ldg(c.coef + e);
      }
    }
    const T vt = __shfl_sync(0xffffffffu, dt, src);
    const T vh = __shfl_sync(0xffffffffu, dnh, src);
    const T vs = __shfl_sync(0xffffffffu, ds, src);
    if (e < cc.ce) Erow[e] = cf * (kd == GCP_VAR_X ? vt : (kd == GCP_VAR_XHAT ? -vh : vs));
  }
}

// Certification variant: round-to-nearest sums with their round-up absolute
// sums and term counts (for Higham's bound), per kind.
template <typename Tg>
__device__ __forceinline__ void cut_sums_row_cert(const CutCSC<double>& c, const ChunkCuts<double>& cc,
                                                  const Tg* grow, int N, int lane, double (&sum)[3],
                                                  double (&abs_)[3], int (&cnt_)[3]) {
  for (int q = 0; q < 3; ++q) { sum[q] = 0.0; abs_[q] = 0.0; cnt_[q] = 0; }
  for (int b0 = cc.cb; b0 < cc.ce; b0 += 32) {
    int kd = cc.kind, cut = cc.cut;
    double cf = cc.coef;
    if (b0 != cc.cb) {
      const int e = b0 + lane;
      kd = -1; cut = -1; cf = 0.0;
      if (e < cc.ce) {
        cut = __ldg(c.cut + e);
        kd = __ldg(c.kind + e);
        cf = __ldg(c.coef + e);
        if (cut < 0 || cut >= N) { dev_error(2, e, N); cut = -1; kd = -1; }
      }
    }
    double val = 0.0, av = 0.0;
    if (cut >= 0) {
      const double gv = (double)grow[cut];
      val = cf * gv;
      av = __dmul_ru(fabs(cf), fabs(gv));
    }
    const int lo_e = max(cc.e0, b0), n = max(0, min(cc.e1, b0 + 32) - lo_e);
    const int mx = __reduce_max_sync(0xffffffffu, n);
    for (int q = 0; q < mx; ++q) {
      const int src = (lo_e + q - b0) & 31;
      const double v = __shfl_sync(0xffffffffu, val, src);
      const double a = __shfl_sync(0xffffffffu, av, src);
      const int kq = __shfl_sync(0xffffffffu, kd, src);
      if (q < n && kq >= 0 && kq <= 2) {
        sum[kq] += v;
        abs_[kq] = __dadd_ru(abs_[kq], a);
        ++cnt_[kq];
      }
    }
  }
}

// One ascent step on x. Adam (Kingma & Ba): bias-corrected moments; the
// float chain uses the fast reciprocal divide (a step size, not a bound).
template <typename T>
__device__ __forceinline__ T step_apply(const StepArgs<T>& st, T x, T grad, T lr, T* m, T* v) {
  if (st.mode == 1) return x + lr * grad;
  T mm = st.b1 * (*m) + (T(1) - st.b1) * grad;
  T vv = st.b2 * (*v) + (T(1) - st.b2) * grad * grad;
  *m = mm;
  *v = vv;
  if constexpr (std::is_same<T, float>::value) {
    return x + lr * __fdividef(mm * st.ic1, __fsqrt_rn(vv * st.ic2) + st.eps);
  } else {
    return x + lr * (mm / st.c1) / (sqrt(vv / st.c2) + st.eps);
  }
}

// ------------------------------------------------------------------ eval
template <typename T, typename Top>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_relax_eval(RelaxArgs<T, Top> a) {
  ChunkWarp w;
  if (!chunk_warp((int)(a.R / a.K), a.d, w)) return;
  const int j = w.j;
  T lo = T(0), hi = T(0), bj = T(0), iv = T(0);
  if (w.on) {
    lo = __ldg(a.lo + j);
    hi = __ldg(a.hi + j);
    bj = __ldg(a.bias + j);
    iv = a.inv_ul ? __ldg(a.inv_ul + j) : (hi > lo ? T(1) / (hi - lo) : T(0));
  }
  int sign = 0;
  const int slot = lane_split(a.sp, w.s, a.M, a.layer, w.c, w.lane, sign);
  if (slot >= 0) {
    if (sign > 0) lo = tmax(lo, T(0)); else hi = tmin(hi, T(0));
  }
  const int cls = hi <= T(0) ? 0 : (lo >= T(0) ? 1 : 2);   // inactive / active / unstable
  ChunkCuts<T> cc;
  chunk_cuts(a.csc, a.N, a.d, w.c, w.lane, cc);
  for (int k = 0; k < a.K; ++k) {
    const int64_t r = (int64_t)w.s * a.K + k;
    const int64_t ij = r * a.d + j;
    T yv = T(0), al = T(0), bv = T(0);
    if (w.on) {
      yv = __ldg(a.y + (a.y_per_spec ? (int64_t)k : r) * a.d + j);
      if (cls == 2) al = __ldg(a.alpha + ij);
      if (slot >= 0) bv = __ldg(a.beta + r * a.M + slot);
    }
    T t, gg, sq;
    cut_sums_row(a.csc, cc, a.gamma + r * a.N, a.N, w.c, w.lane, t, gg, sq);
    T term = T(0);
    if (w.on) {
      if (slot >= 0) t += sign > 0 ? -bv : bv;   // split row -x <= 0 (x >= 0) or x <= 0
      const T nh = yv - gg;
      T nu;
      if (cls == 0) {            // inactive: xhat = 0, z = 0
        nu = -t;
      } else if (cls == 1) {     // active: xhat = x, z = 1
        nu = nh - t;
        term = sq;
      } else {                   // unstable: Lemma A.1 with q = -s
        const T C = tmax(nh, T(0));
        const T pi = tmin(tmax((hi * C - sq) * iv, T(0)), C);
        term = lo * pi - tmax(T(0), hi * (C - pi) + lo * pi - sq);
        nu = pi - al * tmax(-nh, T(0)) - t;
      }
      term -= nu * bj;
      put_operand<Top>(a.nu_out, a.nu_lo, ij, nu);
      a.nuhat_out[ij] = nh;
    }
    term = warp_sum(term);
    if (w.lane == 0) a.obj_part[(int64_t)w.c * a.R + r] = term;
  }
}

// ------------------------------------------------------------------ adjoint
template <typename T, typename Top>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_relax_adj(AdjArgs<T, Top> a) {
  ChunkWarp w;
  if (!chunk_warp((int)(a.R / a.K), a.d, w)) return;
  const int j = w.j;
  T lo = T(0), hi = T(0), bj = T(0), iv = T(0);
  if (w.on) {
    lo = __ldg(a.lo + j);
    hi = __ldg(a.hi + j);
    bj = __ldg(a.bias + j);
    iv = a.inv_ul ? __ldg(a.inv_ul + j) : (hi > lo ? T(1) / (hi - lo) : T(0));
  }
  int sign = 0;
  const int slot = lane_split(a.sp, w.s, a.M, a.layer, w.c, w.lane, sign);
  if (slot >= 0) {
    if (sign > 0) lo = tmax(lo, T(0)); else hi = tmin(hi, T(0));
  }
  const int cls = hi <= T(0) ? 0 : (lo >= T(0) ? 1 : 2);
  ChunkCuts<T> cc;
  chunk_cuts(a.csc, a.N, a.d, w.c, w.lane, cc);
  for (int k = 0; k < a.K; ++k) {
    const int64_t r = (int64_t)w.s * a.K + k;
    const int64_t ij = r * a.d + j;
    const T wr = a.seed ? a.seed[r] : T(1);
    T nbv = T(0), nh = T(0), al = T(0);
    if (w.on) {
      nbv = __ldg(a.nubar + ij);
      if (cls == 2) {
        nh = __ldg(a.nuhat + ij);
        al = a.alpha[ij];
      }
    }
    T t, gg, sq;
    cut_sums_row(a.csc, cc, a.gamma + r * a.N, a.N, w.c, w.lane, t, gg, sq);
    const T nb = nbv - wr * bj;   // dg/dnu^(i)
    T dnu_dnh = T(0), dh_dnh = T(0), dnu_ds = T(0), dh_ds = T(0);
    if (w.on) {
      if (cls != 2) {
        if (cls == 1) { dnu_dnh = T(1); dh_ds = wr; }     // active
        if (a.st.mode == 0) a.g_alpha[ij] = T(0);
      } else {
        if (nh > T(0)) {
          const T p0 = (hi * nh - sq) * iv;
          if (p0 > T(0) && p0 < nh) {          // pi* = p0
            dnu_dnh = hi * iv;
            dh_dnh = wr * lo * hi * iv;
            dnu_ds = -iv;
            dh_ds = -wr * lo * iv;
          } else if (p0 >= nh) {               // pi* = C, h = s when l C - s > 0
            dnu_dnh = T(1);
            dh_ds = (lo * nh - sq > T(0)) ? wr : T(0);
          }
        } else {
          if (nh < T(0)) dnu_dnh = al;         // nu = alpha * nuhat
          dh_ds = (sq < T(0)) ? wr : T(0);     // h = min(s, 0)
        }
        const T g_alpha = nb * (-tmax(-nh, T(0)));
        if (a.st.mode == 0) {
          a.g_alpha[ij] = g_alpha;
        } else {
          T na = step_apply(a.st, al, g_alpha, a.st.lr_a, a.m_alpha ? a.m_alpha + ij : nullptr,
                            a.v_alpha ? a.v_alpha + ij : nullptr);
          a.alpha[ij] = tmin(tmax(na, T(0)), T(1));
        }
      }
    }
    const T dg_dnh = nb * dnu_dnh + dh_dnh;
    const T dg_ds = nb * dnu_ds + dh_ds;
    const T dg_dt = -nb;
    if (a.E) cut_writes_row(a.csc, cc, w.c, w.lane, dg_dt, dg_dnh, dg_ds, a.E + r * a.csc.n_total);
    if (!w.on) continue;
    if (a.a_out) put_operand<Top>(a.a_out, a.a_lo, ij, dg_dnh);
    if (slot >= 0) {
      const int64_t bi = r * a.M + slot;
      const T gb = (sign > 0 ? T(-1) : T(1)) * dg_dt;
      if (a.st.mode == 0) {
        a.g_beta[bi] = gb;
      } else {
        T nbv2 = step_apply(a.st, a.beta[bi], gb, a.st.lr_b, a.m_beta ? a.m_beta + bi : nullptr,
                            a.v_beta ? a.v_beta + bi : nullptr);
        a.beta[bi] = tmax(nbv2, T(0));
      }
    }
  }
}

// ------------------------------------------------------------------ concretization
template <typename T, typename Top>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_concretize(ConcArgs<T, Top> a) {
  ChunkWarp w;
  if (!chunk_warp((int)(a.R / a.K), a.d0, w)) return;
  const int j = w.j;
  T xl = T(0), xh = T(0);
  if (w.on) {
    xl = __ldg(a.x_lo + j);
    xh = __ldg(a.x_hi + j);
  }
  ChunkCuts<T> cc;
  chunk_cuts(a.csc, a.N, a.d0, w.c, w.lane, cc);
  for (int k = 0; k < a.K; ++k) {
    const int64_t r = (int64_t)w.s * a.K + k;
    const int64_t ij = r * a.d0 + j;
    const T wr = a.seed ? a.seed[r] : T(1);
    const T yv = w.on ? __ldg(a.y0 + ij) : T(0);
    T h0, ug, us;
    cut_sums_row(a.csc, cc, a.gamma + r * a.N, a.N, w.c, w.lane, h0, ug, us);   // layer 0: kind x only
    const T c0 = -yv + h0;
    const T xs = c0 > T(0) ? xl : (c0 < T(0) ? xh : T(0.5) * (xl + xh));
    if (a.E) cut_writes_row(a.csc, cc, w.c, w.lane, wr * xs, T(0), T(0), a.E + r * a.csc.n_total);
    T term = w.on ? tmin(c0 * xl, c0 * xh) : T(0);
    if (w.on && a.a0_out) put_operand<Top>(a.a0_out, a.a0_lo, ij, -wr * xs);
    term = warp_sum(term);
    if (w.lane == 0) a.obj_part[(int64_t)w.c * a.R + r] = term;
  }
}

// g[r] = c_k^T b^(L) - gamma_r^T d + sum of the partials; one warp per row.
template <typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_finalize(FinalArgs<T> a) {
  const int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (r >= a.R) return;
  const int lane = threadIdx.x & 31;
  T g = T(0);
  for (int n = lane; n < a.N; n += 32) g -= a.gamma[r * a.N + n] * a.d[n];
  for (int q = lane; q < a.P; q += 32) g += a.obj_part[(int64_t)q * a.R + r];
  g = warp_sum(g);
  if (lane == 0) a.g[r] = g + a.cb[(int)(r % a.K)];
}

// dg/dgamma_k = -d_k + sum of the cut's entry values (violation of cut k at the
// primal point implied by the duals), then the projected step on gamma.
template <typename T>
__global__ void k_gather(GatherArgs<T> a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.R * a.N) return;
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
  const T w = a.seed ? a.seed[r] : T(1);
  T grad = -w * a.d[n];
  int e0 = a.cut_ptr[n], e1 = a.cut_ptr[n + 1];
  if (e0 < 0 || e1 < e0 || (int64_t)e1 > a.nnz) { dev_error(5, n, a.nnz); e0 = e1 = 0; }
  const T* Er = a.E + r * a.nnz;
  for (int e = e0; e < e1; ++e) {
    const int q = __ldg(a.pos + e);
    if (q < 0 || (int64_t)q >= a.nnz) { dev_error(5, e, a.nnz); continue; }
    grad += Er[q];
  }
  if (a.st.mode == 0) {
    a.g_gamma[i] = grad;
  } else {
    T x = step_apply(a.st, a.gamma[i], grad, a.st.lr_g, a.m_gamma ? a.m_gamma + i : nullptr,
                     a.v_gamma ? a.v_gamma + i : nullptr);
    a.gamma[i] = tmax(x, T(0));
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
  for (int k = 0; k < a.K; ++k) {
    const int64_t r = (int64_t)w.s * a.K + k;
    double sum[3], abs_[3];
    int cnt_[3];
    cut_sums_row_cert(a.csc, cc, a.gamma + r * a.N, a.N, w.lane, sum, abs_, cnt_);
    double part = 0.0;
    if (w.on) {
    // sparse sums in round-to-nearest with their Higham error bounds
    double t = sum[GCP_VAR_X], gg = sum[GCP_VAR_XHAT], sq = sum[GCP_VAR_Z];
    double ta = abs_[GCP_VAR_X];
    int nt = cnt_[GCP_VAR_X];
    double lo = a.lo[j], hi = a.hi[j];
    if (slot >= 0) {
      const double bv = (double)a.beta[r * a.M + slot];
      if (sign > 0) { t -= bv; lo = fmax(lo, 0.0); }
      else { t += bv; hi = fmin(hi, 0.0); }
      ta = __dadd_ru(ta, fabs(bv));
      ++nt;
    }
    const double et = __dmul_ru(gamma_of(nt), ta);
    const double eg = __dmul_ru(gamma_of(cnt_[GCP_VAR_XHAT]), abs_[GCP_VAR_XHAT]);
    const double es = __dmul_ru(gamma_of(cnt_[GCP_VAR_Z]), abs_[GCP_VAR_Z]);
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
      const double p0 = (hi * C - sq) / (hi - lo);
      const double pi = fmin(fmax(p0, 0.0), C);
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
    part = __dadd_rd(part, __dmul_rd(-nu, a.bias[j]));
    a.nu_out[r * a.d + j] = nu;
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
  for (int k = 0; k < K; ++k) {
    const int64_t r = (int64_t)w.s * K + k;
    double sum[3], abs_[3];
    int cnt_[3];
    cut_sums_row_cert(csc, cc, gamma + r * N, N, w.lane, sum, abs_, cnt_);
    double part = 0.0;
    if (w.on) {
      const double h = sum[GCP_VAR_X];
      const double eh = __dmul_ru(gamma_of(cnt_[GCP_VAR_X]), abs_[GCP_VAR_X]);
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

// host-side extent checks shared by the launchers
inline bool chk_splits(const SplitsDev& sp, int64_t R, int K) {
  const double S = K > 0 ? (double)(R / K) : 0.0;
  return reg_check(sp.ptr, (S + 1) * 4.0, "split ptr") & reg_check(sp.layer, sp.n * 2.0, "split layer") &
         reg_check(sp.index, sp.n * 4.0, "split index") & reg_check(sp.sign, (double)sp.n, "split sign");
}
template <typename T>
inline bool chk_csc(const CutCSC<T>& c, int d) {
  return reg_check(c.ptr, (d + 1) * 4.0, "csc ptr") & reg_check(c.cut, c.n_total * 4.0, "csc cut") &
         reg_check(c.kind, (double)c.n_total, "csc kind") & reg_check(c.coef, c.n_total * (double)sizeof(T), "csc coef") &
         reg_check(c.nrn, c.n_total * 4.0, "csc nrn");
}

// Algorithmic bytes per launch: every per-(row, neuron) array read or written
// once, one gamma read (and E write) per cut entry and row, partial sums.
template <typename T, typename Top>
void relax_eval(cudaStream_t st, const RelaxArgs<T, Top>& a) {
  if (a.R <= 0 || a.d <= 0) return;
  char nm[48];
  snprintf(nm, sizeof nm, "relax_eval_%s%s", tsfx<T>(), sizeof(Top) == 2 ? "_bf16" : "");
  const double bytes = (double)a.R * a.d * (3.0 * sizeof(T) + sizeof(Top)) +
                       (double)a.R * (a.csc.n_entries + (a.d + 31) / 32) * sizeof(T);
  const double Rd = (double)a.R * a.d, tb = sizeof(T);
  if (!(reg_check(a.y, (a.y_per_spec ? (double)a.K : (double)a.R) * a.d * tb, "relax y") &
        reg_check(a.lo, a.d * tb, "lo") & reg_check(a.hi, a.d * tb, "hi") & reg_check(a.bias, a.d * tb, "bias") &
        reg_check(a.inv_ul, a.inv_ul ? a.d * tb : 0.0, "inv_ul") &
        reg_check(a.alpha, Rd * tb, "alpha") & reg_check(a.beta, (double)a.M * a.R * tb, "beta") &
        reg_check(a.gamma, (a.csc.n_total ? (double)a.N * a.R : 0.0) * tb, "gamma") & chk_splits(a.sp, a.R, a.K) &
        chk_csc(a.csc, a.d) & reg_check(a.nu_out, Rd * sizeof(Top), "nu out") &
        reg_check(a.nu_lo, a.nu_lo ? Rd * 4.0 : 0.0, "nu lo") &
        reg_check(a.nuhat_out, Rd * tb, "nuhat out") & reg_check(a.obj_part, ((a.d + 31) / 32) * (double)a.R * tb, "obj part")))
    return;
  int tk = prof_begin(st, nm, 0.0, bytes);
  k_relax_eval<T, Top><<<chunk_blocks(a.R, a.K, a.d), kWarpsPerBlock * 32, 0, st>>>(a);
  prof_end(st, tk);
}
template <typename T, typename Top>
void relax_adjoint(cudaStream_t st, const AdjArgs<T, Top>& a) {
  if (a.R <= 0 || a.d <= 0) return;
  char nm[48];
  snprintf(nm, sizeof nm, "relax_adj_%s%s", tsfx<T>(), sizeof(Top) == 2 ? "_bf16" : "");
  const double bytes = (double)a.R * a.d * (4.0 * sizeof(T) + (a.a_out ? sizeof(Top) : 0)) +
                       (double)a.R * a.csc.n_entries * 2.0 * sizeof(T);
  const double Rd = (double)a.R * a.d, tb = sizeof(T);
  const bool m0 = a.st.mode == 0, m2 = a.st.mode == 2;
  if (!(reg_check(a.nubar, Rd * tb, "nubar") & reg_check(a.seed, a.seed ? a.R * tb : 0.0, "seed") &
        reg_check(a.lo, a.d * tb, "lo") & reg_check(a.hi, a.d * tb, "hi") & reg_check(a.bias, a.d * tb, "bias") &
        reg_check(a.inv_ul, a.inv_ul ? a.d * tb : 0.0, "inv_ul") &
        reg_check(a.alpha, Rd * tb, "alpha") & reg_check(a.beta, (double)a.M * a.R * tb, "beta") &
        reg_check(a.gamma, (a.csc.n_total ? (double)a.N * a.R : 0.0) * tb, "gamma") &
        reg_check(a.nuhat, Rd * tb, "nuhat") & chk_splits(a.sp, a.R, a.K) & chk_csc(a.csc, a.d) &
        reg_check(a.a_out, a.a_out ? Rd * sizeof(Top) : 0.0, "a out") &
        reg_check(a.a_lo, (a.a_out && a.a_lo) ? Rd * 4.0 : 0.0, "a lo") &
        reg_check(a.E, a.csc.n_entries ? (double)a.csc.n_total * a.R * tb : 0.0, "E") &
        reg_check(a.g_alpha, m0 ? Rd * tb : 0.0, "g_alpha") &
        reg_check(a.g_beta, m0 ? (double)a.M * a.R * tb : 0.0, "g_beta") &
        reg_check(a.m_alpha, m2 ? Rd * tb : 0.0, "m_alpha") & reg_check(a.v_alpha, m2 ? Rd * tb : 0.0, "v_alpha") &
        reg_check(a.m_beta, m2 ? (double)a.M * a.R * tb : 0.0, "m_beta") &
        reg_check(a.v_beta, m2 ? (double)a.M * a.R * tb : 0.0, "v_beta")))
    return;
  int tk = prof_begin(st, nm, 0.0, bytes);
  k_relax_adj<T, Top><<<chunk_blocks(a.R, a.K, a.d), kWarpsPerBlock * 32, 0, st>>>(a);
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
        reg_check(a.obj_part, ((a.d0 + 31) / 32) * (double)a.R * tb, "obj part")))
    return;
  int tk = prof_begin(st, nm, 0.0, bytes);
  k_concretize<T, Top><<<chunk_blocks(a.R, a.K, a.d0), kWarpsPerBlock * 32, 0, st>>>(a);
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
  k_finalize<T><<<row_blocks(a.R), kWarpsPerBlock * 32, 0, st>>>(a);
  prof_end(st, tk);
}
template <typename T>
void gather_gamma(cudaStream_t st, const GatherArgs<T>& a) {
  if (a.R <= 0 || a.N <= 0) return;
  const double tb = sizeof(T), NR = (double)a.N * a.R;
  const bool m0 = a.st.mode == 0, m2 = a.st.mode == 2;
  if (!(reg_check(a.cut_ptr, (a.N + 1) * 4.0, "cut ptr") & reg_check(a.pos, a.nnz * 4.0, "cut pos") &
        reg_check(a.E, (double)a.nnz * a.R * tb, "E") &
        reg_check(a.d, a.N * tb, "d") & reg_check(a.seed, a.seed ? a.R * tb : 0.0, "seed") &
        reg_check(a.gamma, NR * tb, "gamma") & reg_check(a.g_gamma, m0 ? NR * tb : 0.0, "g_gamma") &
        reg_check(a.m_gamma, m2 ? NR * tb : 0.0, "m_gamma") & reg_check(a.v_gamma, m2 ? NR * tb : 0.0, "v_gamma") &
        reg_check(a.cut_lo, a.cut_lo ? (double)(a.R / a.K) * 4.0 : 0.0, "cut lo") &
        reg_check(a.cut_hi, a.cut_hi ? (double)(a.R / a.K) * 4.0 : 0.0, "cut hi")))
    return;
  int tk = prof_begin(st, sizeof(T) == 8 ? "gather_gamma_f64" : "gather_gamma_f32", 0.0,
                      (double)a.R * (a.nnz + 2.0 * a.N) * sizeof(T));
  k_gather<T><<<(unsigned)((a.R * a.N + 255) / 256), 256, 0, st>>>(a);
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
        reg_check(a.gamma, (a.csc.n_total ? (double)a.N * a.R : 0.0) * tb, "gamma") & chk_splits(a.sp, a.R, a.K) &
        chk_csc(a.csc, a.d) & reg_check(a.nu_out, Rd * 8.0, "cert nu") &
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

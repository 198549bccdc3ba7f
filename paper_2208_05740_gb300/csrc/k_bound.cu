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

// entry range of neuron j, checked against the entry count
template <typename T>
__device__ __forceinline__ void csc_range(const CutCSC<T>& c, int j, int& e0, int& e1) {
  e0 = c.ptr[j];
  e1 = c.ptr[j + 1];
  if (e0 < 0 || e1 < e0 || (int64_t)e1 > c.n_total) {
    dev_error(1, j, c.n_total);
    e0 = e1 = 0;
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

// Warp coordinates: (row r, neuron chunk c, neuron j = 32c + lane). Returns
// false for warps past the end (the whole warp leaves together).
struct WarpPos {
  int64_t r;
  int c, j, lane;
  bool on;
};
__device__ __forceinline__ bool warp_pos(int64_t R, int d, WarpPos& p) {
  const int nch = (d + 31) >> 5;
  const int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (w >= R * nch) return false;
  p.r = w / nch;
  p.c = (int)(w - p.r * nch);
  p.lane = threadIdx.x & 31;
  p.j = p.c * 32 + p.lane;
  p.on = p.j < d;
  return true;
}

// Sparse cut sums for neuron j of row r: t = H^T gamma, g = G^T gamma, s = Q^T gamma.
template <typename T, typename Tg>
__device__ __forceinline__ void cut_sums(const CutCSC<T>& c, const Tg* grow, int N, int j, T& t, T& g, T& s) {
  t = T(0); g = T(0); s = T(0);
  int e0, e1;
  csc_range(c, j, e0, e1);
  for (int e = e0; e < e1; ++e) {
    const int k = c.cut[e];
    if (k < 0 || k >= N) { dev_error(2, e, N); continue; }
    const T v = c.coef[e] * (T)grow[k];
    const int kd = c.kind[e];
    if (kd == GCP_VAR_X) t += v;
    else if (kd == GCP_VAR_XHAT) g += v;
    else s += v;
  }
}

template <typename T>
__device__ __forceinline__ T step_apply(const StepArgs<T>& st, T x, T grad, T lr, T* m, T* v) {
  if (st.mode == 1) return x + lr * grad;
  T mm = st.b1 * (*m) + (T(1) - st.b1) * grad;
  T vv = st.b2 * (*v) + (T(1) - st.b2) * grad * grad;
  *m = mm;
  *v = vv;
  return x + lr * (mm / st.c1) / (sqrt(vv / st.c2) + st.eps);
}

// ------------------------------------------------------------------ eval
template <typename T, typename Top>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_relax_eval(RelaxArgs<T, Top> a) {
  WarpPos p;
  if (!warp_pos(a.R, a.d, p)) return;
  const int64_t r = p.r;
  const int j = p.j;
  const int s = (int)(r / a.K), k = (int)(r - (int64_t)s * a.K);
  T term = T(0);
  if (p.on) {
    T t, gg, sq;
    cut_sums(a.csc, a.gamma + r * a.N, a.N, j, t, gg, sq);
    T lo = a.lo[j], hi = a.hi[j];
    int q0, q1;
    split_range(a.sp, s, a.M, q0, q1);
    for (int q = q0; q < q1; ++q)
      if (a.sp.layer[q] == a.layer && a.sp.index[q] == j) {
        const T bv = a.beta[r * a.M + (q - q0)];
        if (a.sp.sign[q] > 0) { t -= bv; lo = tmax(lo, T(0)); }   // row -x <= 0
        else { t += bv; hi = tmin(hi, T(0)); }                    // row  x <= 0
      }
    const T nh = a.y[(a.y_per_spec ? (int64_t)k : r) * a.d + j] - gg;
    T nu;
    if (hi <= T(0)) {            // inactive: xhat = 0, z = 0
      nu = -t;
    } else if (lo >= T(0)) {     // active: xhat = x, z = 1
      nu = nh - t;
      term = sq;
    } else {                     // unstable: Lemma A.1 with q = -s
      const T C = tmax(nh, T(0));
      const T p0 = (hi * C - sq) / (hi - lo);
      const T pi = tmin(tmax(p0, T(0)), C);
      term = lo * pi - tmax(T(0), hi * (C - pi) + lo * pi - sq);
      const T tau = a.alpha[r * a.d + j] * tmax(-nh, T(0));
      nu = pi - tau - t;
    }
    term -= nu * a.bias[j];
    put_operand<Top>(a.nu_out, a.nu_lo, r * a.d + j, nu);
    a.nuhat_out[r * a.d + j] = nh;
  }
  term = warp_sum(term);
  if (p.lane == 0) a.obj_part[(int64_t)p.c * a.R + r] = term;
}

// ------------------------------------------------------------------ adjoint
template <typename T, typename Top>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_relax_adj(AdjArgs<T, Top> a) {
  WarpPos p;
  if (!warp_pos(a.R, a.d, p) || !p.on) return;
  const int64_t r = p.r;
  const int j = p.j;
  const int s = (int)(r / a.K);
  const T w = a.seed ? a.seed[r] : T(1);
  const int64_t ij = r * a.d + j;
  const T nb = a.nubar[ij] - w * a.bias[j];   // dg/dnu^(i)
  T t, gg, sq;
  cut_sums(a.csc, a.gamma + r * a.N, a.N, j, t, gg, sq);
  T lo = a.lo[j], hi = a.hi[j];
  int q0, q1;
  split_range(a.sp, s, a.M, q0, q1);
  int split_q = -1;
  for (int q = q0; q < q1; ++q)
    if (a.sp.layer[q] == a.layer && a.sp.index[q] == j) {
      split_q = q;
      if (a.sp.sign[q] > 0) lo = tmax(lo, T(0)); else hi = tmin(hi, T(0));
    }
  T dnu_dnh = T(0), dh_dnh = T(0), dnu_ds = T(0), dh_ds = T(0);
  const bool unstable = !(hi <= T(0)) && !(lo >= T(0));
  if (!unstable) {
    if (!(hi <= T(0))) { dnu_dnh = T(1); dh_ds = w; }     // active
    if (a.st.mode == 0) a.g_alpha[ij] = T(0);
  } else {
    const T nh = a.nuhat[ij];
    const T al = a.alpha[ij];
    if (nh > T(0)) {
      const T ul = hi - lo;
      const T p0 = (hi * nh - sq) / ul;
      if (p0 > T(0) && p0 < nh) {          // pi* = p0
        dnu_dnh = hi / ul;
        dh_dnh = w * lo * hi / ul;
        dnu_ds = -T(1) / ul;
        dh_ds = -w * lo / ul;
      } else if (p0 >= nh) {               // pi* = C, h = s when l C - s > 0
        dnu_dnh = T(1);
        dh_ds = (lo * nh - sq > T(0)) ? w : T(0);
      }
    } else {
      if (nh < T(0)) dnu_dnh = al;         // nu = alpha * nuhat
      dh_ds = (sq < T(0)) ? w : T(0);      // h = min(s, 0)
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
  const T dg_dnh = nb * dnu_dnh + dh_dnh;
  const T dg_ds = nb * dnu_ds + dh_ds;
  const T dg_dt = -nb;
  if (a.a_out) put_operand<Top>(a.a_out, a.a_lo, ij, dg_dnh);
  int e0, e1;
  csc_range(a.csc, j, e0, e1);
  for (int e = e0; e < e1; ++e) {
    const int kd = a.csc.kind[e];
    const T v = kd == GCP_VAR_X ? dg_dt : (kd == GCP_VAR_XHAT ? -dg_dnh : dg_ds);
    const int row = a.csc.eid[e];
    if (row < 0 || (int64_t)row >= a.csc.n_total) { dev_error(4, e, a.csc.n_total); continue; }
    a.E[r * a.csc.n_total + row] = a.csc.coef[e] * v;
  }
  if (split_q >= 0) {
    const int64_t bi = r * a.M + (split_q - q0);
    const T gb = (a.sp.sign[split_q] > 0 ? T(-1) : T(1)) * dg_dt;
    if (a.st.mode == 0) {
      a.g_beta[bi] = gb;
    } else {
      T nbv = step_apply(a.st, a.beta[bi], gb, a.st.lr_b, a.m_beta ? a.m_beta + bi : nullptr,
                         a.v_beta ? a.v_beta + bi : nullptr);
      a.beta[bi] = tmax(nbv, T(0));
    }
  }
}

// ------------------------------------------------------------------ concretization
template <typename T, typename Top>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_concretize(ConcArgs<T, Top> a) {
  WarpPos p;
  if (!warp_pos(a.R, a.d0, p)) return;
  const int64_t r = p.r;
  const int j = p.j;
  T term = T(0);
  if (p.on) {
    const T w = a.seed ? a.seed[r] : T(1);
    const T* grow = a.gamma + r * a.N;
    T h0 = T(0);
    int e0, e1;
    csc_range(a.csc, j, e0, e1);
    for (int e = e0; e < e1; ++e) {
      const int kc = a.csc.cut[e];
      if (kc < 0 || kc >= a.N) { dev_error(2, e, a.N); continue; }
      h0 += a.csc.coef[e] * grow[kc];
    }
    const T c0 = -a.y0[r * a.d0 + j] + h0;
    const T xl = a.x_lo[j], xh = a.x_hi[j];
    term = tmin(c0 * xl, c0 * xh);
    const T xs = c0 > T(0) ? xl : (c0 < T(0) ? xh : T(0.5) * (xl + xh));
    if (a.a0_out) put_operand<Top>(a.a0_out, a.a0_lo, r * a.d0 + j, -w * xs);
    if (a.E)
      for (int e = e0; e < e1; ++e) {
        const int row = a.csc.eid[e];
        if (row < 0 || (int64_t)row >= a.csc.n_total) { dev_error(4, e, a.csc.n_total); continue; }
        a.E[r * a.csc.n_total + row] = a.csc.coef[e] * w * xs;
      }
  }
  term = warp_sum(term);
  if (p.lane == 0) a.obj_part[(int64_t)p.c * a.R + r] = term;
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
  const T w = a.seed ? a.seed[r] : T(1);
  T grad = -w * a.d[n];
  int e0 = a.cut_ptr[n], e1 = a.cut_ptr[n + 1];
  if (e0 < 0 || e1 < e0 || (int64_t)e1 > a.nnz) { dev_error(5, n, a.nnz); e0 = e1 = 0; }
  const T* Er = a.E + r * a.nnz;
  for (int e = e0; e < e1; ++e) grad += Er[e];
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
  WarpPos p;
  if (!warp_pos(a.R, a.d, p)) return;
  const int64_t r = p.r;
  const int j = p.j;
  const int s = (int)(r / a.K), k = (int)(r - (int64_t)s * a.K);
  double part = 0.0;
  if (p.on) {
    const int64_t yi = (a.y_per_spec ? (int64_t)k : r) * a.d + j;
    const Td* grow = a.gamma + r * a.N;
    // sparse sums in round-to-nearest with their Higham error bounds
    double t = 0, gg = 0, sq = 0, ta = 0, ga = 0, sa = 0;
    int nt = 0, ng = 0, ns = 0;
    int e0, e1;
    csc_range(a.csc, j, e0, e1);
    for (int e = e0; e < e1; ++e) {
      const int kc = a.csc.cut[e];
      if (kc < 0 || kc >= a.N) { dev_error(2, e, a.N); continue; }
      const double gv = (double)grow[kc];
      const double v = a.csc.coef[e] * gv;
      const double av = __dmul_ru(fabs(a.csc.coef[e]), fabs(gv));
      const int kd = a.csc.kind[e];
      if (kd == GCP_VAR_X) { t += v; ta = __dadd_ru(ta, av); ++nt; }
      else if (kd == GCP_VAR_XHAT) { gg += v; ga = __dadd_ru(ga, av); ++ng; }
      else { sq += v; sa = __dadd_ru(sa, av); ++ns; }
    }
    double lo = a.lo[j], hi = a.hi[j];
    int q0, q1;
    split_range(a.sp, s, a.M, q0, q1);
    for (int q = q0; q < q1; ++q)
      if (a.sp.layer[q] == a.layer && a.sp.index[q] == j) {
        const double bv = (double)a.beta[r * a.M + (q - q0)];
        if (a.sp.sign[q] > 0) { t -= bv; lo = fmax(lo, 0.0); }
        else { t += bv; hi = fmin(hi, 0.0); }
        ta = __dadd_ru(ta, fabs(bv));
        ++nt;
      }
    const double et = __dmul_ru(gamma_of(nt), ta);
    const double eg = __dmul_ru(gamma_of(ng), ga);
    const double es = __dmul_ru(gamma_of(ns), sa);
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
  if (p.lane == 0) a.obj_part[(int64_t)p.c * a.R + r] = part;
}

template <typename Td>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_certify_conc(int64_t R, int K, int N, int d0,
                                                                       const double* y0, const float* y0abs,
                                                                       double gamma_n, const double* x_lo,
                                                                       const double* x_hi, const Td* gamma,
                                                                       CutCSC<double> csc, double* obj_part) {
  WarpPos p;
  if (!warp_pos(R, d0, p)) return;
  const int64_t r = p.r;
  const int j = p.j;
  double part = 0.0;
  if (p.on) {
    const Td* grow = gamma + r * N;
    double h = 0, ha = 0;
    int n = 0;
    int e0, e1;
    csc_range(csc, j, e0, e1);
    for (int e = e0; e < e1; ++e) {
      const int kc = csc.cut[e];
      if (kc < 0 || kc >= N) { dev_error(2, e, N); continue; }
      const double gv = (double)grow[kc];
      h += csc.coef[e] * gv;
      ha = __dadd_ru(ha, __dmul_ru(fabs(csc.coef[e]), fabs(gv)));
      ++n;
    }
    const double eh = __dmul_ru(gamma_of(n), ha);
    const double y = y0[r * d0 + j];
    const double ey = __dmul_ru(gamma_n, (double)y0abs[r * d0 + j]);
    const double c_lo = __dadd_rd(__dsub_rd(-y, ey), __dsub_rd(h, eh));
    const double c_hi = __dadd_ru(__dadd_ru(-y, ey), __dadd_ru(h, eh));
    part = box_min_rd(c_lo, c_hi, x_lo[j], x_hi[j]);
  }
  part = warp_sum_rd(part);
  if (p.lane == 0) obj_part[(int64_t)p.c * R + r] = part;
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

// one warp per (row, 32-neuron chunk)
inline unsigned warp_blocks(int64_t R, int d) {
  const int64_t warps = R * (int64_t)((d + 31) / 32);
  return (unsigned)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
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
inline double chunks(int d) { return (double)((d + kChunk - 1) / kChunk); }

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
         reg_check(c.eid, c.n_total * 4.0, "csc eid");
}

// Algorithmic bytes per launch: every per-(row, neuron) array read or written
// once, one gamma read (and E write) per cut entry and row, partial sums.
template <typename T, typename Top>
void relax_eval(cudaStream_t st, const RelaxArgs<T, Top>& a) {
  if (a.R <= 0 || a.d <= 0) return;
  char nm[48];
  snprintf(nm, sizeof nm, "relax_eval_%s%s", tsfx<T>(), sizeof(Top) == 2 ? "_bf16" : "");
  const double bytes = (double)a.R * a.d * (3.0 * sizeof(T) + sizeof(Top)) +
                       (double)a.R * (a.csc.n_entries + chunks(a.d)) * sizeof(T);
  const double Rd = (double)a.R * a.d, tb = sizeof(T);
  if (!(reg_check(a.y, (a.y_per_spec ? (double)a.K : (double)a.R) * a.d * tb, "relax y") &
        reg_check(a.lo, a.d * tb, "lo") & reg_check(a.hi, a.d * tb, "hi") & reg_check(a.bias, a.d * tb, "bias") &
        reg_check(a.alpha, Rd * tb, "alpha") & reg_check(a.beta, (double)a.M * a.R * tb, "beta") &
        reg_check(a.gamma, (a.csc.n_total ? (double)a.N * a.R : 0.0) * tb, "gamma") & chk_splits(a.sp, a.R, a.K) &
        chk_csc(a.csc, a.d) & reg_check(a.nu_out, Rd * sizeof(Top), "nu out") &
        reg_check(a.nu_lo, a.nu_lo ? Rd * 4.0 : 0.0, "nu lo") &
        reg_check(a.nuhat_out, Rd * tb, "nuhat out") & reg_check(a.obj_part, chunks(a.d) * a.R * tb, "obj part")))
    return;
  int tk = prof_begin(st, nm, 0.0, bytes);
  k_relax_eval<T, Top><<<warp_blocks(a.R, a.d), kWarpsPerBlock * 32, 0, st>>>(a);
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
  k_relax_adj<T, Top><<<warp_blocks(a.R, a.d), kWarpsPerBlock * 32, 0, st>>>(a);
  prof_end(st, tk);
}
template <typename T, typename Top>
void concretize(cudaStream_t st, const ConcArgs<T, Top>& a) {
  if (a.R <= 0 || a.d0 <= 0) return;
  char nm[48];
  snprintf(nm, sizeof nm, "concretize_%s", tsfx<T>());
  const double bytes = (double)a.R * a.d0 * (sizeof(T) + (a.a0_out ? sizeof(Top) : 0)) +
                       (double)a.R * (a.csc.n_entries * (a.E ? 2.0 : 1.0) + chunks(a.d0)) * sizeof(T);
  const double Rd = (double)a.R * a.d0, tb = sizeof(T);
  if (!(reg_check(a.y0, Rd * tb, "y0") & reg_check(a.x_lo, a.d0 * tb, "x_lo") & reg_check(a.x_hi, a.d0 * tb, "x_hi") &
        reg_check(a.gamma, (a.csc.n_total ? (double)a.N * a.R : 0.0) * tb, "gamma") &
        reg_check(a.seed, a.seed ? a.R * tb : 0.0, "seed") & chk_csc(a.csc, a.d0) &
        reg_check(a.a0_out, a.a0_out ? Rd * sizeof(Top) : 0.0, "a0 out") &
        reg_check(a.a0_lo, (a.a0_out && a.a0_lo) ? Rd * 4.0 : 0.0, "a0 lo") &
        reg_check(a.E, (a.E && a.csc.n_entries) ? (double)a.csc.n_total * a.R * tb : 0.0, "E") &
        reg_check(a.obj_part, chunks(a.d0) * a.R * tb, "obj part")))
    return;
  int tk = prof_begin(st, nm, 0.0, bytes);
  k_concretize<T, Top><<<warp_blocks(a.R, a.d0), kWarpsPerBlock * 32, 0, st>>>(a);
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
  if (!(reg_check(a.cut_ptr, (a.N + 1) * 4.0, "cut ptr") & reg_check(a.E, (double)a.nnz * a.R * tb, "E") &
        reg_check(a.d, a.N * tb, "d") & reg_check(a.seed, a.seed ? a.R * tb : 0.0, "seed") &
        reg_check(a.gamma, NR * tb, "gamma") & reg_check(a.g_gamma, m0 ? NR * tb : 0.0, "g_gamma") &
        reg_check(a.m_gamma, m2 ? NR * tb : 0.0, "m_gamma") & reg_check(a.v_gamma, m2 ? NR * tb : 0.0, "v_gamma")))
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
                       (double)a.R * (a.csc.n_entries * sizeof(Td) + chunks(a.d) * 8.0);
  const double Rd = (double)a.R * a.d, yr = (a.y_per_spec ? (double)a.K : (double)a.R) * a.d, tb = sizeof(Td);
  if (!(reg_check(a.y, yr * 8.0, "cert y") & reg_check(a.yabs, yr * 4.0, "cert yabs") &
        reg_check(a.lo, a.d * 8.0, "lo") & reg_check(a.hi, a.d * 8.0, "hi") & reg_check(a.bias, a.d * 8.0, "bias") &
        reg_check(a.alpha, Rd * tb, "alpha") & reg_check(a.beta, (double)a.M * a.R * tb, "beta") &
        reg_check(a.gamma, (a.csc.n_total ? (double)a.N * a.R : 0.0) * tb, "gamma") & chk_splits(a.sp, a.R, a.K) &
        chk_csc(a.csc, a.d) & reg_check(a.nu_out, Rd * 8.0, "cert nu") &
        reg_check(a.obj_part, chunks(a.d) * a.R * 8.0, "cert part")))
    return;
  int tk = prof_begin(st, "certify_relax_f64", 0.0, bytes);
  k_certify_relax<Td><<<warp_blocks(a.R, a.d), kWarpsPerBlock * 32, 0, st>>>(a);
  prof_end(st, tk);
}
template <typename Td>
void certify_concretize(cudaStream_t st, int64_t R, int K, int N, int d0, const double* y0, const float* y0abs,
                        double gamma_n, const double* x_lo, const double* x_hi, const Td* gamma,
                        CutCSC<double> csc, double* obj_part) {
  if (R <= 0 || d0 <= 0) return;
  if (!(reg_check(y0, (double)R * d0 * 8.0, "cert y0") & reg_check(y0abs, (double)R * d0 * 4.0, "cert y0abs") &
        reg_check(x_lo, d0 * 8.0, "x_lo") & reg_check(x_hi, d0 * 8.0, "x_hi") & chk_csc(csc, d0) &
        reg_check(obj_part, chunks(d0) * R * 8.0, "cert part")))
    return;
  int tk = prof_begin(st, "certify_conc_f64", 0.0, (double)R * d0 * 12.0);
  k_certify_conc<Td><<<warp_blocks(R, d0), kWarpsPerBlock * 32, 0, st>>>(R, K, N, d0, y0, y0abs, gamma_n, x_lo, x_hi,
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

// Linear operators of the propagation chain (SIMT versions).
//
// Backward step of Theorem 3.1:  y^(i-1) = W^(i)^T nu^(i)   (dense: gemm_nt with
//   B = W^(i)^T stored [d_{i-1}, d_i]; conv: conv_T, the transposed convolution).
// Reverse-mode step (adjoint):  nubar^(i) = W^(i) a        (dense: gemm_nt with
//   B = W^(i) stored [d_i, d_{i-1}]; conv: conv_fwd).
// Certification: the same products in float64 plus sum |W||nu| rounded up, the
//   quantity in Higham's bound |fl(y) - y| <= gamma_n * sum |W||nu|.
#include <cstdio>

#include "gcp_internal.cuh"

namespace gcp {

namespace {

template <typename Tacc, typename Tin>
__device__ __forceinline__ Tacc load_as(const Tin* p) { return static_cast<Tacc>(*p); }
template <>
__device__ __forceinline__ float load_as<float, __nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }

constexpr int BM = 64, BN = 64, BK = 16;

// 64x64 output tile per 256-thread block; each thread owns rows ty+16i, cols tx+16j.
template <typename Tin, typename Tacc, bool ABS>
__global__ void __launch_bounds__(256) k_gemm_nt(int64_t M, int N, int K, const Tin* __restrict__ A, int a_mod,
                                                 const Tin* __restrict__ B, Tacc* __restrict__ C,
                                                 float* __restrict__ Cabs) {
  __shared__ Tacc As[BK][BM + 1];
  __shared__ Tacc Bs[BK][BN + 1];
  __shared__ float Aa[ABS ? BK : 1][ABS ? BM + 1 : 1];
  __shared__ float Ba[ABS ? BK : 1][ABS ? BN + 1 : 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.y * BM;
  const int n0 = blockIdx.x * BN;
  Tacc acc[4][4];
  float aacc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { acc[i][j] = Tacc(0); aacc[i][j] = 0.f; }
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int idx = tid + 256 * q, row = idx >> 4, kk = idx & 15;
      int64_t gm = m0 + row;
      int gk = k0 + kk;
      Tacc va = Tacc(0), vb = Tacc(0);
      if (gm < M && gk < K) {
        int64_t ar = a_mod ? (gm % a_mod) : gm;
        va = load_as<Tacc>(A + ar * K + gk);
      }
      int gn = n0 + row;
      if (gn < N && gk < K) vb = load_as<Tacc>(B + (int64_t)gn * K + gk);
      As[kk][row] = va;
      Bs[kk][row] = vb;
      if constexpr (ABS) {
        Aa[kk][row] = __double2float_ru(fabs((double)va));
        Ba[kk][row] = __double2float_ru(fabs((double)vb));
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Tacc a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      if constexpr (ABS) {
        float aa[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) aa[i] = Aa[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = Ba[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) aacc[i][j] = __fmaf_ru(aa[i], bb[j], aacc[i][j]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn < N) {
        C[gm * N + gn] = acc[i][j];
        if constexpr (ABS) Cabs[gm * N + gn] = aacc[i][j];
      }
    }
  }
}

// out[r,o,oh,ow] = sum_{c,kh,kw} W[o,c,kh,kw] in[r,c,oh*s+kh-p,ow*s+kw-p], each
// thread computing kConvFT output channels of one output pixel (every source
// value it loads serves all of them).
constexpr int kConvFT = 4;
template <typename Tin, typename Tacc>
__global__ void __launch_bounds__(256) k_conv_fwd_tile(int64_t R, LayerGeom g, const Tin* __restrict__ W,
                                                       const Tin* __restrict__ in, Tacc* __restrict__ out) {
  const int HWo = g.h_out * g.w_out, ckk = g.c_in * g.k * g.k;
  const int nct = (g.c_out + kConvFT - 1) / kConvFT;
  const int64_t n = R * (int64_t)nct * HWo;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / ((int64_t)nct * HWo);
    const int rem = (int)(idx - r * nct * HWo);
    const int o0 = (rem / HWo) * kConvFT;
    const int p2 = rem - (o0 / kConvFT) * HWo;
    const int oh = p2 / g.w_out, ow = p2 - oh * g.w_out;
    const Tin* ir = in + r * g.d_in;
    Tacc acc[kConvFT];
#pragma unroll
    for (int t = 0; t < kConvFT; ++t) acc[t] = Tacc(0);
    for (int c = 0; c < g.c_in; ++c)
      for (int kh = 0; kh < g.k; ++kh) {
        const int ih = oh * g.stride + kh - g.pad;
        if (ih < 0 || ih >= g.h_in) continue;
        for (int kw = 0; kw < g.k; ++kw) {
          const int iw = ow * g.stride + kw - g.pad;
          if (iw < 0 || iw >= g.w_in) continue;
          const Tacc v = load_as<Tacc>(ir + (c * g.h_in + ih) * g.w_in + iw);
#pragma unroll
          for (int t = 0; t < kConvFT; ++t) {
            const int o = o0 + t < g.c_out ? o0 + t : g.c_out - 1;   // a valid address; not stored
            acc[t] = fma(load_as<Tacc>(W + (size_t)o * ckk + (c * g.k + kh) * g.k + kw), v, acc[t]);
          }
        }
      }
    Tacc* orow = out + r * g.d_out + p2;
#pragma unroll
    for (int t = 0; t < kConvFT; ++t)
      if (o0 + t < g.c_out) orow[(int64_t)(o0 + t) * HWo] = acc[t];
  }
}


// out[r,c,ih,iw] = sum over the taps (kh,kw) that reach (ih,iw) and over the
// channels o of W[o,c,kh,kw] in[r,o,(ih+p-kh)/s,(iw+p-kw)/s]. Threads run in
// the order row, channel, then output pixels phase by phase: pixels with the
// same ih mod s and iw mod s are reached by the same taps, so the threads of a
// warp run the same taps. ABS: also sum |W||in| in float rounding up, from
// |W| and |in| given in float rounded up.
template <typename Tin, typename Tacc, bool ABS>
__global__ void k_conv_T(int64_t R, LayerGeom g, const Tin* __restrict__ W, const Tin* __restrict__ in,
                         Tacc* __restrict__ out, const float* __restrict__ Wabs, const float* __restrict__ inabs,
                         float* __restrict__ outabs) {
  const int s = g.stride, HW = g.h_in * g.w_in, HWo = g.h_out * g.w_out, ckk = g.c_in * g.k * g.k;
  const int64_t n = R * (int64_t)g.d_in;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / g.d_in;
    const int rem = (int)(idx - r * g.d_in);
    const int c = rem / HW;
    int q = rem - c * HW;   // position in phase order
    int ph = 0, pw = 0, Wf = 1;
    for (int f = 0; f < s * s; ++f) {
      ph = f / s;
      pw = f - ph * s;
      const int Hf = ph < g.h_in ? (g.h_in - ph + s - 1) / s : 0;
      Wf = pw < g.w_in ? (g.w_in - pw + s - 1) / s : 0;
      if (q < Hf * Wf) break;
      q -= Hf * Wf;
    }
    const int ih = ph + s * (q / Wf), iw = pw + s * (q % Wf);
    const int rh = (ph + g.pad) % s, rw = (pw + g.pad) % s;
    const Tin* ir = in + r * g.d_out;
    const float* ia = ABS ? inabs + r * g.d_out : nullptr;
    Tacc acc = Tacc(0);
    float aacc = 0.f;
    for (int kh = rh; kh < g.k; kh += s) {
      const int th = ih + g.pad - kh;
      if (th < 0) break;   // larger kh only lower th
      const int oh = th / s;
      if (oh >= g.h_out) continue;
      for (int kw = rw; kw < g.k; kw += s) {
        const int tw = iw + g.pad - kw;
        if (tw < 0) break;
        const int ow = tw / s;
        if (ow >= g.w_out) continue;
        const int wo = (c * g.k + kh) * g.k + kw, xo = oh * g.w_out + ow;
        for (int o = 0; o < g.c_out; ++o) {
          acc = fma(load_as<Tacc>(W + o * ckk + wo), load_as<Tacc>(ir + o * HWo + xo), acc);
          if constexpr (ABS) aacc = __fmaf_ru(Wabs[o * ckk + wo], ia[o * HWo + xo], aacc);
        }
      }
    }
    const int64_t oi = r * g.d_in + c * HW + ih * g.w_in + iw;
    out[oi] = acc;
    if constexpr (ABS) outabs[oi] = aacc;
  }
}

// The same product with each thread computing kConvCT output channels of one
// output pixel: every source value it loads serves all of them, where the
// kernel above loads it once per output channel. The sums run over the taps
// and channels in the same order, so each output is the same number.
constexpr int kConvCT = 4;
template <typename Tin, typename Tacc>
__global__ void __launch_bounds__(256) k_conv_T_tile(int64_t R, LayerGeom g, const Tin* __restrict__ W,
                                                     const Tin* __restrict__ in, Tacc* __restrict__ out) {
  const int s = g.stride, HW = g.h_in * g.w_in, HWo = g.h_out * g.w_out, ckk = g.c_in * g.k * g.k;
  const int nct = (g.c_in + kConvCT - 1) / kConvCT;
  const int64_t n = R * (int64_t)nct * HW;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / ((int64_t)nct * HW);
    const int rem = (int)(idx - r * nct * HW);
    const int c0 = (rem / HW) * kConvCT;
    int q = rem - (c0 / kConvCT) * HW;   // position in phase order
    int ph = 0, pw = 0, Wf = 1;
    for (int f = 0; f < s * s; ++f) {
      ph = f / s;
      pw = f - ph * s;
      const int Hf = ph < g.h_in ? (g.h_in - ph + s - 1) / s : 0;
      Wf = pw < g.w_in ? (g.w_in - pw + s - 1) / s : 0;
      if (q < Hf * Wf) break;
      q -= Hf * Wf;
    }
    const int ih = ph + s * (q / Wf), iw = pw + s * (q % Wf);
    const int rh = (ph + g.pad) % s, rw = (pw + g.pad) % s;
    const Tin* ir = in + r * g.d_out;
    Tacc acc[kConvCT];
#pragma unroll
    for (int t = 0; t < kConvCT; ++t) acc[t] = Tacc(0);
    for (int kh = rh; kh < g.k; kh += s) {
      const int th = ih + g.pad - kh;
      if (th < 0) break;   // larger kh only lower th
      const int oh = th / s;
      if (oh >= g.h_out) continue;
      for (int kw = rw; kw < g.k; kw += s) {
        const int tw = iw + g.pad - kw;
        if (tw < 0) break;
        const int ow = tw / s;
        if (ow >= g.w_out) continue;
        const int xo = oh * g.w_out + ow;
        for (int o = 0; o < g.c_out; ++o) {
          const Tacc v = load_as<Tacc>(ir + o * HWo + xo);
#pragma unroll
          for (int t = 0; t < kConvCT; ++t) {
            const int c = c0 + t < g.c_in ? c0 + t : g.c_in - 1;   // a valid address; not stored
            acc[t] = fma(load_as<Tacc>(W + o * ckk + (c * g.k + kh) * g.k + kw), v, acc[t]);
          }
        }
      }
    }
    Tacc* orow = out + r * g.d_in + ih * g.w_in + iw;
#pragma unroll
    for (int t = 0; t < kConvCT; ++t)
      if (c0 + t < g.c_in) orow[(int64_t)(c0 + t) * HW] = acc[t];
  }
}

// Row-staged forms of the two SIMT convolutions: the weights staged in shared
// memory once per CTA, then one row at a time: the row's source map staged in
// shared memory (read once from global memory), then kConvCT / kConvFT output
// channels of one output pixel per work item, pixels fastest (a warp's pixels
// share a phase, hence their taps). The sums run in the same order as the
// kernels above, so every output is the same number.
template <typename Tin, typename Tacc>
__global__ void __launch_bounds__(256) k_conv_T_row(int64_t R, LayerGeom g, const Tin* __restrict__ W,
                                                    const Tin* __restrict__ in, Tacc* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char conv_sm[];
  Tacc* src = reinterpret_cast<Tacc*>(conv_sm);   // [d_out]
  Tacc* ws = src + g.d_out;                       // [c_out, c_in, k, k]
  const int s = g.stride, HW = g.h_in * g.w_in, HWo = g.h_out * g.w_out, ckk = g.c_in * g.k * g.k;
  const int nct = (g.c_in + kConvCT - 1) / kConvCT, items = nct * HW;
  for (int i = threadIdx.x; i < g.c_out * ckk; i += blockDim.x) ws[i] = load_as<Tacc>(W + i);
  for (int64_t r = blockIdx.x; r < R; r += gridDim.x) {
    __syncthreads();   // the previous row's items are done with src
    for (int i = threadIdx.x; i < g.d_out; i += blockDim.x) src[i] = load_as<Tacc>(in + r * g.d_out + i);
    __syncthreads();
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int c0 = (it / HW) * kConvCT;
      int q = it - (c0 / kConvCT) * HW;   // position in phase order
      int ph = 0, pw = 0, Wf = 1;
      for (int f = 0; f < s * s; ++f) {
        ph = f / s;
        pw = f - ph * s;
        const int Hf = ph < g.h_in ? (g.h_in - ph + s - 1) / s : 0;
        Wf = pw < g.w_in ? (g.w_in - pw + s - 1) / s : 0;
        if (q < Hf * Wf) break;
        q -= Hf * Wf;
      }
      const int ih = ph + s * (q / Wf), iw = pw + s * (q % Wf);
      const int rh = (ph + g.pad) % s, rw = (pw + g.pad) % s;
      Tacc acc[kConvCT];
#pragma unroll
      for (int t = 0; t < kConvCT; ++t) acc[t] = Tacc(0);
      for (int kh = rh; kh < g.k; kh += s) {
        const int th = ih + g.pad - kh;
        if (th < 0) break;
        const int oh = th / s;
        if (oh >= g.h_out) continue;
        for (int kw = rw; kw < g.k; kw += s) {
          const int tw = iw + g.pad - kw;
          if (tw < 0) break;
          const int ow = tw / s;
          if (ow >= g.w_out) continue;
          const int xo = oh * g.w_out + ow;
          for (int o = 0; o < g.c_out; ++o) {
            const Tacc v = src[o * HWo + xo];
#pragma unroll
            for (int t = 0; t < kConvCT; ++t) {
              const int c = c0 + t < g.c_in ? c0 + t : g.c_in - 1;   // a valid address; not stored
              acc[t] = fma(ws[o * ckk + (c * g.k + kh) * g.k + kw], v, acc[t]);
            }
          }
        }
      }
      Tacc* orow = out + r * g.d_in + ih * g.w_in + iw;
#pragma unroll
      for (int t = 0; t < kConvCT; ++t)
        if (c0 + t < g.c_in) orow[(int64_t)(c0 + t) * HW] = acc[t];
    }
  }
}

// Row staging of the float row kernels: with DB the next row's source map
// streams into a second buffer (16-byte cp.async) while the block computes
// on the current one; the row length is a multiple of 4 floats and the rows
// are 16-byte aligned (checked by the launcher).
__device__ __forceinline__ void row_async(float* dst, const float* src, int n) {
  for (int i = threadIdx.x * 4; i < n; i += blockDim.x * 4) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst + i);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src + i) : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void row_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
template <bool DB, typename Tin>
__device__ __forceinline__ float* row_stage(float* buf, const Tin* in, int64_t r, int64_t R, int n, int iter) {
  if constexpr (DB) {
    float* cur = buf + (iter & 1) * n;
    __syncthreads();   // the previous row's items are done with the other buffer
    const int64_t rn = r + gridDim.x;
    if (rn < R) row_async(buf + ((iter + 1) & 1) * n, reinterpret_cast<const float*>(in) + rn * n, n);
    else asm volatile("cp.async.commit_group;\n" ::: "memory");
    row_async_wait_prev();   // this row's copies (committed one iteration ago) are done
    __syncthreads();
    return cur;
  } else {
    __syncthreads();   // the previous row's items are done with buf
    for (int i = threadIdx.x; i < n; i += blockDim.x) buf[i] = load_as<float>(in + r * n + i);
    __syncthreads();
    return buf;
  }
}

// Float form of k_conv_T_row with TP output pixels per work item: adjacent
// pixels of one phase row (the same taps, source columns ow, ow + 1, ...)
// share each weight load, and the weights are staged as [c_out][k][k][4 * nct]
// so one 16-byte load gives a tile's four channels. Each output adds the same
// terms in the same order as k_conv_T_row (a skipped tap is a predicate), so
// every output is the same number. TP = 4 where there are several channel
// tiles and enough items (conv_pixels; the CNN's 64 -> 32-channel layer: 20%
// faster than TP = 2), 2 otherwise (its 3-channel input layer: 36% slower
// with TP = 4). Work items
// run channel tile fastest, as in k_conv_fwd_row2 (the 64 -> 32-channel layer
// of the FP32 chain 6.1 -> 5.2 ms per launch).
template <typename Tin, bool DB, int TP>
__global__ void __launch_bounds__(256) k_conv_T_row2(int64_t R, LayerGeom g, const Tin* __restrict__ W,
                                                     const Tin* __restrict__ in, float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char conv_sm[];
  const int s = g.stride, HW = g.h_in * g.w_in, HWo = g.h_out * g.w_out, kk = g.k * g.k;
  const int nct = (g.c_in + kConvCT - 1) / kConvCT, C4 = nct * kConvCT;
  float* ws = reinterpret_cast<float*>(conv_sm);   // [c_out][k][k][C4]
  float* src = ws + (size_t)g.c_out * kk * C4;     // [d_out], twice with DB
  for (int i = threadIdx.x; i < g.c_out * kk * C4; i += blockDim.x) {
    const int c = i % C4, tap = (i / C4) % kk, o = i / (C4 * kk);
    ws[i] = c < g.c_in ? load_as<float>(W + (int64_t)o * g.c_in * kk + c * kk + tap) : 0.f;
  }
  // work items per channel tile: every phase's rows in groups of TP pixels
  int per_tile = 0;
  for (int f = 0; f < s * s; ++f) {
    const int ph = f / s, pw = f - ph * s;
    const int Hf = ph < g.h_in ? (g.h_in - ph + s - 1) / s : 0, Wf = pw < g.w_in ? (g.w_in - pw + s - 1) / s : 0;
    per_tile += Hf * ((Wf + TP - 1) / TP);
  }
  const int items = nct * per_tile;
  if (DB && blockIdx.x < R) row_async(src, reinterpret_cast<const float*>(in) + blockIdx.x * (int64_t)g.d_out, g.d_out);
  int iter = 0;
  for (int64_t r = blockIdx.x; r < R; r += gridDim.x, ++iter) {
    const float* srcr = row_stage<DB>(src, in, r, R, g.d_out, iter);
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int ct = it % nct, c0 = ct * kConvCT;
      int q = it / nct;
      int ph = 0, pw = 0, Wf = 1, G = 1;
      for (int f = 0; f < s * s; ++f) {
        ph = f / s;
        pw = f - ph * s;
        const int Hf = ph < g.h_in ? (g.h_in - ph + s - 1) / s : 0;
        Wf = pw < g.w_in ? (g.w_in - pw + s - 1) / s : 0;
        G = (Wf + TP - 1) / TP;
        if (q < Hf * G) break;
        q -= Hf * G;
      }
      const int i = q / G, j0 = (q - i * G) * TP;
      const int ih = ph + s * i, iw0 = pw + s * j0;
      const int rh = (ph + g.pad) % s, rw = (pw + g.pad) % s;
      float acc[TP][kConvCT];
#pragma unroll
      for (int p = 0; p < TP; ++p)
#pragma unroll
        for (int t = 0; t < kConvCT; ++t) acc[p][t] = 0.f;
      for (int kh = rh; kh < g.k; kh += s) {
        const int th = ih + g.pad - kh;
        if (th < 0) break;
        const int oh = th / s;
        if (oh >= g.h_out) continue;
        for (int kw = rw; kw < g.k; kw += s) {
          // pixel p: iw = iw0 + s p, source column (iw + pad - kw) / s
          const int tw0 = iw0 + g.pad - kw;
          bool ok[TP];
          int xo[TP];
#pragma unroll
          for (int p = 0; p < TP; ++p) {
            const int tw = tw0 + s * p;
            ok[p] = j0 + p < Wf && tw >= 0 && tw / s < g.w_out;
            xo[p] = ok[p] ? oh * g.w_out + tw / s : 0;
          }
          const float* wt = ws + (kh * g.k + kw) * C4 + c0;
          for (int o = 0; o < g.c_out; ++o) {
            const float4 w4 = *reinterpret_cast<const float4*>(wt + (size_t)o * kk * C4);
            const float wv[kConvCT] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int p = 0; p < TP; ++p) {
              if (!ok[p]) continue;
              const float v = srcr[o * HWo + xo[p]];
#pragma unroll
              for (int t = 0; t < kConvCT; ++t) acc[p][t] = fmaf(wv[t], v, acc[p][t]);
            }
          }
        }
      }
#pragma unroll
      for (int p = 0; p < TP; ++p) {
        if (j0 + p >= Wf) continue;
        float* orow = out + r * g.d_in + ih * g.w_in + iw0 + s * p;
#pragma unroll
        for (int t = 0; t < kConvCT; ++t)
          if (c0 + t < g.c_in) orow[(int64_t)(c0 + t) * HW] = acc[p][t];
      }
    }
  }
}

template <typename Tin, typename Tacc>
__global__ void __launch_bounds__(256) k_conv_fwd_row(int64_t R, LayerGeom g, const Tin* __restrict__ W,
                                                      const Tin* __restrict__ in, Tacc* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char conv_sm[];
  Tacc* src = reinterpret_cast<Tacc*>(conv_sm);   // [d_in]
  Tacc* ws = src + g.d_in;                        // [c_out, c_in, k, k]
  const int HWo = g.h_out * g.w_out, ckk = g.c_in * g.k * g.k;
  const int nct = (g.c_out + kConvFT - 1) / kConvFT, items = nct * HWo;
  for (int i = threadIdx.x; i < g.c_out * ckk; i += blockDim.x) ws[i] = load_as<Tacc>(W + i);
  for (int64_t r = blockIdx.x; r < R; r += gridDim.x) {
    __syncthreads();
    for (int i = threadIdx.x; i < g.d_in; i += blockDim.x) src[i] = load_as<Tacc>(in + r * g.d_in + i);
    __syncthreads();
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int o0 = (it / HWo) * kConvFT;
      const int p2 = it - (o0 / kConvFT) * HWo;
      const int oh = p2 / g.w_out, ow = p2 - oh * g.w_out;
      Tacc acc[kConvFT];
#pragma unroll
      for (int t = 0; t < kConvFT; ++t) acc[t] = Tacc(0);
      for (int c = 0; c < g.c_in; ++c)
        for (int kh = 0; kh < g.k; ++kh) {
          const int ih = oh * g.stride + kh - g.pad;
          if (ih < 0 || ih >= g.h_in) continue;
          for (int kw = 0; kw < g.k; ++kw) {
            const int iw = ow * g.stride + kw - g.pad;
            if (iw < 0 || iw >= g.w_in) continue;
            const Tacc v = src[(c * g.h_in + ih) * g.w_in + iw];
#pragma unroll
            for (int t = 0; t < kConvFT; ++t) {
              const int o = o0 + t < g.c_out ? o0 + t : g.c_out - 1;   // a valid address; not stored
              acc[t] = fma(ws[o * ckk + (c * g.k + kh) * g.k + kw], v, acc[t]);
            }
          }
        }
      Tacc* orow = out + r * g.d_out + p2;
#pragma unroll
      for (int t = 0; t < kConvFT; ++t)
        if (o0 + t < g.c_out) orow[(int64_t)(o0 + t) * HWo] = acc[t];
    }
  }
}

// Float form of k_conv_fwd_row with FP adjacent output pixels (columns
// ow .. ow + FP - 1 of one output row) per work item sharing each weight
// load, the weights staged as [c_in][k][k][4 * nft] (one 16-byte load per tap
// gives a tile's four output channels). Work items run channel tile fastest:
// the lanes of a warp that share a pixel group read the same source words
// (broadcasts), where pixel groups fastest put up to eight lanes of a stride-2
// convolution on one shared-memory bank (CNN FP32 chain 1,825 -> 1,673 ms per
// step); with that ordering four pixels per item beat two (1,621 -> 1,554 ms)
// where a row still has an item for each of the block's threads
// (conv_pixels). KS = 3: the kernel size known at compile time and the tap
// loops unrolled (the CNN FP32 chain's forward products 3.8 -> 3.0 ms per
// launch; the BF16 chain's bf16-source input layer measured 8% slower, so it
// keeps the general loops). The same terms are added in the same order as
// k_conv_fwd_row, so every output is the same number.
template <typename Tin, bool DB, int FP, int KS>
__global__ void __launch_bounds__(256) k_conv_fwd_row2(int64_t R, LayerGeom g, const Tin* __restrict__ W,
                                                       const Tin* __restrict__ in, float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char conv_sm[];
  const int K = KS ? KS : g.k;
  constexpr int UK = KS ? KS : 1;
  const int HWo = g.h_out * g.w_out, kk = K * K;
  const int nft = (g.c_out + kConvFT - 1) / kConvFT, O4 = nft * kConvFT;
  float* ws = reinterpret_cast<float*>(conv_sm);   // [c_in][k][k][O4]
  float* src = ws + (size_t)g.c_in * kk * O4;      // [d_in], twice with DB
  for (int i = threadIdx.x; i < g.c_in * kk * O4; i += blockDim.x) {
    const int o = i % O4, tap = (i / O4) % kk, c = i / (O4 * kk);
    ws[i] = o < g.c_out ? load_as<float>(W + (int64_t)o * g.c_in * kk + c * kk + tap) : 0.f;
  }
  const int G = (g.w_out + FP - 1) / FP;   // pixel groups per output row
  const int per_tile = g.h_out * G, items = nft * per_tile;
  if (DB && blockIdx.x < R) row_async(src, reinterpret_cast<const float*>(in) + blockIdx.x * (int64_t)g.d_in, g.d_in);
  int iter = 0;
  for (int64_t r = blockIdx.x; r < R; r += gridDim.x, ++iter) {
    const float* srcr = row_stage<DB>(src, in, r, R, g.d_in, iter);
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int ft = it % nft, o0 = ft * kConvFT;
      const int q = it / nft, oh = q / G, ow0 = (q - oh * G) * FP;
      float acc[FP][kConvFT];
#pragma unroll
      for (int p = 0; p < FP; ++p)
#pragma unroll
        for (int t = 0; t < kConvFT; ++t) acc[p][t] = 0.f;
      for (int c = 0; c < g.c_in; ++c)
#pragma unroll UK
        for (int kh = 0; kh < K; ++kh) {
          const int ih = oh * g.stride + kh - g.pad;
          if (ih < 0 || ih >= g.h_in) continue;
          const float* srow = srcr + (c * g.h_in + ih) * g.w_in;
          const float* wt = ws + ((size_t)c * kk + kh * K) * O4 + o0;
#pragma unroll UK
          for (int kw = 0; kw < K; ++kw) {
            const float4 w4 = *reinterpret_cast<const float4*>(wt + kw * O4);
            const float wv[kConvFT] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int p = 0; p < FP; ++p) {
              const int iw = (ow0 + p) * g.stride + kw - g.pad;
              if (ow0 + p >= g.w_out || iw < 0 || iw >= g.w_in) continue;
              const float v = srow[iw];
#pragma unroll
              for (int t = 0; t < kConvFT; ++t) acc[p][t] = fmaf(wv[t], v, acc[p][t]);
            }
          }
        }
#pragma unroll
      for (int p = 0; p < FP; ++p) {
        if (ow0 + p >= g.w_out) continue;
        float* orow = out + r * g.d_out + oh * g.w_out + ow0 + p;
#pragma unroll
        for (int t = 0; t < kConvFT; ++t)
          if (o0 + t < g.c_out) orow[(int64_t)(o0 + t) * HWo] = acc[p][t];
      }
    }
  }
}

// Dynamic shared memory of a row-staged convolution, opted in once per kernel
// (false: the row does not fit; use the tiled kernel).
constexpr size_t kConvRowSmem = 112 * 1024;   // two blocks per SM
// The double-buffered float form only where it keeps three blocks per SM:
// the CNN input layer's transposed product, 1.93 -> 1.73 ms per launch; the
// FP32 chain's 64 -> 32-channel transposed convolution at two blocks per SM
// measured 4.8 -> 5.3 ms.
constexpr size_t kConvRowDbSmem = 75 * 1024;
template <typename Kern>
bool conv_row_smem(Kern kern, size_t bytes) {
  if (bytes > kConvRowSmem) return false;
  return smem_opt_in(reinterpret_cast<const void*>(kern), bytes);
}

// Pixels per work item of the row-staged float convolutions: four where the
// row's items at four pixels still cover the block's 256 threads (and, for a
// transposed product, the layer has several channel tiles), else two. The
// residual network's 16-channel 8x8 layers have 64 items per row at four
// pixels: with four, its FP32 chain measured 189 -> 224 ms per step; with one
// pixel per item (twice the items of two) 197 ms.
int conv_pixels(const LayerGeom& g, int dir) {
  constexpr int kThreads = 256;
  auto items = [&](int P) -> int64_t {
    if (dir == 0) return (int64_t)((g.c_out + kConvFT - 1) / kConvFT) * g.h_out * ((g.w_out + P - 1) / P);
    const int s = g.stride;
    int64_t per_tile = 0;
    for (int f = 0; f < s * s; ++f) {
      const int ph = f / s, pw = f - ph * s;
      const int Hf = ph < g.h_in ? (g.h_in - ph + s - 1) / s : 0, Wf = pw < g.w_in ? (g.w_in - pw + s - 1) / s : 0;
      per_tile += (int64_t)Hf * ((Wf + P - 1) / P);
    }
    return (int64_t)((g.c_in + kConvCT - 1) / kConvCT) * per_tile;
  };
  return items(4) >= kThreads && (dir == 0 || g.c_in > kConvCT) ? 4 : 2;
}

// Launch a row-staged float convolution with P = 2 or 4 pixels per item
// (false: its shared memory could not be opted in).
template <typename Tin, bool DB, int P, int KS>
bool fwd_row2_p(cudaStream_t st, unsigned nblk, size_t bytes, int64_t R, const LayerGeom& g, const Tin* W,
                const Tin* in, float* out) {
  if (!conv_row_smem(k_conv_fwd_row2<Tin, DB, P, KS>, bytes)) return false;
  k_conv_fwd_row2<Tin, DB, P, KS><<<nblk, 256, bytes, st>>>(R, g, W, in, out);
  return true;
}
template <typename Tin, bool DB>
bool fwd_row2(int P, cudaStream_t st, unsigned nblk, size_t bytes, int64_t R, const LayerGeom& g, const Tin* W,
              const Tin* in, float* out) {
  if (std::is_same<Tin, float>::value && g.k == 3)
    return P == 4 ? fwd_row2_p<Tin, DB, 4, 3>(st, nblk, bytes, R, g, W, in, out)
                  : fwd_row2_p<Tin, DB, 2, 3>(st, nblk, bytes, R, g, W, in, out);
  return P == 4 ? fwd_row2_p<Tin, DB, 4, 0>(st, nblk, bytes, R, g, W, in, out)
                : fwd_row2_p<Tin, DB, 2, 0>(st, nblk, bytes, R, g, W, in, out);
}
template <typename Tin, bool DB, int P>
bool T_row2_p(cudaStream_t st, unsigned nblk, size_t bytes, int64_t R, const LayerGeom& g, const Tin* W, const Tin* in,
              float* out) {
  if (!conv_row_smem(k_conv_T_row2<Tin, DB, P>, bytes)) return false;
  k_conv_T_row2<Tin, DB, P><<<nblk, 256, bytes, st>>>(R, g, W, in, out);
  return true;
}
template <typename Tin, bool DB>
bool T_row2(int P, cudaStream_t st, unsigned nblk, size_t bytes, int64_t R, const LayerGeom& g, const Tin* W,
            const Tin* in, float* out) {
  return P == 4 ? T_row2_p<Tin, DB, 4>(st, nblk, bytes, R, g, W, in, out)
                : T_row2_p<Tin, DB, 2>(st, nblk, bytes, R, g, W, in, out);
}

// The transposed 1x1 convolution without padding (a residual block's
// projection shortcut): out[r,c,ih,iw] = sum_o W[o,c] in[r,o,ih/s,iw/s] where s
// divides ih and iw (and ih/s, iw/s lie in the source map), else 0. One thread
// per output element in storage order, so the stores coalesce; the source row
// (c_out x h_out x w_out) is re-read from L1/L2 by the c_in output channels.
template <typename Tin, typename Tacc, bool ABS>
__global__ void __launch_bounds__(256) k_conv_T_1x1(int64_t R, LayerGeom g, const Tin* __restrict__ W,
                                                    const Tin* __restrict__ in, Tacc* __restrict__ out,
                                                    const float* __restrict__ Wabs, const float* __restrict__ inabs,
                                                    float* __restrict__ outabs) {
  const int s = g.stride, HW = g.h_in * g.w_in, HWo = g.h_out * g.w_out;
  const int64_t n = R * (int64_t)g.d_in;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / g.d_in;
    const int rem = (int)(idx - r * g.d_in);
    const int c = rem / HW, p = rem - c * HW;
    const int ih = p / g.w_in, iw = p - ih * g.w_in;
    const int oh = ih / s, ow = iw / s;
    Tacc acc = Tacc(0);
    float aacc = 0.f;
    if (ih == oh * s && iw == ow * s && oh < g.h_out && ow < g.w_out) {
      const Tin* ir = in + r * g.d_out + oh * g.w_out + ow;
      const float* ia = ABS ? inabs + r * g.d_out + oh * g.w_out + ow : nullptr;
      for (int o = 0; o < g.c_out; ++o) {
        acc = fma(load_as<Tacc>(W + o * g.c_in + c), load_as<Tacc>(ir + (int64_t)o * HWo), acc);
        if constexpr (ABS) aacc = __fmaf_ru(Wabs[o * g.c_in + c], ia[(int64_t)o * HWo], aacc);
      }
    }
    out[idx] = acc;
    if constexpr (ABS) outabs[idx] = aacc;
  }
}

template <typename T>
const char* tname();
template <>
const char* tname<double>() { return "f64"; }
template <>
const char* tname<float>() { return "f32"; }
template <>
const char* tname<__nv_bfloat16>() { return "bf16"; }

// multiply-adds of one row of a convolution (padding taps excluded)
double conv_macs(const LayerGeom& g) {
  auto taps = [&](int n_out, int n_in) {
    int64_t t = 0;
    for (int o = 0; o < n_out; ++o)
      for (int k = 0; k < g.k; ++k) {
        int i = o * g.stride + k - g.pad;
        t += (i >= 0 && i < n_in);
      }
    return (double)t;
  };
  return (double)g.c_out * g.c_in * taps(g.h_out, g.h_in) * taps(g.w_out, g.w_in);
}

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 64) b = 152 * 64;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

template <typename Tin, typename Tacc>
void gemm_nt(cudaStream_t st, int64_t M, int N, int K, const Tin* A, int a_mod, const Tin* B, Tacc* C) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((N + BN - 1) / BN, (unsigned)((M + BM - 1) / BM));
  char nm[32];
  snprintf(nm, sizeof nm, "gemm_simt_%s", tname<Tin>());
  const double arows = a_mod ? (double)a_mod : (double)M;
  if (!(reg_check(A, arows * K * sizeof(Tin), "gemm A") & reg_check(B, (double)N * K * sizeof(Tin), "gemm B") &
        reg_check(C, (double)M * N * sizeof(Tacc), "gemm C")))
    return;
  int tk = prof_begin(st, nm, 2.0 * M * N * K, (arows * K + (double)N * K) * sizeof(Tin) + (double)M * N * sizeof(Tacc));
  k_gemm_nt<Tin, Tacc, false><<<grid, 256, 0, st>>>(M, N, K, A, a_mod, B, C, nullptr);
  prof_end(st, tk);
}

void gemm_nt_abs(cudaStream_t st, int64_t M, int N, int K, const double* A, int a_mod, const double* B,
                 double* C, float* Cabs) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((N + BN - 1) / BN, (unsigned)((M + BM - 1) / BM));
  const double arows = a_mod ? (double)a_mod : (double)M;
  if (!(reg_check(A, arows * K * 8.0, "gemm A") & reg_check(B, (double)N * K * 8.0, "gemm B") &
        reg_check(C, (double)M * N * 8.0, "gemm C") & reg_check(Cabs, (double)M * N * 4.0, "gemm Cabs")))
    return;
  int tk = prof_begin(st, "gemm_simt_f64_certify", 2.0 * M * N * K, (arows * K + (double)N * K) * 8.0 + (double)M * N * 12.0);
  k_gemm_nt<double, double, true><<<grid, 256, 0, st>>>(M, N, K, A, a_mod, B, C, Cabs);
  prof_end(st, tk);
}

template <typename Tin, typename Tacc>
void conv_fwd(cudaStream_t st, int64_t R, const LayerGeom& g, const Tin* W, const Tin* in, Tacc* out) {
  int64_t n = R * (int64_t)g.d_out;
  if (n <= 0) return;
  const double nw = (double)g.c_out * g.c_in * g.k * g.k;
  if (!(reg_check(W, nw * sizeof(Tin), "conv W") & reg_check(in, (double)R * g.d_in * sizeof(Tin), "conv in") &
        reg_check(out, (double)R * g.d_out * sizeof(Tacc), "conv out")))
    return;
  char nm[32];
  snprintf(nm, sizeof nm, "conv_fwd_%s", tname<Tin>());
  int tk = prof_begin(st, nm, 2.0 * R * conv_macs(g), (double)R * (g.d_in * sizeof(Tin) + g.d_out * sizeof(Tacc)));
  const size_t row_bytes = ((size_t)g.d_in + (size_t)g.c_out * g.c_in * g.k * g.k) * sizeof(Tacc);
  const size_t wbytes = (size_t)g.c_in * g.k * g.k * (size_t)(((g.c_out + kConvFT - 1) / kConvFT) * kConvFT) * 4;
  const size_t row2_bytes = (size_t)g.d_in * 4 + wbytes, row2d_bytes = (size_t)g.d_in * 8 + wbytes;
  const unsigned nblk = (unsigned)std::min<int64_t>(R, 152 * 8);
  bool done = false;
  const int fp = conv_pixels(g, 0);
  if constexpr (std::is_same<Tin, float>::value && std::is_same<Tacc, float>::value) {
    if (g.d_in % 4 == 0 && ((uintptr_t)in & 15) == 0 && row2d_bytes <= kConvRowDbSmem)
      done = fwd_row2<float, true>(fp, st, nblk, row2d_bytes, R, g, W, in, out);
  }
  if (!done && std::is_same<Tacc, float>::value)
    done = fwd_row2<Tin, false>(fp, st, nblk, row2_bytes, R, g, W, in, reinterpret_cast<float*>(out));
  if (done) {
  } else if (conv_row_smem(k_conv_fwd_row<Tin, Tacc>, row_bytes))
    k_conv_fwd_row<Tin, Tacc><<<(unsigned)std::min<int64_t>(R, 152 * 8), 256, row_bytes, st>>>(R, g, W, in, out);
  else
    k_conv_fwd_tile<Tin, Tacc><<<grid_for(R * (int64_t)((g.c_out + kConvFT - 1) / kConvFT) * g.h_out * g.w_out, 256),
                                 256, 0, st>>>(R, g, W, in, out);
  prof_end(st, tk);
}

template <typename Tin, typename Tacc>
void conv_T(cudaStream_t st, int64_t R, const LayerGeom& g, const Tin* W, const Tin* in, Tacc* out) {
  int64_t n = R * (int64_t)g.d_in;
  if (n <= 0) return;
  const double nw = (double)g.c_out * g.c_in * g.k * g.k;
  if (!(reg_check(W, nw * sizeof(Tin), "convT W") & reg_check(in, (double)R * g.d_out * sizeof(Tin), "convT in") &
        reg_check(out, (double)R * g.d_in * sizeof(Tacc), "convT out")))
    return;
  char nm[32];
  snprintf(nm, sizeof nm, "conv_T_%s", tname<Tin>());
  int tk = prof_begin(st, nm, 2.0 * R * conv_macs(g), (double)R * (g.d_out * sizeof(Tin) + g.d_in * sizeof(Tacc)));
  const size_t wbytes = (size_t)g.c_out * g.k * g.k * (size_t)(((g.c_in + kConvCT - 1) / kConvCT) * kConvCT) * 4;
  const size_t row2_bytes = (size_t)g.d_out * 4 + wbytes, row2d_bytes = (size_t)g.d_out * 8 + wbytes;
  const unsigned nblk = (unsigned)std::min<int64_t>(R, 152 * 8);
  const int tp = conv_pixels(g, 1);
  bool done = false;
  const bool k1x1 = g.k == 1 && g.pad == 0;
  if constexpr (std::is_same<Tin, float>::value && std::is_same<Tacc, float>::value) {
    if (!k1x1 && g.d_out % 4 == 0 && ((uintptr_t)in & 15) == 0 && row2d_bytes <= kConvRowDbSmem)
      done = T_row2<float, true>(tp, st, nblk, row2d_bytes, R, g, W, in, out);
  }
  if (!done && !k1x1 && std::is_same<Tacc, float>::value)
    done = T_row2<Tin, false>(tp, st, nblk, row2_bytes, R, g, W, in, reinterpret_cast<float*>(out));
  if (done) {
  } else if (k1x1)
    k_conv_T_1x1<Tin, Tacc, false><<<grid_for(n, 256), 256, 0, st>>>(R, g, W, in, out, nullptr, nullptr, nullptr);
  else if (conv_row_smem(k_conv_T_row<Tin, Tacc>,
                         ((size_t)g.d_out + (size_t)g.c_out * g.c_in * g.k * g.k) * sizeof(Tacc)))
    k_conv_T_row<Tin, Tacc><<<(unsigned)std::min<int64_t>(R, 152 * 8), 256,
                              ((size_t)g.d_out + (size_t)g.c_out * g.c_in * g.k * g.k) * sizeof(Tacc), st>>>(
        R, g, W, in, out);
  else
    k_conv_T_tile<Tin, Tacc><<<grid_for(R * (int64_t)((g.c_in + kConvCT - 1) / kConvCT) * g.h_in * g.w_in, 256), 256, 0,
                               st>>>(R, g, W, in, out);
  prof_end(st, tk);
}

void conv_T_abs(cudaStream_t st, int64_t R, const LayerGeom& g, const double* W, const float* Wabs, const double* in,
                const float* inabs, double* out, float* outabs) {
  int64_t n = R * (int64_t)g.d_in;
  if (n <= 0) return;
  const double nw = (double)g.c_out * g.c_in * g.k * g.k;
  if (!(reg_check(W, nw * 8.0, "convT W") & reg_check(Wabs, nw * 4.0, "convT |W|") &
        reg_check(in, (double)R * g.d_out * 8.0, "convT in") & reg_check(inabs, (double)R * g.d_out * 4.0, "convT |in|") &
        reg_check(out, (double)R * g.d_in * 8.0, "convT out") & reg_check(outabs, (double)R * g.d_in * 4.0, "convT abs")))
    return;
  int tk = prof_begin(st, "conv_T_f64_certify", 2.0 * R * conv_macs(g), (double)R * (g.d_out * 12.0 + g.d_in * 12.0));
  if (g.k == 1 && g.pad == 0)
    k_conv_T_1x1<double, double, true><<<grid_for(n, 256), 256, 0, st>>>(R, g, W, in, out, Wabs, inabs, outabs);
  else
    k_conv_T<double, double, true><<<grid_for(n, 256), 256, 0, st>>>(R, g, W, in, out, Wabs, inabs, outabs);
  prof_end(st, tk);
}

// ---------------------------------------------------------------- skip connections
namespace {

// Elementwise over R x d, grid-stride; rows of y start at r * ld + off.
template <typename Ts, typename Td, bool CERT>
__global__ void __launch_bounds__(256) k_skip_add(int64_t R, int d, int ld, int off, const Ts* __restrict__ src,
                                                  const float* __restrict__ src_abs, int src_mod, Td* __restrict__ y,
                                                  float* __restrict__ yabs) {
  const int64_t n = R * d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / d;
    const int j = (int)(e - r * d);
    const int64_t rs = src_mod ? r % src_mod : r;
    const Td v = (Td)src[rs * d + j];
    const int64_t yi = r * ld + off + j;
    y[yi] += v;
    if constexpr (CERT)
      yabs[yi] = __fadd_ru(yabs[yi], src_abs ? src_abs[rs * d + j] : __double2float_ru(fabs((double)v)));
  }
}

// The same four elements at a time (float accumulation, widths, stride and
// offset multiples of 4, 16-byte aligned rows): 16-byte loads and stores.
__device__ __forceinline__ float4 load4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 load4(const __nv_bfloat16* p) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
template <typename Ts>
__global__ void __launch_bounds__(256) k_skip_add4(int64_t R, int d, int ld, int off, const Ts* __restrict__ src,
                                                   int src_mod, float* __restrict__ y) {
  const int d4 = d / 4;
  const int64_t n = R * d4;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / d4;
    const int j = 4 * (int)(e - r * d4);
    const int64_t rs = src_mod ? r % src_mod : r;
    const float4 v = load4(src + rs * d + j);
    float4* yp = reinterpret_cast<float4*>(y + r * ld + off + j);
    float4 a = *yp;
    a.x += v.x; a.y += v.y; a.z += v.z; a.w += v.w;
    *yp = a;
  }
}

}  // namespace

template <typename Ts, typename Td>
void skip_add(cudaStream_t st, int64_t R, int d, int ld, int off, const Ts* src, int src_mod, Td* y) {
  if (R <= 0 || d <= 0) return;
  const double srows = src_mod ? (double)src_mod : (double)R;
  if (off < 0 || off + d > ld)
    return (void)reg_check(nullptr, 1.0, "skip add: row window outside the destination");
  if (!(reg_check(src, srows * d * sizeof(Ts), "skip src") & reg_check(y, (double)R * ld * sizeof(Td), "skip y")))
    return;
  int tk = prof_begin(st, "skip_add", (double)R * d, (double)R * d * (sizeof(Ts) + 2 * sizeof(Td)));
  if constexpr (std::is_same<Td, float>::value) {
    if (d % 4 == 0 && ld % 4 == 0 && off % 4 == 0 && ((uintptr_t)y & 15) == 0 &&
        ((uintptr_t)src & (4 * sizeof(Ts) - 1)) == 0) {
      k_skip_add4<Ts><<<grid_for(R * (d / 4), 256), 256, 0, st>>>(R, d, ld, off, src, src_mod, y);
      prof_end(st, tk);
      return;
    }
  }
  k_skip_add<Ts, Td, false><<<grid_for(R * d, 256), 256, 0, st>>>(R, d, ld, off, src, nullptr, src_mod, y, nullptr);
  prof_end(st, tk);
}

void skip_add_cert(cudaStream_t st, int64_t R, int d, int ld, int off, const double* src, const float* src_abs,
                   int src_mod, double* y, float* yabs) {
  if (R <= 0 || d <= 0) return;
  const double srows = src_mod ? (double)src_mod : (double)R;
  if (off < 0 || off + d > ld)
    return (void)reg_check(nullptr, 1.0, "skip add: row window outside the destination");
  if (!(reg_check(src, srows * d * 8.0, "skip src") & reg_check(src_abs, src_abs ? srows * d * 4.0 : 0.0, "skip src abs") &
        reg_check(y, (double)R * ld * 8.0, "skip y") & reg_check(yabs, (double)R * ld * 4.0, "skip yabs")))
    return;
  int tk = prof_begin(st, "skip_add_certify", (double)R * d, (double)R * d * 24.0);
  k_skip_add<double, double, true><<<grid_for(R * d, 256), 256, 0, st>>>(R, d, ld, off, src, src_abs, src_mod, y,
                                                                            yabs);
  prof_end(st, tk);
}

// ---------------------------------------------------------------- branch and bound warm start
namespace {
__global__ void __launch_bounds__(128) k_bab_warm(int64_t R, int n_layers, const int* __restrict__ dims,
                                                  float* const* __restrict__ alpha, float* __restrict__ beta, int M,
                                                  float* __restrict__ gamma, int N, const WarmSrc* __restrict__ src) {
  for (int64_t r = blockIdx.x; r < R; r += gridDim.x) {
    const WarmSrc w = src[r];
    if (!w.alpha) continue;
    int64_t off = 0;
    for (int l = 0; l < n_layers; ++l) {
      const int d = dims[l];
      float* dst = alpha[l] + r * d;
      for (int j = threadIdx.x; j < d; j += blockDim.x) dst[j] = w.alpha[off + j];
      off += d;
    }
    for (int m = threadIdx.x; m < M; m += blockDim.x) beta[r * M + m] = m < w.np ? w.beta[m] : 0.f;
    for (int e = threadIdx.x; e < N; e += blockDim.x) gamma[r * N + e] = w.gamma[e];
  }
}
}  // namespace

void bab_warm_start(cudaStream_t st, int64_t R, int n_layers, const int* dims_dev, float* const* alpha_dev, int64_t na,
                    float* beta, int M, float* gamma, int N, const WarmSrc* src) {
  if (R <= 0) return;
  if (!(reg_check(dims_dev, n_layers * 4.0, "warm dims") & reg_check(alpha_dev, n_layers * 8.0, "warm alpha ptrs") &
        reg_check(beta, (double)R * M * 4.0, "warm beta") & reg_check(gamma, (double)R * N * 4.0, "warm gamma") &
        reg_check(src, (double)R * sizeof(WarmSrc), "warm sources")))
    return;
  int tk = prof_begin(st, "bab_warm_start", 0.0, (double)R * (na + M + N) * 8.0);
  k_bab_warm<<<(unsigned)std::min<int64_t>(R, 152 * 16), 128, 0, st>>>(R, n_layers, dims_dev, alpha_dev, beta, M,
                                                                        gamma, N, src);
  prof_end(st, tk);
}

// ---------------------------------------------------------------- branch and bound: branching score
namespace {
// a beats b: larger score, then lower layer, then lower index
__device__ __forceinline__ bool score_better(float sa, int la, int ja, float sb, int lb, int jb) {
  if (sa != sb) return sa > sb;
  if (la != lb) return la < lb;
  return ja < jb;
}
constexpr int kScoreThreads = 256;
__global__ void __launch_bounds__(kScoreThreads) k_bab_score(int S, int K, int n_layers,
                                                             const ScoreLayer* __restrict__ layers,
                                                             const int32_t* __restrict__ sp_tab, int M,
                                                             int32_t* __restrict__ picks) {
  __shared__ int32_t codes[kMaxSplits];
  __shared__ float ws[kScoreThreads / 32];
  __shared__ int wl[kScoreThreads / 32], wj[kScoreThreads / 32];
  for (int q = blockIdx.x; q < S; q += gridDim.x) {
    const int nm = M < kMaxSplits ? M : kMaxSplits;
    __syncthreads();
    for (int m = threadIdx.x; m < nm; m += blockDim.x) codes[m] = sp_tab[(int64_t)q * M + m];
    __syncthreads();
    float best = 0.f;
    int bl = 1 << 30, bj = 1 << 30;
    for (int l = 0; l < n_layers; ++l) {
      const ScoreLayer L = layers[l];
      for (int j = threadIdx.x; j < L.d; j += blockDim.x) {
        const float lo = L.lo[j], hi = L.hi[j];
        if (!(lo < 0.f && hi > 0.f)) continue;
        bool split = false;
        for (int m = 0; m < nm; ++m) {
          const int c = codes[m];
          split |= c >= 0 && (c >> 24) == L.layer && (c & 0x7fffff) == j;
        }
        if (split) continue;
        float cs = 0.f;
        for (int k = 0; k < K; ++k) cs += fmaxf(L.nuhat[((int64_t)q * K + k) * L.d + j], 0.f);
        const float sc = (-lo * hi / (hi - lo)) * cs;
        if (sc > 0.f && score_better(sc, L.layer, j, best, bl, bj)) {
          best = sc;
          bl = L.layer;
          bj = j;
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float s2 = __shfl_down_sync(0xffffffffu, best, o);
      const int l2 = __shfl_down_sync(0xffffffffu, bl, o), j2 = __shfl_down_sync(0xffffffffu, bj, o);
      if (score_better(s2, l2, j2, best, bl, bj)) {
        best = s2;
        bl = l2;
        bj = j2;
      }
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
      ws[w] = best;
      wl[w] = bl;
      wj[w] = bj;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int v = 1; v < kScoreThreads / 32; ++v)
        if (score_better(ws[v], wl[v], wj[v], best, bl, bj)) {
          best = ws[v];
          bl = wl[v];
          bj = wj[v];
        }
      picks[q] = best > 0.f ? (bl << 24) | bj : -1;
    }
  }
}
}  // namespace

void bab_branch_score(cudaStream_t st, int S, int K, int n_layers, const ScoreLayer* layers_dev,
                      const int32_t* sp_tab, int M, int32_t* picks) {
  if (S <= 0) return;
  if (!(reg_check(layers_dev, n_layers * (double)sizeof(ScoreLayer), "score layers") &
        reg_check(sp_tab, (double)S * (M > 0 ? M : 1) * 4.0, "split table") & reg_check(picks, S * 4.0, "picks")))
    return;
  int tk = prof_begin(st, "bab_branch_score", 0.0, 0.0);
  k_bab_score<<<(unsigned)std::min(S, 152 * 8), kScoreThreads, 0, st>>>(S, K, n_layers, layers_dev, sp_tab, M,
                                                                         picks);
  prof_end(st, tk);
}

template void skip_add<double, double>(cudaStream_t, int64_t, int, int, int, const double*, int, double*);
template void skip_add<float, float>(cudaStream_t, int64_t, int, int, int, const float*, int, float*);
template void skip_add<__nv_bfloat16, float>(cudaStream_t, int64_t, int, int, int, const __nv_bfloat16*, int, float*);

template void gemm_nt<double, double>(cudaStream_t, int64_t, int, int, const double*, int, const double*, double*);
template void gemm_nt<float, float>(cudaStream_t, int64_t, int, int, const float*, int, const float*, float*);
template void gemm_nt<__nv_bfloat16, float>(cudaStream_t, int64_t, int, int, const __nv_bfloat16*, int,
                                            const __nv_bfloat16*, float*);
template void conv_fwd<double, double>(cudaStream_t, int64_t, const LayerGeom&, const double*, const double*, double*);
template void conv_fwd<float, float>(cudaStream_t, int64_t, const LayerGeom&, const float*, const float*, float*);
template void conv_fwd<__nv_bfloat16, float>(cudaStream_t, int64_t, const LayerGeom&, const __nv_bfloat16*,
                                             const __nv_bfloat16*, float*);
template void conv_T<double, double>(cudaStream_t, int64_t, const LayerGeom&, const double*, const double*, double*);
template void conv_T<float, float>(cudaStream_t, int64_t, const LayerGeom&, const float*, const float*, float*);
template void conv_T<__nv_bfloat16, float>(cudaStream_t, int64_t, const LayerGeom&, const __nv_bfloat16*,
                                           const __nv_bfloat16*, float*);

}  // namespace gcp

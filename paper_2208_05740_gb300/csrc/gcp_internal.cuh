// Internal declarations shared by the libgcp translation units.
//
// Data layout on the device (R rows = subdomains x spec rows, r = s*K + k):
//   chain operands nu / a          [R, d_i]  row-major, operand dtype
//   GEMM outputs y / nubar         [R, d_i]  row-major, epilogue dtype T
//   alpha^(i), nuhat^(i)           [R, d_i]  row-major, T
//   beta                           [R, M]    (split slot m of the row's subdomain)
//   gamma                          [R, N]
//   E (cut-entry values)           [R, nnz]  entries in CSC (layer, neuron, kind) order
//   objective partials             [P, R]
// A warp of the per-neuron kernels handles 32 consecutive neurons of one row,
// so dense arrays move whole lines and the sparse cut gathers of a warp stay
// inside that row's gamma / E vectors.
#pragma once

#include <vector>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

#include "../../include/gcp.h"

namespace gcp {

constexpr int kMaxSplits = 64;     // per subdomain (validated on the host)
constexpr int kChunk = 32;         // neurons per warp step of the per-neuron kernels

struct LayerGeom {
  int kind, d_in, d_out;
  int c_in, h_in, w_in, c_out, h_out, w_out, k, stride, pad;
};
// The mixed-precision chain's backward products run on three bf16 terms,
// nu_hi W_hi + nu_lo W_hi + nu_hi W_lo (hi = bf16(x), lo = bf16(x - hi)), in
// one tensor-core product with float accumulation. Dense layers concatenate
// them along K: operand [nu_hi | nu_lo | nu_hi] against [W_hi | W_hi | W_lo]
// (kDenseTerms planes). Convolutions stage the operand as twice the source
// channels, [nu_hi | nu_lo] (kConvTerms planes), multiply each A block by
// [W_hi | W_hi] and, as a second weight operand, by [W_lo | 0].
constexpr int kDenseTerms = 3, kConvTerms = 2;
constexpr int kMaxTerms = 3;
// The geometry whose transposed product takes the convolution's operand:
// output channels (the transposed product's source channels) times kConvTerms.
inline LayerGeom split_geom(LayerGeom g) {
  g.c_out *= kConvTerms;
  g.d_out *= kConvTerms;
  return g;
}

// Cut entries of one layer in CSC order (per neuron), pointers already offset.
template <typename T>
struct CutCSC {
  const int32_t* ptr;   // [d+1] global entry offsets
  const int32_t* cut;   // cut id per entry
  const int8_t* kind;   // GCP_VAR_*
  const T* coef;
  const int32_t* eid;   // CSR position of the entry
  const int32_t* nrn;   // neuron index of the entry within its layer
  int64_t n_entries;    // entries of this layer (host-side accounting only)
  int64_t n_total;      // entries of all layers (host-side validation only)
  int max_span4;        // entries of this layer's fullest 128-neuron span (host-side launch choice only)
};

struct SplitsDev {
  const int32_t* ptr;   // [S+1]
  const int16_t* layer;
  const int32_t* index;
  const int8_t* sign;
  int64_t n;            // total split entries (host-side validation only)
  const int32_t* tab;   // [S, M] split codes by slot, -1 = none (see split_code)
};
// Split code of one slot: layer << 24 | (sign > 0) << 23 | neuron index.
inline int32_t split_code_of(int layer, int index, int sign) {
  return (int32_t)(((uint32_t)layer << 24) | ((sign > 0 ? 1u : 0u) << 23) | (uint32_t)index);
}

// Optimiser step applied inside the adjoint epilogues / cut gather.
// mode 0: write gradients (no update); 1: projected gradient ascent; 2: Adam.
template <typename T>
struct StepArgs {
  int mode;
  T lr_a, lr_b, lr_g;
  T b1, b2, eps, c1, c2;  // Adam moments and bias corrections 1-b1^t, 1-b2^t
  T ic1, ic2;             // 1/c1, 1/c2
};

template <typename T, typename Top>
struct RelaxArgs {
  int64_t R;
  int K, d, layer;
  int M, N;             // split slots and cuts (extents of beta / gamma)
  const T* y;           // [R, d] or [K, d] when y_per_spec
  int y_per_spec;
  const T* lo;          // root bounds [d]
  const T* hi;
  const T* inv_ul;      // 1 / (hi - lo) of root-unstable neurons [d]
  const T* bias;        // b^(layer) [d]
  const T* alpha;       // [R, d]
  const T* beta;        // [R, M]
  const T* gamma;       // [R, N]
  SplitsDev sp;
  CutCSC<T> csc;
  Top* nu_out;          // [R, d]   (tf32-rounded high part when nu_lo is set)
  float* nu_lo;         // [R, d]   low part nu - nu_out for the 3-pass tf32 GEMM, or nullptr
  T* nuhat_out;         // [R, d]
  T* obj_part;          // [ceil(d/32), R]: one partial per row and neuron chunk
  // directly optimised ReLU duals pi = theta * [nuhat]_+ on unstable neurons
  // (nullptr: Lemma A.1's closed form); theta_init: use the closed form and
  // write the theta that reproduces it
  T* theta;             // [R, d]
  int theta_init;
  // Outputs of the mixed-precision chain (bf16 operands, T = float), each
  // written only where set: nu in T, for the products that stay on the SIMT
  // units and for identity skip connections (which would otherwise carry an
  // operand rounding into y^(m) unaveraged); and nu's multi-term operand, row
  // r = [hi | lo] (split_terms 2) or [hi | lo | hi] (3) with hi = bf16(nu) and
  // lo = bf16(nu - hi), for the tensor-core products (nu_out is then nullptr).
  T* nu_full;           // [R, d]
  Top* nu_split;        // [R, split_terms * d]
  int split_terms;
};

template <typename T, typename Top>
struct AdjArgs {
  int64_t R;
  int K, d, layer;
  int M, N;
  const T* nubar;       // [R, d]  (W^(i) a, bias not yet subtracted)
  const T* seed;        // per-row seed of the reverse pass, nullptr = 1
  const T* lo;
  const T* hi;
  const T* inv_ul;      // 1 / (hi - lo) of root-unstable neurons [d]
  const T* bias;
  T* alpha;             // [R, d], updated in place when mode != 0
  const T* gamma;       // [R, N]
  const T* nuhat;       // [R, d]
  SplitsDev sp;
  CutCSC<T> csc;
  Top* a_out;           // [R, d] dg/dnuhat (nullptr for the last hidden layer)
  float* a_lo;          // low part for the 3-pass tf32 GEMM, or nullptr
  T* E;                 // [R, nnz], entries in CSC order
  T* g_alpha;           // [R, d]  (mode 0)
  T* g_beta;            // [R, M]  dg/dbeta of the layer's splits (all modes; the gather steps beta)
  T* m_alpha; T* v_alpha;  // Adam state (mode 2)
  StepArgs<T> st;
  // directly optimised pi = theta * [nuhat]_+ (nullptr: closed form); theta
  // is stepped in place at alpha's rate when mode != 0, its gradient written
  // to g_theta in mode 0
  T* theta;             // [R, d]
  T* g_theta;           // [R, d] (mode 0, may be nullptr)
  T* m_theta; T* v_theta;  // Adam state (mode 2)
};

template <typename T, typename Top>
struct ConcArgs {
  int64_t R;
  int K, d0;
  int N;
  const T* y0;          // [R, d0]
  const T* x_lo;
  const T* x_hi;
  const T* gamma;
  const T* seed;
  CutCSC<T> csc;        // layer 0 entries (kind X only)
  Top* a0_out;          // [R, d0] = -seed * x*  (start of the reverse pass)
  float* a0_lo;         // low part for the 3-pass tf32 GEMM, or nullptr
  T* E;
  T* obj_part;          // [ceil(d0/32), R]
};

template <typename T>
struct FinalArgs {
  int64_t R;
  int K, N, P;
  const T* cb;          // [K]  c_k^T b^(L)
  const T* d;           // [N]
  const T* gamma;       // [R, N]
  const T* obj_part;    // [P, R]
  T* g;                 // [R]
};

template <typename T>
struct GatherArgs {
  int64_t R;
  int N;
  const int32_t* cut_ptr;  // [N+1] CSR by cut
  const int32_t* pos;      // [nnz] CSC position (column of E) of each CSR entry
  const T* E;              // [R, nnz], entries in CSC order
  const T* d;
  const T* seed;
  T* gamma;             // [R, N] updated when mode != 0
  T* g_gamma;           // [R, N] mode 0
  T* m_gamma; T* v_gamma;
  StepArgs<T> st;
  int64_t nnz;          // cut entries (host-side accounting only)
  int K;                // spec rows per subdomain
  const int32_t* cut_lo;  // [S] cuts the row's query owns: [cut_lo, cut_hi), or nullptr = all
  const int32_t* cut_hi;
  // beta step (modes 1 and 2): dg/dbeta from the adjoint, slots holding a split
  int M;
  const int32_t* sp_tab;  // [S, M] split codes, -1 = empty slot
  T* beta;                // [R, M]
  const T* g_beta;        // [R, M]
  T* m_beta; T* v_beta;
};

// Certification pass (float64, outward rounding). Td: dual storage type.
template <typename Td>
struct CertArgs {
  int64_t R;
  int K, d, layer;
  int M, N;
  const double* y;       // [R, d] or [K, d]
  const float* yabs;     // sum |W||nu| rounded up, same layout as y
  int y_per_spec;
  double gamma_n;        // Higham's gamma_n for the GEMM's reduction length
  const double* lo;
  const double* hi;
  const double* bias;
  const Td* alpha;
  const Td* beta;
  const Td* gamma;
  SplitsDev sp;
  CutCSC<double> csc;
  double* nu_out;        // [R, d]
  float* nuabs_out;      // [R, d] |nu| in float rounded up, or nullptr
  double* obj_part;      // [ceil(d/32), R] rounded-down partial sums
  const Td* theta;       // [R, d] pi = theta * [nuhat]_+ on unstable neurons, or nullptr (closed form)
};

// ---------------------------------------------------------------- programmatic dependent launch
// The per-iteration kernels are launched with programmatic stream
// serialization: a kernel may begin (its static setup: bounds, split tables,
// cut metadata, barriers, TMEM) while the previous kernel on the stream
// drains, and executes griddep_wait() before it reads anything an earlier
// kernel wrote or writes global memory. griddep_launch() at kernel start lets
// the next kernel begin launching.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<A&&>(args)...);
}

// ---------------------------------------------------------------- launch validation
// Every device allocation of the library is registered; before each launch the
// launcher checks, on the host, that each pointer argument lies inside a live
// allocation with room for the largest extent the kernel can touch. A launch
// that fails the check is skipped and the problem is recorded for the API
// call to report (GCP_EDEVICE), so a bad argument never reaches the GPU.
// Allocations are keyed by device: a pointer passes only on the device it was
// allocated on (the current device at the check). Caller-owned arrays that
// take part in one call are registered beside the library's allocations by
// token, so a caller pointer equal to (or inside) a library allocation never
// replaces or removes the library's own entry. Problems are recorded per
// host thread: each API call (and each serving worker) reads its own.
void reg_alloc(const void* p, size_t bytes);
void reg_free(const void* p);
uint64_t reg_foreign(const void* p, size_t bytes);   // returns a token for reg_unforeign
void reg_unforeign(uint64_t token);
bool reg_check(const void* p, double bytes, const char* what);
// first problem this thread recorded since it last asked (empty if none); clears it
std::string reg_take_error();
// first failed in-kernel index check since the last call (synchronises st)
std::string take_device_error(cudaStream_t st);

// ---------------------------------------------------------------- profiling
// Count a launch and, if its kernel is selected, bracket it with CUDA events.
int prof_begin(cudaStream_t st, const char* name, double flops, double bytes);
void prof_end(cudaStream_t st, int token);
// Times a launch of an idempotent kernel (one that recomputes its outputs
// from inputs it does not write) is issued: 2 while profiling with this
// kernel selected by gcp_profile_repeat, else 1.
int prof_repeats(const char* name);
// Opts kernel `kern` in to `bytes` of dynamic shared memory on the current
// device (once per kernel, device and size; kernels of the same type are told
// apart by their address). False if the runtime refuses.
bool smem_opt_in(const void* kern, size_t bytes);

// ---------------------------------------------------------------- launchers
// GEMM: C[M,N] = A[M,K] * B[N,K]^T, A row m read from row (a_mod ? m % a_mod : m).
template <typename Tin, typename Tacc>
void gemm_nt(cudaStream_t st, int64_t M, int N, int K, const Tin* A, int a_mod, const Tin* B, Tacc* C);
void gemm_nt_abs(cudaStream_t st, int64_t M, int N, int K, const double* A, int a_mod, const double* B,
                 double* C, float* Cabs);
template <typename Tin, typename Tacc>
void conv_fwd(cudaStream_t st, int64_t R, const LayerGeom& g, const Tin* W, const Tin* in, Tacc* out);
template <typename Tin, typename Tacc>
void conv_T(cudaStream_t st, int64_t R, const LayerGeom& g, const Tin* W, const Tin* in, Tacc* out);
// certification: y = W^T nu in float64 and sum |W||nu| in float rounded up,
// from |W| and |nu| given in float rounded up
void conv_T_abs(cudaStream_t st, int64_t R, const LayerGeom& g, const double* W, const float* Wabs, const double* in,
                const float* inabs, double* out, float* outabs);

// Skip connections: y[r, off + j] += src[r', j] for r < R, j < d, where
// r' = r % src_mod (src_mod > 0: one source row per spec row) or r; y rows
// have stride ld, source rows stride d.
template <typename Ts, typename Td>
void skip_add(cudaStream_t st, int64_t R, int d, int ld, int off, const Ts* src, int src_mod, Td* y);
// the same in the certification: float64 sum in round-to-nearest and the
// magnitude bound yabs += src_abs (or |src| where src_abs is null) in float
// rounded up
void skip_add_cert(cudaStream_t st, int64_t R, int d, int ld, int off, const double* src, const float* src_abs,
                   int src_mod, double* y, float* yabs);

// Branch and bound warm start: row r of a new batch copies its parent's row
// src[r] (alpha over the layer blocks alpha_dev[l] of width dims[l], beta
// slots below np, the rest 0, gamma); rows whose src.alpha is null keep the
// defaults.
struct WarmSrc {
  const float* alpha;   // [na] parent's row, layers concatenated
  const float* beta;    // parent's beta row (np valid slots)
  const float* gamma;   // [N]
  int np;
  int pad_;
};
void bab_warm_start(cudaStream_t st, int64_t R, int n_layers, const int* dims_dev, float* const* alpha_dev, int64_t na,
                    float* beta, int M, float* gamma, int N, const WarmSrc* src);
// Branching neuron of every subdomain from its current duals: over the
// root-unstable neurons the subdomain has not split, the largest
// w_j * sum_k [nuhat_j]_+ (rows k of the subdomain) with w_j = -l_j u_j / (u_j - l_j):
// the part of the bound that the triangle relaxation's intercept costs at
// neuron j (Lemma A.1 without cuts: pi* = u C / (u - l), h = l pi* = -w_j C with
// C = [nuhat]_+), which a split of j removes. Ties go to the lower layer, then
// the lower index. picks[s] = layer << 24 | index, or -1 when every score is 0.
struct ScoreLayer {
  const float* nuhat;   // [R, d] of the batch's last evaluation
  const float* lo;      // root bounds [d]
  const float* hi;
  int d, layer;
};
void bab_branch_score(cudaStream_t st, int S, int K, int n_layers, const ScoreLayer* layers_dev,
                      const int32_t* sp_tab, int M, int32_t* picks);

// tcgen05 GEMMs (k_tc.cu); false = shape or driver not supported, use SIMT.
// B must not be written by kernels still in flight when the GEMM launches
// (the weights and their slices are static): its first tiles load before the
// programmatic dependency wait.
bool tc_available(int K, bool bf16);
// flop_scale scales the flops the profiler counts (1/3 for a product whose K
// is tripled by the three-term operands: the product is counted once)
bool gemm_tc_bf16(cudaStream_t st, int64_t M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C,
                  double flop_scale = 1.0);
// A plain fp32 (split into tf32 parts in the kernel); B given as tf32 high and low parts
bool gemm_tc_tf32x3(cudaStream_t st, int64_t M, int N, int K, const float* A, const float* B, const float* Blo,
                    float* C);
std::string take_tc_error(cudaStream_t st);

// Float64 product on the tensor cores by exact slices (the error-free
// transformation of Ozaki, Ogita, Oishi and Rump for matrix products). Each
// row of a float64 operand is scaled by 2^-e (e its largest magnitude's
// exponent) and cut into s slices of b bits, small integers stored exactly in
// bf16; the slice products are bf16 tensor-core GEMMs whose fp32 sums are
// exact integers (s * K * (2^b - 1)^2 < 2^22), and the slice pairs with
// i + j = t share one GEMM over K' = (t - 1) K (the slices of A in order along
// K, those of B in reverse order). The float64 result adds the terms
// 2^(e_r + f_c - b t) T_t from the smallest up; |result - exact| <=
// cerr * 2^(e_r + f_c) * K, written (rounded up) as the error scale beside
// the product.
struct SliceB {
  __nv_bfloat16* planes = nullptr;   // [N, s * K]: slice s .. 1 of each row
  int32_t* exps = nullptr;           // [N] row exponents (kSliceBadExp: not finite)
  int b = 0, s = 0;
  double cerr = 0.0;
};
constexpr int32_t kSliceBadExp = 1 << 30;
bool slice_params(int K, int& b, int& s, double& cerr);
// slices of the rows of A [M, K] (row stride K): planes [M, s * K], slice
// order 1 .. s, or s .. 1 with `reverse`
bool slice_rows(cudaStream_t st, int64_t M, int K, const double* A, int b, int s, bool reverse,
                __nv_bfloat16* planes, int32_t* exps);
// y [M, N] = A [M, K] * B^T in float64 with its error scale yabs; ap / ae / T
// are workspace: the slices of A ([M, s * K] bf16, [M] int32) and the s
// exact slice sums ([s, M, N] fp32)
bool gemm_f64_slices(cudaStream_t st, int64_t M, int N, int K, const double* A, const SliceB& B,
                     __nv_bfloat16* ap, int32_t* ae, float* T, double* y, float* yabs);

// Phase plan of the tensor-core convolution. dir 0 (out = conv(src)) is one
// phase: every output pixel, all k*k taps. dir 1 (out = conv^T(src), stride
// s) splits the output pixels into s*s phases (ph, pw): pixels ih = ph + s*i,
// iw = pw + s*j, reached only by the taps kh = rh + s*a, kw = rw + s*b with
// rh = (ph + pad) mod s, rw = (pw + pad) mod s, from source pixel
// ((ih + pad - kh) / s, (iw + pad - kw) / s). Phase f's weight columns are
// k-blocks kb0 .. kb0 + nkb - 1 of the packed weight: k = (kb0 * 64) +
// (a * nkw + b) * Csp + c, c the source channel (Csp = channels padded to 8).
constexpr int kMaxConvPhases = 16;
// Division by an invariant divisor d >= 1 for 0 <= n < 2^31: q = (t + n) >> s
// with t = high word of n * m, s = ceil(log2 d), m = floor(2^32 (2^s - d) / d)
// + 1 -- the round-up multiplier method of Granlund and Montgomery (1994)
// with its 33-bit multiplier 2^32 + m; t + n stays below 2^32 for n < 2^31.
struct FastDiv {
  uint32_t m = 1;
  int s = 0;
  FastDiv() = default;
  __host__ explicit FastDiv(uint32_t d) {
    while ((1ull << s) < d) ++s;
    m = static_cast<uint32_t>(((1ull << 32) * ((1ull << s) - d)) / d + 1);
  }
  __host__ __device__ int div(int n) const {
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(static_cast<uint32_t>(n), m);
#else
    const uint32_t t = static_cast<uint32_t>((static_cast<uint64_t>(static_cast<uint32_t>(n)) * m) >> 32);
#endif
    return static_cast<int>((t + static_cast<uint32_t>(n)) >> s);
  }
};

struct ConvPhase {
  int ph, pw, Hf, Wf;        // the phase's output pixels form an Hf x Wf grid
  int rh, rw, nkh, nkw;      // its taps
  int kb0, nkb;              // its weight k-blocks
  int tile0, ntiles;         // its 128-row GEMM tiles (set for a given batch by the launcher)
  FastDiv dPf, dWf;          // division by Hf * Wf and by Wf (set by the launcher)
};
struct ConvPlan {
  int dir, Cs, Hs, Ws, Csp;  // source map
  int Co, Ho, Wo;            // output map
  int k, stride, pad;
  int nph, Kp, Np;           // phases, packed weight [Np, Kp]
  FastDiv dS;                // division by the stride (set by the launcher)
  ConvPhase f[kMaxConvPhases];
};
__host__ __device__ inline bool conv_plan(const LayerGeom& g, int dir, ConvPlan& c) {
  c.dir = dir;
  c.k = g.k; c.stride = g.stride; c.pad = g.pad;
  if (dir == 0) {
    c.Cs = g.c_in; c.Hs = g.h_in; c.Ws = g.w_in; c.Co = g.c_out; c.Ho = g.h_out; c.Wo = g.w_out;
  } else {
    c.Cs = g.c_out; c.Hs = g.h_out; c.Ws = g.w_out; c.Co = g.c_in; c.Ho = g.h_in; c.Wo = g.w_in;
  }
  c.Csp = (c.Cs + 7) / 8 * 8;
  c.Np = (c.Co + 15) / 16 * 16;
  const int s = dir == 0 ? 1 : g.stride;
  if (g.k < 1 || g.stride < 1 || s * s > kMaxConvPhases) return false;
  c.nph = s * s;
  int kb = 0;
  for (int q = 0; q < c.nph; ++q) {
    ConvPhase& f = c.f[q];
    f.ph = q / s; f.pw = q % s;
    f.Hf = f.ph < c.Ho ? (c.Ho - f.ph + s - 1) / s : 0;
    f.Wf = f.pw < c.Wo ? (c.Wo - f.pw + s - 1) / s : 0;
    f.rh = (f.ph + g.pad) % s; f.rw = (f.pw + g.pad) % s;
    f.nkh = f.rh < g.k ? (g.k - f.rh + s - 1) / s : 0;
    f.nkw = f.rw < g.k ? (g.k - f.rw + s - 1) / s : 0;
    if (f.nkh * f.nkw == 0 && f.Hf * f.Wf > 0) return false;   // pixels no tap reaches
    f.kb0 = kb;
    f.nkb = (f.nkh * f.nkw * c.Csp + 63) / 64;
    kb += f.nkb;
  }
  c.Kp = kb * 64;
  return true;
}

// Convolution on the tensor cores (implicit GEMM, bf16 operands, fp32 out):
// dir 0 out = conv(src) [R, d_out], dir 1 out = conv^T(src) [R, d_in]. Wp is
// the weight packed for that direction's plan, [Np, Kp]. false = shape not
// supported (use the SIMT convolution). flop_scale as for gemm_tc_bf16.
constexpr int kConvMaxKb = 96;   // K blocks of 64 columns a plan may have with a second weight operand
// b2 (optional): a second weight operand that each A block is also
// multiplied by, the tiles of Wp2 [Np, 64 * nb2] listed per K block of the
// plan in map (-1: none); its products are added to the same accumulator.
struct ConvSecondB {
  const __nv_bfloat16* W = nullptr;
  int nb2 = 0;
  std::vector<int8_t> map;
};
bool conv_tc_bf16(cudaStream_t st, int64_t R, const LayerGeom& g, int dir, const __nv_bfloat16* Wp, int Kp, int Np,
                  const __nv_bfloat16* src, float* out, double flop_scale = 1.0, const ConvSecondB* b2 = nullptr);
// Whether conv_tc_bf16 takes this plan at any row count (its staging fits
// shared memory and its accumulators TMEM), with nb2 second-operand tiles.
bool conv_tc_fits(const LayerGeom& g, int dir, int Kp, int Np, int nb2 = 0);

template <typename T, typename Top>
void relax_eval(cudaStream_t st, const RelaxArgs<T, Top>& a);
template <typename T, typename Top>
void relax_adjoint(cudaStream_t st, const AdjArgs<T, Top>& a);
template <typename T, typename Top>
void concretize(cudaStream_t st, const ConcArgs<T, Top>& a);
template <typename T>
void finalize_bound(cudaStream_t st, const FinalArgs<T>& a);
template <typename T>
void gather_gamma(cudaStream_t st, const GatherArgs<T>& a);

template <typename Td>
void certify_relax(cudaStream_t st, const CertArgs<Td>& a);
template <typename Td>
void certify_concretize(cudaStream_t st, int64_t R, int K, int N, int d0, const double* y0, const float* y0abs,
                        double gamma_n, const double* x_lo, const double* x_hi, const Td* gamma,
                        CutCSC<double> csc, double* obj_part);
template <typename Td>
void certify_finalize(cudaStream_t st, int64_t R, int K, int N, int P, const double* C, const double* bL, int dL,
                      const double* d, const Td* gamma, const double* obj_part, double* out);

// layout helpers
template <typename Ts, typename Td>
void transpose_cast(cudaStream_t st, int64_t rows, int64_t cols, const Ts* src, Td* dst);  // dst[c,r] = src[r,c]
template <typename Ts, typename Td>
void cast_copy(cudaStream_t st, int64_t n, const Ts* src, Td* dst);
template <typename T>
void default_alpha(cudaStream_t st, int64_t R, int K, int d, int layer, const T* lo, const T* hi, SplitsDev sp,
                   T* alpha);

}  // namespace gcp

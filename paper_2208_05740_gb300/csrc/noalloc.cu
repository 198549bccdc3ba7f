// Bound evaluation that allocates no device memory.
//
// Some callers cannot call cudaMalloc: serving processes that reserve the
// whole GPU for their own memory pool up front, so that any further
// allocation fails, and latency-critical loops where the device-wide
// synchronisation of cudaMalloc and cudaFree is not acceptable. For them this
// file provides gcp_bound_dense_noalloc: the FP32 bound of dense ReLU
// networks without cuts or splits, every input and the output passed in by
// the caller, and the scratch of the chain kept in a fixed device array of
// this file.
#include <cstdint>
#include <mutex>
#include <vector>

#include "gcp_internal.cuh"

namespace gcp {
namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB, held by every GPU that loads the library

// File-scope scratch of the no-allocation entry point. Host code must not use
// this name as an address: the device address comes from cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
std::vector<void*> g_addr;  // device address of the scratch, per device

// Once per device, with that device current: look up the scratch address.
cudaError_t scratch_of(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if ((int)g_addr.size() <= dev) g_addr.resize(dev + 1, nullptr);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
    reg_alloc(p, kScratchBytes);  // let the launch checks see the scratch
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

// Caller arrays take part in the launch checks while the call enqueues work.
struct CallerArrays {
  std::vector<uint64_t> regs;
  bool add(const void* p, size_t bytes) {
    if (bytes == 0) return true;
    if (!p) return false;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      return false;
    }
    regs.push_back(reg_foreign(p, bytes));
    return true;
  }
  ~CallerArrays() {
    for (uint64_t t : regs) reg_unforeign(t);
  }
};

size_t up256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace
}  // namespace gcp

using namespace gcp;

extern "C" gcp_status gcp_bound_dense_noalloc(int32_t n_layers, const int32_t* dims, const float* const* WT,
                                              const float* const* bias, const float* const* lo,
                                              const float* const* hi, const float* const* alpha,
                                              const float* x_lo, const float* x_hi, const float* y_last,
                                              const float* cb, int32_t K, int64_t R, float* out, void* stream) {
  if (n_layers < 1 || !dims || K < 1 || R < 0 || R % K != 0) return GCP_EINVAL;
  if (n_layers > 1 && (!WT || !bias || !lo || !hi || !alpha)) return GCP_EINVAL;
  if (n_layers == 1 && R != K) return GCP_EINVAL;  // a linear network has one row per spec row
  const int L = n_layers;
  for (int i = 0; i <= L; ++i)
    if (dims[i] <= 0) return GCP_EINVAL;
  if (R == 0) return GCP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GCP_ECUDA;
  void* base = nullptr;
  if (scratch_of(dev, &base) != cudaSuccess) return GCP_ECUDA;

  // scratch layout: nu [R, dmax], y [R, dmax], nuhat [R, dmax], partials [P, R],
  // zero split offsets [S+1], zero cut offsets [dmax+1]
  int dmax = 1, P = 0;
  for (int i = 0; i < L; ++i) {
    dmax = dims[i] > dmax ? dims[i] : dmax;
    P += (dims[i] + kChunk - 1) / kChunk;
  }
  const int64_t S = R / K;
  const size_t b_mat = up256((size_t)R * dmax * 4), b_part = up256((size_t)P * R * 4);
  const size_t b_sp = up256((size_t)(S + 1) * 4), b_csc = up256((size_t)(dmax + 1) * 4);
  const size_t need = 3 * b_mat + b_part + b_sp + b_csc;
  if (need > kScratchBytes) return GCP_EBUDGET;
  char* p = static_cast<char*>(base);
  float* nu = reinterpret_cast<float*>(p);
  float* y = reinterpret_cast<float*>(p + b_mat);
  float* nuhat = reinterpret_cast<float*>(p + 2 * b_mat);
  float* part = reinterpret_cast<float*>(p + 3 * b_mat);
  int32_t* sp_ptr = reinterpret_cast<int32_t*>(p + 3 * b_mat + b_part);
  int32_t* csc_ptr = reinterpret_cast<int32_t*>(p + 3 * b_mat + b_part + b_sp);
  // no splits and no cuts: their offset arrays must read as zeros
  if (cudaMemsetAsync(sp_ptr, 0, b_sp + b_csc, st) != cudaSuccess) return GCP_ECUDA;

  CallerArrays ca;
  bool ok = ca.add(x_lo, (size_t)dims[0] * 4) && ca.add(x_hi, (size_t)dims[0] * 4) &&
            ca.add(y_last, (size_t)K * dims[L - 1] * 4) && ca.add(cb, (size_t)K * 4) && ca.add(out, (size_t)R * 4);
  for (int i = 1; i < L && ok; ++i)
    ok = ca.add(WT[i - 1], (size_t)dims[i - 1] * dims[i] * 4) && ca.add(bias[i - 1], (size_t)dims[i] * 4) &&
         ca.add(lo[i - 1], (size_t)dims[i] * 4) && ca.add(hi[i - 1], (size_t)dims[i] * 4) &&
         ca.add(alpha[i - 1], (size_t)R * dims[i] * 4);
  if (!ok) return GCP_EINVAL;

  SplitsDev sp{sp_ptr, nullptr, nullptr, nullptr, 0};
  int poff = 0;
  for (int i = L - 1; i >= 1; --i) {
    RelaxArgs<float, float> a{};
    a.R = R; a.K = K; a.d = dims[i]; a.layer = i; a.M = 0; a.N = 0;
    a.y = (i == L - 1) ? y_last : y;
    a.y_per_spec = (i == L - 1);
    a.lo = lo[i - 1]; a.hi = hi[i - 1]; a.bias = bias[i - 1];
    a.inv_ul = nullptr;   // divide in the kernel
    a.alpha = alpha[i - 1];
    a.sp = sp;
    a.csc = CutCSC<float>{csc_ptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, 0};
    a.nu_out = nu;
    a.nuhat_out = nuhat;
    a.obj_part = part + (int64_t)poff * R;
    relax_eval<float, float>(st, a);
    poff += (dims[i] + kChunk - 1) / kChunk;
    gemm_nt<float, float>(st, R, dims[i - 1], dims[i], nu, 0, WT[i - 1], y);
  }
  ConcArgs<float, float> c{};
  c.R = R; c.K = K; c.d0 = dims[0]; c.N = 0;
  c.y0 = (L == 1) ? y_last : y;
  c.x_lo = x_lo; c.x_hi = x_hi;
  c.csc = CutCSC<float>{csc_ptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, 0};
  c.obj_part = part + (int64_t)poff * R;
  concretize<float, float>(st, c);
  poff += (dims[0] + kChunk - 1) / kChunk;
  FinalArgs<float> fa{R, K, 0, poff, cb, nullptr, nullptr, part, out};
  finalize_bound<float>(st, fa);
  if (!reg_take_error().empty()) return GCP_EDEVICE;
  return cudaGetLastError() == cudaSuccess ? GCP_OK : GCP_ECUDA;
}

// Self-test of the chain's GEMM kernels on caller data (not a step of the
// method): C = A * B^T through the chosen kernel, host arrays in and out.
#include <cstring>
#include <vector>

#include "gcp_internal.cuh"

namespace {
float tf32_hi_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;
  u = (u + 0x1000u) & 0xffffe000u;
  float h;
  std::memcpy(&h, &u, 4);
  return h;
}
}  // namespace

using namespace gcp;

extern "C" gcp_status gcp_selftest_gemm(int32_t kind, int64_t M, int32_t N, int32_t K, const float* A, const float* B,
                                        float* C) {
  if (kind < 0 || kind > 2 || M <= 0 || N <= 0 || K <= 0 || !A || !B || !C) return GCP_EINVAL;
  const size_t na = (size_t)M * K, nb = (size_t)N * K, nc = (size_t)M * N;
  std::vector<void*> bufs;
  auto dalloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    reg_alloc(p, bytes);
    bufs.push_back(p);
    return p;
  };
  auto cleanup = [&]() {
    for (void* p : bufs) {
      reg_free(p);
      cudaFree(p);
    }
  };
  gcp_status st = GCP_OK;
  float* dC = (float*)dalloc(nc * 4);
  if (!dC) { cleanup(); return GCP_ENOMEM; }
  bool ran = false;
  if (kind == 0) {
    std::vector<__nv_bfloat16> ha(na), hb(nb);
    for (size_t i = 0; i < na; ++i) ha[i] = __float2bfloat16_rn(A[i]);
    for (size_t i = 0; i < nb; ++i) hb[i] = __float2bfloat16_rn(B[i]);
    auto* da = (__nv_bfloat16*)dalloc(na * 2);
    auto* db = (__nv_bfloat16*)dalloc(nb * 2);
    if (!da || !db) { cleanup(); return GCP_ENOMEM; }
    cudaMemcpy(da, ha.data(), na * 2, cudaMemcpyHostToDevice);
    cudaMemcpy(db, hb.data(), nb * 2, cudaMemcpyHostToDevice);
    ran = gemm_tc_bf16(nullptr, M, N, K, da, db, dC);
  } else if (kind == 1) {
    // A goes in as plain fp32 (the kernel splits it); B as tf32 high and low parts
    std::vector<float> bh(nb), bl(nb);
    for (size_t i = 0; i < nb; ++i) { bh[i] = tf32_hi_host(B[i]); bl[i] = B[i] - bh[i]; }
    float *da = (float*)dalloc(na * 4), *dbh = (float*)dalloc(nb * 4), *dbl = (float*)dalloc(nb * 4);
    if (!da || !dbh || !dbl) { cleanup(); return GCP_ENOMEM; }
    cudaMemcpy(da, A, na * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(dbh, bh.data(), nb * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(dbl, bl.data(), nb * 4, cudaMemcpyHostToDevice);
    ran = gemm_tc_tf32x3(nullptr, M, N, K, da, dbh, dbl, dC);
  } else {
    float *da = (float*)dalloc(na * 4), *db = (float*)dalloc(nb * 4);
    if (!da || !db) { cleanup(); return GCP_ENOMEM; }
    cudaMemcpy(da, A, na * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(db, B, nb * 4, cudaMemcpyHostToDevice);
    gemm_nt<float, float>(nullptr, M, N, K, da, 0, db, dC);
    ran = true;
  }
  if (!ran) st = GCP_EINVAL;
  if (!reg_take_error().empty()) st = GCP_EDEVICE;
  if (st == GCP_OK && cudaDeviceSynchronize() != cudaSuccess) st = GCP_ECUDA;
  if (st == GCP_OK && !take_tc_error(nullptr).empty()) st = GCP_EDEVICE;
  if (st == GCP_OK && cudaMemcpy(C, dC, nc * 4, cudaMemcpyDeviceToHost) != cudaSuccess) st = GCP_ECUDA;
  cleanup();
  return st;
}

extern "C" gcp_status gcp_selftest_gemm_f64(int64_t M, int32_t N, int32_t K, const double* A, const double* B,
                                            double* C, float* Cabs, double* cerr) {
  if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !C || !Cabs || !cerr) return GCP_EINVAL;
  SliceB sl;
  if (!slice_params(K, sl.b, sl.s, sl.cerr) || !tc_available(K, true)) return GCP_EINVAL;
  const size_t na = (size_t)M * K, nb = (size_t)N * K, nc = (size_t)M * N;
  std::vector<void*> bufs;
  auto dalloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    reg_alloc(p, bytes);
    bufs.push_back(p);
    return p;
  };
  auto cleanup = [&]() {
    for (void* p : bufs) {
      reg_free(p);
      cudaFree(p);
    }
  };
  double *da = (double*)dalloc(na * 8), *db = (double*)dalloc(nb * 8), *dc = (double*)dalloc(nc * 8);
  float* dca = (float*)dalloc(nc * 4);
  sl.planes = (__nv_bfloat16*)dalloc(nb * sl.s * 2);
  sl.exps = (int32_t*)dalloc((size_t)N * 4);
  auto* ap = (__nv_bfloat16*)dalloc(na * sl.s * 2);
  auto* ae = (int32_t*)dalloc((size_t)M * 4);
  auto* sums = (float*)dalloc(nc * sl.s * 4);
  if (!da || !db || !dc || !dca || !sl.planes || !sl.exps || !ap || !ae || !sums) { cleanup(); return GCP_ENOMEM; }
  cudaMemcpy(da, A, na * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(db, B, nb * 8, cudaMemcpyHostToDevice);
  gcp_status st = GCP_OK;
  slice_rows(nullptr, N, K, db, sl.b, sl.s, true, sl.planes, sl.exps);
  if (!gemm_f64_slices(nullptr, M, N, K, da, sl, ap, ae, sums, dc, dca)) st = GCP_EINVAL;
  if (!reg_take_error().empty()) st = GCP_EDEVICE;
  if (st == GCP_OK && cudaDeviceSynchronize() != cudaSuccess) st = GCP_ECUDA;
  if (st == GCP_OK && !take_tc_error(nullptr).empty()) st = GCP_EDEVICE;
  if (st == GCP_OK && cudaMemcpy(C, dc, nc * 8, cudaMemcpyDeviceToHost) != cudaSuccess) st = GCP_ECUDA;
  if (st == GCP_OK && cudaMemcpy(Cabs, dca, nc * 4, cudaMemcpyDeviceToHost) != cudaSuccess) st = GCP_ECUDA;
  if (st == GCP_OK) *cerr = sl.cerr;
  cleanup();
  return st;
}

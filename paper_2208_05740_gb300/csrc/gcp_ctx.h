// Host-side object model of a libgcp context: nets, cut sets, duals batches.
#pragma once

#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gcp_internal.cuh"

namespace gcp {

struct Ctx;

struct Net {
  Ctx* ctx = nullptr;
  int L = 0, K = 0;
  std::vector<int> dims;             // d_0 .. d_L
  std::vector<LayerGeom> geom;       // layer i at index i-1
  std::vector<double*> W64, WT64, b64;
  std::vector<float*> W32, WT32, b32;
  std::vector<__nv_bfloat16*> W16, WT16;
  std::vector<float*> W32hi, W32lo, WT32hi, WT32lo;  // tf32 split of the dense weights
  // convolution weights packed for the tensor-core implicit GEMM (bf16):
  // forward [cf_np, cf_kp] and transposed [ct_np, ct_kp]; nullptr for dense layers
  std::vector<__nv_bfloat16*> CF16, CT16;
  std::vector<float*> Wabs32;        // |W| in float rounded up (convolution layers; certification)
  std::vector<SliceB> WTsl;          // exact bf16 slices of W^T (dense layers; float64 certification)
  std::vector<int> cf_kp, cf_np, ct_kp, ct_np;
  // the mixed-precision chain's backward products with multi-term bf16
  // operands: dense layers [d_in, 3 d_out] = rows of [W_hi^T | W_hi^T | W_lo^T];
  // convolutions packed for the transposed plan of split_geom(g) (source
  // channels doubled): [W_hi | W_hi], and [W_lo | 0] as a second weight
  // operand over the same A blocks; nullptr where that product stays on the
  // SIMT units (with nu in float)
  std::vector<__nv_bfloat16*> WT16x3, CT16s;
  std::vector<int> cts_kp, cts_np;
  std::vector<ConvSecondB> CTs_b2;
  double *xlo64 = nullptr, *xhi64 = nullptr;
  float *xlo32 = nullptr, *xhi32 = nullptr;
  double *C64 = nullptr, *negC64 = nullptr, *bL64 = nullptr;
  double* YL64 = nullptr;            // [K, d_{L-1}] = -W^(L)^T c_k
  float* YL32 = nullptr;
  double* cb64 = nullptr;            // [K] = c_k^T b^(L)
  float* cb32 = nullptr;
  // skip connections: skip[i-1] = s >= 1 when layer i adds S xhat^(s-1);
  // consumer[m] = the layer that adds xhat^(m), or 0; sc_map[i-1] = the map
  // index (L+1, L+2, ... in geom and the weight vectors) of layer i's
  // projection S, 0 for the identity
  std::vector<int> skip, consumer, sc_map;
  int skip_off = 0;                  // the last layer's identity skip adds xhat^(m)[skip_off ..]
  // [K, d_m] = -S^T c_k of a skip on the last layer from xhat^(m), m < L-1
  // (from m = L-1 it is folded into YL)
  double* SK64 = nullptr;
  float* SK32 = nullptr;
  std::vector<double*> lo64, hi64;   // hidden layer i at index i-1
  std::vector<float*> lo32, hi32;    // rounded outwards
  std::vector<double*> invul64;      // 1 / (hi - lo) where lo < 0 < hi, else 0
  std::vector<std::vector<int32_t>> unstable;  // root-unstable neurons of hidden layer i at index i-1 (host)
  std::vector<float*> invul32;
  std::vector<void*> owned;
  ~Net();
};

struct CutSet {
  int net_id = 0;
  std::vector<int64_t> ptr;
  std::vector<int16_t> layer;
  std::vector<int8_t> kind;
  std::vector<int32_t> index;
  std::vector<double> coef, d;
};

struct CutDev {
  Ctx* ctx = nullptr;
  int N = 0;
  int64_t nnz = 0;
  int32_t* cut_ptr = nullptr;        // [N+1] CSR by cut (entry ids)
  double* d64 = nullptr;
  float* d32 = nullptr;
  int32_t* csc_ptr = nullptr;        // per layer segments of d_i + 1 offsets
  int32_t* csc_cut = nullptr;
  int8_t* csc_kind = nullptr;
  double* csc_coef64 = nullptr;
  float* csc_coef32 = nullptr;
  int32_t* csc_eid = nullptr;
  int32_t* csc_nrn = nullptr;
  int32_t* csr_pos = nullptr;        // CSC position of each CSR entry
  std::vector<int64_t> poff;         // segment start of layer i in csc_ptr
  std::vector<int64_t> layer_nnz;    // entries per layer
  std::vector<int32_t> span4_max;    // per layer: entries of the fullest 128-neuron span
  std::vector<void*> owned;
  bool pooled = false;               // blocks go back to the context's pool (serving batches)
  ~CutDev();
};

struct Batch {
  Ctx* ctx = nullptr;
  Net* net = nullptr;
  int net_id = 0;
  int S = 0, K = 0, M = 0, N = 0;
  int64_t R = 0, nnz = 0, nsp = 0;
  int parts = 1;                     // queries sharing this batch
  int32_t* sub_cut_lo = nullptr;     // [S] first cut of the subdomain's query (several parts only)
  int32_t* sub_cut_hi = nullptr;     // [S] end of the query's cuts
  bool fp64 = false;
  bool tc = true;                    // use the tcgen05 GEMMs where shapes allow
  // the adjoint recomputes each layer's nuhat from the top instead of reading
  // it stored by the evaluation (decided at the first adjoint evaluation)
  bool recompute = false, recompute_decided = false;
  // every evaluation keeps each layer's nuhat (as the adjoint's evaluations
  // do), for the branching score of branch and bound
  bool keep_nuhat = false;
  CutDev cuts;
  int32_t* sp_ptr = nullptr;
  int16_t* sp_layer = nullptr;
  int32_t* sp_index = nullptr;
  int8_t* sp_sign = nullptr;
  int32_t* sp_tab = nullptr;         // [S, max(M,1)] split codes by slot
  std::vector<void*> alpha;          // hidden layer i at index i-1, [R, d_i]
  void* beta = nullptr;              // [R, M]
  void* gamma = nullptr;             // [R, N]
  // the workspace "theta" holds directly optimised ReLU duals (pi = theta
  // [nuhat]_+) that every pass uses instead of the closed form
  bool theta_on = false;
  std::vector<void*> owned;
  std::map<std::string, void*> lazy; // workspace by name
  std::map<std::string, size_t> lazy_bytes;
  // serving batches: the one stream that uses this batch's memory; its blocks
  // go back to the context's pool once that stream has drained
  cudaStream_t pool_stream = nullptr;
  void* ws(const std::string& name, size_t bytes, gcp_status* st);
  int64_t dmax() const;
  int n_partials() const;
  ~Batch();
};

struct Serve;

struct Ctx {
  int device = 0;
  uint64_t budget = 0, used = 0;
  // whether this thread's last failed allocation was refused by the budget
  // (rather than by cudaMalloc); per thread, as serving workers allocate
  // concurrently
  bool over_budget() const;
  cudaStream_t own_stream = nullptr, stream = nullptr;
  std::recursive_mutex mu;
  std::mutex alloc_mu;               // allocations may come from serving worker threads
  std::string err;
  int next_id = 1;
  std::map<int, std::unique_ptr<Net>> nets;
  std::map<int, std::unique_ptr<CutSet>> cutsets;
  std::map<Batch*, std::unique_ptr<Batch>> batches;
  std::unordered_map<void*, size_t> sizes;
  // Freed blocks kept for reuse by size class. Only the serving loop's merged
  // batches use it: they are created and destroyed every round, and a
  // cudaFree waits for the whole device, stalling the other networks'
  // streams. A block enters the pool only after the stream that used it has
  // drained, so a reuse from any stream is safe. `used` counts live blocks,
  // `cached` the pooled ones; both count against the budget.
  std::map<size_t, std::vector<void*>> pool;
  uint64_t cached = 0;
  Serve* serve = nullptr;

  gcp_status fail(gcp_status st, const char* fmt, ...);
  gcp_status cuda(cudaError_t e, const char* what);
  void* alloc(size_t bytes);
  void release(void* p);             // cudaFree (waits for the device)
  void recycle(void* p);             // into the pool: no device work may use p any more
  void trim();                       // cudaFree every pooled block
};

// Allocations made while an AllocPool guard is alive on the calling thread
// are rounded up to a size class and may reuse pooled blocks.
struct AllocPool {
  AllocPool();
  ~AllocPool();
  bool prev;
};

// shared by api.cu and serve.cu. last_skip_off: the last layer's skip adds
// xhat^(m)[off .. off + d_L) instead of all of xhat^(m) (bounds of a block of
// rows of a residual layer; 0 through the public entry point)
gcp_status init_net(Ctx& c, const gcp_layer_desc* layers, int n_layers, const double* x_lo, const double* x_hi,
                    const double* spec_c, int n_spec, const double* inter_lo, const double* inter_hi, int* out_id,
                    int last_skip_off = 0);
gcp_status bound_batch(Ctx& c, Batch& b, int prec, int certify, double* out_bound, double* out_cert);
gcp_status add_cuts(Ctx& c, int net_id, int n_cuts, const int64_t* row_ptr, const int16_t* layer, const int8_t* kind,
                    const int32_t* index, const double* coef, const double* d, int* cutset_id, int* first_cut);
gcp_status optimize_batch(Ctx& c, Batch& b, const gcp_opt_params* p, double* out_bound, double* out_cert,
                          double* out_err);
gcp_status duals_create(Ctx& c, int net_id, int cutset_id, const gcp_subdomains* sub, int dual_prec, Batch** out);
// Branching picks (layer << 24 | index, or -1) of every subdomain from the
// nuhat the batch's last evaluation kept (keep_nuhat, float duals): S values
// into picks_dev, enqueued on st.
gcp_status branch_picks_from_last_eval(Ctx& c, Batch& b, cudaStream_t st, int32_t* picks_dev);
gcp_status duals_create_parts(Ctx& c, int net_id,
                              const std::vector<std::pair<const CutSet*, const gcp_subdomains*>>& parts,
                              int dual_prec, Batch** out);
gcp_status sync_check(Ctx& c, cudaStream_t st, const char* what);
gcp_status reset_duals(Ctx& c, Batch& b, bool a, bool be, bool g);
gcp_status optimize_on(Ctx& c, Batch& b, const gcp_opt_params& p, cudaStream_t st, double* cert_dev);
gcp_status eval_dispatch(Ctx& c, Batch& b, cudaStream_t st, int prec, bool adj_start, const void* seed,
                         bool theta_init = false);
gcp_status certify_dispatch(Ctx& c, Batch& b, cudaStream_t st, double* out_dev);
void serve_shutdown(Ctx& c);

}  // namespace gcp

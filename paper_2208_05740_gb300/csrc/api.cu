// Host implementation of the C ABI in include/gcp.h.
//
// Owns device memory (budgeted per context), validates every argument on the
// host (the kernels trust indices), and sequences the kernels of
//   eval     : Theorem 3.1 backwards from nu^(L) = -c to the input box,
//   adjoint  : its reverse-mode derivative (forward through W^(i)),
//   update   : projected ascent on (alpha, beta, gamma),
//   certify  : the float64 outward-rounded Lagrangian at the reached duals.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <type_traits>
#include <numeric>
#include <type_traits>
#include <string>
#include <unordered_map>
#include <vector>

#include "gcp_ctx.h"

namespace gcp {

// ------------------------------------------------------------------ errors
gcp_status Ctx::fail(gcp_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  err = buf;
  return st;
}

gcp_status Ctx::cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return GCP_OK;
  return fail(GCP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

namespace {
thread_local bool t_pool = false;

// 256-byte steps up to 64 KiB, then four classes per power of two (at most
// 25% above the request), so that batches of nearby sizes share blocks.
size_t size_class(size_t b) {
  b = (b + 255) & ~size_t(255);
  if (b <= (size_t(64) << 10)) return b;
  int k = 63;
  while (!((b >> k) & 1)) --k;
  const size_t step = size_t(1) << (k - 2);
  return (b + step - 1) & ~(step - 1);
}

// pooled bytes kept at most (a quarter of the budget; 8 GiB without one)
uint64_t pool_cap(const Ctx& c) { return c.budget ? c.budget / 4 : uint64_t(8) << 30; }

// cudaFree pooled blocks, largest classes first, until at most `keep` bytes remain
void trim_to(Ctx& c, uint64_t keep) {
  while (c.cached > keep && !c.pool.empty()) {
    auto it = std::prev(c.pool.end());
    if (it->second.empty()) {
      c.pool.erase(it);
      continue;
    }
    cudaFree(it->second.back());
    it->second.pop_back();
    c.cached -= it->first;
  }
}
}  // namespace

AllocPool::AllocPool() : prev(t_pool) { t_pool = true; }
AllocPool::~AllocPool() { t_pool = prev; }

namespace {
thread_local bool t_over_budget = false;
}  // namespace

bool Ctx::over_budget() const { return t_over_budget; }

void* Ctx::alloc(size_t bytes) {
  std::lock_guard<std::mutex> lk(alloc_mu);
  t_over_budget = false;
  if (bytes == 0) bytes = 16;
  bytes = t_pool ? size_class(bytes) : (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  auto it = t_pool ? pool.find(bytes) : pool.end();
  if (it != pool.end() && !it->second.empty()) {
    p = it->second.back();
    it->second.pop_back();
    cached -= bytes;
  } else {
    if (budget && used + bytes > budget) {
      t_over_budget = true;
      return nullptr;
    }
    if (budget && used + cached + bytes > budget) trim_to(*this, budget - used - bytes);
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      if (!cached) return nullptr;
      trim_to(*this, 0);
      if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
    }
  }
  sizes[p] = bytes;
  used += bytes;
  reg_alloc(p, bytes);
  return p;
}

void Ctx::release(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(alloc_mu);
  auto it = sizes.find(p);
  if (it != sizes.end()) {
    used -= it->second;
    sizes.erase(it);
  }
  reg_free(p);
  cudaFree(p);
}

void Ctx::recycle(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(alloc_mu);
  auto it = sizes.find(p);
  if (it == sizes.end()) return;
  const size_t bytes = it->second;
  used -= bytes;
  sizes.erase(it);
  reg_free(p);
  const uint64_t cap = pool_cap(*this);
  if (cached + bytes > cap) trim_to(*this, cap > bytes ? cap - bytes : 0);
  if (cached + bytes > cap) {
    cudaFree(p);
    return;
  }
  pool[bytes].push_back(p);
  cached += bytes;
}

void Ctx::trim() {
  std::lock_guard<std::mutex> lk(alloc_mu);
  trim_to(*this, 0);
  pool.clear();
}

template <typename T>
T* upload(Ctx& c, const T* host, size_t n, gcp_status* st) {
  T* d = static_cast<T*>(c.alloc(n * sizeof(T)));
  if (!d) {
    *st = c.over_budget() ? c.fail(GCP_EBUDGET, "device memory budget exceeded")
                        : c.fail(GCP_ENOMEM, "cudaMalloc of %zu bytes failed", n * sizeof(T));
    return nullptr;
  }
  if (n && host) {
    cudaError_t e = cudaMemcpy(d, host, n * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      *st = c.cuda(e, "upload");
      return nullptr;
    }
  }
  *st = GCP_OK;
  return d;
}

static std::vector<float> to_f32(const double* p, size_t n) {
  std::vector<float> v(n);
  for (size_t i = 0; i < n; ++i) v[i] = (float)p[i];
  return v;
}
// x = hi + lo, hi = x rounded to tf32 (10-bit mantissa) to nearest, ties away
// from zero; lo = x - hi is exact in float.
static float tf32_hi_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;
  u = (u + 0x1000u) & 0xffffe000u;
  float h;
  std::memcpy(&h, &u, 4);
  return h;
}
static void tf32_split(const std::vector<float>& v, std::vector<float>& hi, std::vector<float>& lo) {
  hi.resize(v.size());
  lo.resize(v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    hi[i] = tf32_hi_host(v[i]);
    lo[i] = v[i] - hi[i];
  }
}

// bf16(w) as a double (the high term of the three-term weights; the low term
// is w - bf16_hi(w), rounded to bf16 in turn)
static double bf16_hi(double w) { return (double)__bfloat162float(__float2bfloat16_rn((float)w)); }

static std::vector<__nv_bfloat16> to_bf16(const double* p, size_t n) {
  std::vector<__nv_bfloat16> v(n);
  for (size_t i = 0; i < n; ++i) v[i] = __float2bfloat16_rn((float)p[i]);
  return v;
}

Net::~Net() {
  for (void* p : owned) ctx->release(p);
}
CutDev::~CutDev() {
  for (void* p : owned) pooled ? ctx->recycle(p) : ctx->release(p);
}
Batch::~Batch() {
  if (pool_stream) {
    cudaStreamSynchronize(pool_stream);
    cuts.pooled = true;
    for (void* p : owned) ctx->recycle(p);
    for (auto& kv : lazy) ctx->recycle(kv.second);
    return;
  }
  for (void* p : owned) ctx->release(p);
  for (auto& kv : lazy) ctx->release(kv.second);
}

void* Batch::ws(const std::string& name, size_t bytes, gcp_status* st) {
  auto it = lazy.find(name);
  if (it != lazy.end()) {
    if (lazy_bytes[name] >= bytes) return it->second;
    if (pool_stream) {
      cudaStreamSynchronize(pool_stream);
      ctx->recycle(it->second);
    } else {
      ctx->release(it->second);
    }
    lazy.erase(it);
  }
  void* p = nullptr;
  if (pool_stream) {
    AllocPool g;
    p = ctx->alloc(bytes);
  } else {
    p = ctx->alloc(bytes);
  }
  if (!p) {
    *st = ctx->over_budget() ? ctx->fail(GCP_EBUDGET, "device memory budget exceeded (%s)", name.c_str())
                           : ctx->fail(GCP_ENOMEM, "cudaMalloc of %zu bytes failed (%s)", bytes, name.c_str());
    return nullptr;
  }
  lazy[name] = p;
  lazy_bytes[name] = bytes;
  return p;
}

// Launch-check problems (a skipped launch) and CUDA launch errors of a sequence.
gcp_status launch_status(Ctx& c, const char* what) {
  std::string e = reg_take_error();
  if (!e.empty()) return c.fail(GCP_EDEVICE, "%s: %s", what, e.c_str());
  return c.cuda(cudaGetLastError(), what);
}

// Synchronise and report CUDA errors, then failed in-kernel index checks.
gcp_status sync_check(Ctx& c, cudaStream_t st, const char* what) {
  gcp_status s = c.cuda(cudaStreamSynchronize(st), what);
  if (s) return s;
  std::string e = take_device_error(st);
  if (!e.empty()) return c.fail(GCP_EDEVICE, "%s: %s", what, e.c_str());
  e = take_tc_error(st);
  if (!e.empty()) return c.fail(GCP_EDEVICE, "%s: %s", what, e.c_str());
  return GCP_OK;
}

// Higham's gamma_n = n u / (1 - n u) with a safety factor for the host rounding.
static double gamma_n_host(int64_t n) {
  const double u = std::ldexp(1.0, -53);
  const double nu = (double)n * u;
  return nu / (1.0 - nu) * (1.0 + std::ldexp(1.0, -30));
}

// reduction length of y^(i-1) = W^(i)^T nu^(i) (the K of the backward product)
static int64_t red_len(const LayerGeom& g) {
  return g.kind == GCP_DENSE ? g.d_out : (int64_t)g.c_out * g.k * g.k;
}

// ------------------------------------------------------------------ net
gcp_status init_net(Ctx& c, const gcp_layer_desc* layers, int n_layers, const double* x_lo, const double* x_hi,
                    const double* spec_c, int n_spec, const double* inter_lo, const double* inter_hi, int* out_id,
                    int last_skip_off) {
  if (!layers || n_layers < 1 || !x_lo || !x_hi || !spec_c || n_spec < 1 || !out_id)
    return c.fail(GCP_EINVAL, "gcp_init_net: null argument or empty network/spec");
  auto net = std::make_unique<Net>();
  net->ctx = &c;
  net->L = n_layers;
  net->K = n_spec;
  auto parse = [&](const gcp_layer_desc& d, const char* what, int i, LayerGeom& g) -> gcp_status {
    g = LayerGeom{};
    g.kind = d.kind;
    g.d_in = d.d_in;
    g.d_out = d.d_out;
    if (d.kind == GCP_DENSE) {
      if (d.d_in <= 0 || d.d_out <= 0) return c.fail(GCP_EINVAL, "%s %d: bad dense shape", what, i);
    } else if (d.kind == GCP_CONV2D) {
      g.c_in = d.c_in; g.h_in = d.h_in; g.w_in = d.w_in; g.c_out = d.c_out; g.h_out = d.h_out;
      g.w_out = d.w_out; g.k = d.k; g.stride = d.stride; g.pad = d.pad;
      if (d.c_in <= 0 || d.h_in <= 0 || d.w_in <= 0 || d.c_out <= 0 || d.k <= 0 || d.stride <= 0 || d.pad < 0 ||
          d.h_out != (d.h_in + 2 * d.pad - d.k) / d.stride + 1 || d.w_out != (d.w_in + 2 * d.pad - d.k) / d.stride + 1 ||
          d.d_in != d.c_in * d.h_in * d.w_in || d.d_out != d.c_out * d.h_out * d.w_out || d.h_out <= 0 || d.w_out <= 0)
        return c.fail(GCP_EINVAL, "%s %d: inconsistent conv2d geometry", what, i);
    } else {
      return c.fail(GCP_EINVAL, "%s %d: unknown kind %d", what, i, d.kind);
    }
    if (!d.W) return c.fail(GCP_EINVAL, "%s %d: null W", what, i);
    return GCP_OK;
  };
  for (int i = 0; i < n_layers; ++i) {
    const gcp_layer_desc& d = layers[i];
    LayerGeom g;
    if (gcp_status e = parse(d, "layer", i + 1, g)) return e;
    if (d.kind == GCP_CONV2D && i == n_layers - 1) return c.fail(GCP_EINVAL, "the last (spec) layer must be dense");
    if (i > 0 && d.d_in != layers[i - 1].d_out) return c.fail(GCP_EINVAL, "layer %d: d_in mismatch", i + 1);
    if (!d.b) return c.fail(GCP_EINVAL, "layer %d: null b", i + 1);
    net->geom.push_back(g);
  }
  net->dims.push_back(layers[0].d_in);
  for (int i = 0; i < n_layers; ++i) net->dims.push_back(layers[i].d_out);
  const int L = n_layers;
  const int d0 = net->dims[0], dL = net->dims[L];
  // skip connections: x^(i) += S xhat^(s-1), one consumer per source; the
  // projections S become maps L+1, L+2, ... after the layers
  net->skip.assign(L, 0);
  net->consumer.assign(L, 0);
  net->sc_map.assign(L, 0);
  net->skip_off = last_skip_off;
  std::vector<const gcp_layer_desc*> maps;
  for (int i = 0; i < L; ++i) maps.push_back(&layers[i]);
  if (last_skip_off < 0 || (last_skip_off > 0 && (layers[L - 1].skip == 0 || layers[L - 1].shortcut)))
    return c.fail(GCP_EINVAL, "skip offset without an identity skip on the last layer");
  for (int i = 1; i <= L; ++i) {
    const gcp_layer_desc& d = layers[i - 1];
    const int s = d.skip;
    if (s == 0) {
      if (d.shortcut) return c.fail(GCP_EINVAL, "layer %d: shortcut without a skip", i);
      continue;
    }
    const int off = i == L ? last_skip_off : 0;
    if (s < 0 || s > i) return c.fail(GCP_EINVAL, "layer %d: skip %d must name an earlier xhat (1..%d)", i, s, i);
    const int m = s - 1;
    if (const gcp_layer_desc* sd = d.shortcut) {
      LayerGeom g;
      if (gcp_status e = parse(*sd, "shortcut of layer", i, g)) return e;
      if (sd->d_in != net->dims[m] || sd->d_out != net->dims[i] || sd->b || sd->skip || sd->shortcut ||
          (i == L && sd->kind != GCP_DENSE))
        return c.fail(GCP_EINVAL, "layer %d: the shortcut maps xhat^(%d) (%d) to %d outputs, with b = NULL, no skip "
                      "of its own, dense on the last layer", i, m, net->dims[m], net->dims[i]);
      net->geom.push_back(g);
      maps.push_back(sd);
      net->sc_map[i - 1] = (int)maps.size();
    } else if (i < L ? net->dims[m] != net->dims[i] : (int64_t)off + net->dims[i] > net->dims[m]) {
      return c.fail(GCP_EINVAL, "layer %d: skip from xhat^(%d) of width %d does not fit width %d", i, m,
                    net->dims[m], net->dims[i]);
    }
    if (net->consumer[m]) return c.fail(GCP_EINVAL, "xhat^(%d) feeds two skips (layers %d and %d)", m, net->consumer[m], i);
    net->skip[i - 1] = s;
    net->consumer[m] = i;
  }
  const int n_maps = (int)maps.size();
  int64_t nh = 0;
  for (int i = 1; i < L; ++i) nh += net->dims[i];
  if (nh > 0 && (!inter_lo || !inter_hi)) return c.fail(GCP_EINVAL, "intermediate bounds required");
  for (int j = 0; j < d0; ++j)
    if (!(x_lo[j] <= x_hi[j]) || !std::isfinite(x_lo[j]) || !std::isfinite(x_hi[j]))
      return c.fail(GCP_EINVAL, "input box: x_lo > x_hi or non-finite at %d", j);
  for (int64_t j = 0; j < nh; ++j)
    if (!(inter_lo[j] <= inter_hi[j]) || !std::isfinite(inter_lo[j]) || !std::isfinite(inter_hi[j]))
      return c.fail(GCP_EINVAL, "intermediate bounds: lo > hi or non-finite at %lld", (long long)j);
  for (int64_t j = 0; j < (int64_t)n_spec * dL; ++j)
    if (!std::isfinite(spec_c[j])) return c.fail(GCP_EINVAL, "spec: non-finite entry");
  gcp_status st = GCP_OK;
#define UP(dst, T, host, n)                    \
  do {                                         \
    dst = upload<T>(c, host, n, &st);          \
    if (!dst) return st;                       \
    net->owned.push_back((void*)dst);          \
  } while (0)
  const std::vector<double> no_bias((size_t)*std::max_element(net->dims.begin(), net->dims.end()), 0.0);
  for (int i = 0; i < n_maps; ++i) {
    const gcp_layer_desc& d = *maps[i];
    const LayerGeom& g = net->geom[i];
    const double* bias = d.b ? d.b : no_bias.data();    // projections carry no bias
    size_t nw = g.kind == GCP_DENSE ? (size_t)g.d_out * g.d_in : (size_t)g.c_out * g.c_in * g.k * g.k;
    for (size_t q = 0; q < nw; ++q)
      if (!std::isfinite(d.W[q])) return c.fail(GCP_EINVAL, "map %d: non-finite weight", i + 1);
    for (int q = 0; q < g.d_out; ++q)
      if (!std::isfinite(bias[q])) return c.fail(GCP_EINVAL, "layer %d: non-finite bias", i + 1);
    double *w64, *wt64 = nullptr, *b64;
    float *w32, *wt32 = nullptr, *b32, *w32h = nullptr, *w32l = nullptr, *wt32h = nullptr, *wt32l = nullptr;
    __nv_bfloat16 *w16, *wt16 = nullptr;
    UP(w64, double, d.W, nw);
    auto wf = to_f32(d.W, nw);
    UP(w32, float, wf.data(), nw);
    auto wh = to_bf16(d.W, nw);
    UP(w16, __nv_bfloat16, wh.data(), nw);
    if (g.kind == GCP_DENSE) {
      std::vector<double> t(nw);
      for (int o = 0; o < g.d_out; ++o)
        for (int q = 0; q < g.d_in; ++q) t[(size_t)q * g.d_out + o] = d.W[(size_t)o * g.d_in + q];
      UP(wt64, double, t.data(), nw);
      auto tf = to_f32(t.data(), nw);
      UP(wt32, float, tf.data(), nw);
      auto th = to_bf16(t.data(), nw);
      UP(wt16, __nv_bfloat16, th.data(), nw);
      std::vector<float> hi, lo;
      tf32_split(wf, hi, lo);
      UP(w32h, float, hi.data(), nw);
      UP(w32l, float, lo.data(), nw);
      tf32_split(tf, hi, lo);
      UP(wt32h, float, hi.data(), nw);
      UP(wt32l, float, lo.data(), nw);
    }
    __nv_bfloat16 *cf16 = nullptr, *ct16 = nullptr, *cs16 = nullptr, *wt16x3 = nullptr;
    int cfk = 0, cfn = 0, ctk = 0, ctn = 0, cs_k = 0, cs_n = 0;
    ConvSecondB b2;
    if (g.kind != GCP_DENSE) {
      // columns by the convolution plan of each direction (phases, taps,
      // source channel padded to 8), rows = output channels padded to 16
      // gg: the plan's geometry; for split_geom(g) (the mixed chain's operand
      // [nu_hi | nu_lo] as twice the channels) output channel t c_out + o
      // carries term(weight of o, t): W_hi for both t in the first weight
      // operand, W_lo for t = 0 and 0 for t = 1 in the second
      auto pack_d = [&](bool transposed, int& kp, int& np_, const LayerGeom& gg, int which) {
        ConvPlan cp;
        std::vector<double> p;
        if (!conv_plan(gg, transposed ? 1 : 0, cp)) { kp = np_ = 0; return p; }
        kp = cp.Kp;
        np_ = cp.Np;
        p.assign((size_t)np_ * kp, 0.0);
        const int step = transposed ? g.stride : 1;
        for (int q = 0; q < cp.nph; ++q) {
          const ConvPhase& f = cp.f[q];
          for (int a = 0; a < f.nkh; ++a)
            for (int b = 0; b < f.nkw; ++b) {
              const int kh = f.rh + step * a, kw = f.rw + step * b;
              const size_t col0 = (size_t)f.kb0 * 64 + (size_t)(a * f.nkw + b) * cp.Csp;
              for (int o = 0; o < gg.c_out; ++o)
                for (int ci = 0; ci < g.c_in; ++ci) {
                  const double wf = d.W[(((size_t)(o % g.c_out) * g.c_in + ci) * g.k + kh) * g.k + kw];
                  const int term = o / g.c_out;
                  const double w = which == 0 ? wf : (which == 1 ? bf16_hi(wf) : (term == 0 ? wf - bf16_hi(wf) : 0.0));
                  const int n = transposed ? ci : o, c = transposed ? o : ci;
                  p[(size_t)n * kp + col0 + c] = w;
                }
            }
        }
        return p;
      };
      auto pack = [&](bool transposed, int& kp, int& np_, const LayerGeom& gg) {
        auto p = pack_d(transposed, kp, np_, gg, 0);
        return to_bf16(p.data(), p.size());
      };
      auto pf = pack(false, cfk, cfn, g);
      if (!pf.empty()) UP(cf16, __nv_bfloat16, pf.data(), pf.size());
      auto pt = pack(true, ctk, ctn, g);
      if (!pt.empty()) UP(ct16, __nv_bfloat16, pt.data(), pt.size());
      // the transposed product of the mixed chain on the tensor cores: A from
      // [nu_hi | nu_lo], weights [W_hi | W_hi] and, reusing each A block,
      // [W_lo | 0] (its all-zero K blocks left out). A map of fewer than 8
      // output channels (an input layer's c_in) would fill at most 8 of a
      // tile's 16 columns while its producers stage twice the source
      // channels: it runs in float on the SIMT units instead
      if (g.c_in >= 8) {
        const LayerGeom g2 = split_geom(g);
        auto p1 = pack_d(true, cs_k, cs_n, g2, 1);
        int k2 = 0, n2 = 0;
        auto p2 = pack_d(true, k2, n2, g2, 2);
        if (!p1.empty() && k2 == cs_k && n2 == cs_n && cs_k / 64 <= kConvMaxKb) {
          const int nkb = cs_k / 64;
          b2.map.assign(nkb, -1);
          std::vector<int> keep;
          for (int kb = 0; kb < nkb; ++kb) {
            bool any = false;
            for (int n = 0; n < cs_n && !any; ++n)
              for (int j = 0; j < 64 && !any; ++j) any = p2[(size_t)n * cs_k + kb * 64 + j] != 0.0;
            if (any) {
              b2.map[kb] = (int8_t)keep.size();
              keep.push_back(kb);
            }
          }
          b2.nb2 = (int)keep.size();
          std::vector<double> c2((size_t)cs_n * 64 * std::max(b2.nb2, 1), 0.0);
          for (int n = 0; n < cs_n; ++n)
            for (int t = 0; t < b2.nb2; ++t)
              for (int j = 0; j < 64; ++j)
                c2[(size_t)n * 64 * b2.nb2 + t * 64 + j] = p2[(size_t)n * cs_k + keep[t] * 64 + j];
          if (conv_tc_fits(g2, 1, cs_k, cs_n, b2.nb2)) {
            auto h1 = to_bf16(p1.data(), p1.size());
            auto h2 = to_bf16(c2.data(), c2.size());
            UP(cs16, __nv_bfloat16, h1.data(), h1.size());
            __nv_bfloat16* w2 = nullptr;
            UP(w2, __nv_bfloat16, h2.data(), h2.size());
            b2.W = b2.nb2 > 0 ? w2 : nullptr;
          } else {
            b2 = ConvSecondB{};
          }
        }
      }
    } else if (tc_available(kDenseTerms * g.d_out, true)) {
      // rows of [W_hi^T | W_hi^T | W_lo^T] for the three-term operand [hi | lo | hi]
      const size_t K3 = (size_t)kDenseTerms * g.d_out;
      std::vector<double> t3((size_t)g.d_in * K3);
      for (int q = 0; q < g.d_in; ++q)
        for (int o = 0; o < g.d_out; ++o) {
          const double w = d.W[(size_t)o * g.d_in + q];
          t3[(size_t)q * K3 + o] = t3[(size_t)q * K3 + g.d_out + o] = bf16_hi(w);
          t3[(size_t)q * K3 + 2 * g.d_out + o] = w - bf16_hi(w);
        }
      auto t3h = to_bf16(t3.data(), t3.size());
      UP(wt16x3, __nv_bfloat16, t3h.data(), t3h.size());
    }
    float* wabs = nullptr;
    if (g.kind != GCP_DENSE) {
      std::vector<float> wa(nw);
      for (size_t q = 0; q < nw; ++q) {
        const double v = std::fabs(d.W[q]);
        float f = (float)v;
        if ((double)f < v) f = std::nextafter(f, INFINITY);   // rounded up
        wa[q] = f;
      }
      UP(wabs, float, wa.data(), nw);
    }
    net->Wabs32.push_back(wabs);
    // the certification's float64 product y = W^T nu on the tensor cores: the
    // rows of W^T cut into exact bf16 slices once, here
    SliceB sl;
    if (g.kind == GCP_DENSE && slice_params(g.d_out, sl.b, sl.s, sl.cerr) && tc_available(g.d_out, true)) {
      const size_t np = (size_t)g.d_in * sl.s * g.d_out;
      UP(sl.planes, __nv_bfloat16, nullptr, np);
      UP(sl.exps, int32_t, nullptr, (size_t)g.d_in);
      slice_rows(c.stream, g.d_in, g.d_out, wt64, sl.b, sl.s, true, sl.planes, sl.exps);
      if (!reg_take_error().empty()) return c.fail(GCP_EDEVICE, "layer %d: weight slices", i + 1);
      st = c.cuda(cudaStreamSynchronize(c.stream), "weight slices");
      if (st) return st;
    } else {
      sl = SliceB{};
    }
    net->WTsl.push_back(sl);
    net->CF16.push_back(cf16); net->CT16.push_back(ct16);
    net->cf_kp.push_back(cfk); net->cf_np.push_back(cfn); net->ct_kp.push_back(ctk); net->ct_np.push_back(ctn);
    net->WT16x3.push_back(wt16x3); net->CT16s.push_back(cs16);
    net->cts_kp.push_back(cs16 ? cs_k : 0); net->cts_np.push_back(cs16 ? cs_n : 0); net->CTs_b2.push_back(b2);
    UP(b64, double, bias, g.d_out);
    auto bf = to_f32(bias, g.d_out);
    UP(b32, float, bf.data(), g.d_out);
    net->W64.push_back(w64); net->WT64.push_back(wt64); net->b64.push_back(b64);
    net->W32.push_back(w32); net->WT32.push_back(wt32); net->b32.push_back(b32);
    net->W16.push_back(w16); net->WT16.push_back(wt16);
    net->W32hi.push_back(w32h); net->W32lo.push_back(w32l); net->WT32hi.push_back(wt32h); net->WT32lo.push_back(wt32l);
  }
  UP(net->xlo64, double, x_lo, d0);
  UP(net->xhi64, double, x_hi, d0);
  auto xl = to_f32(x_lo, d0), xh = to_f32(x_hi, d0);
  UP(net->xlo32, float, xl.data(), d0);
  UP(net->xhi32, float, xh.data(), d0);
  UP(net->C64, double, spec_c, (size_t)n_spec * dL);
  std::vector<double> negc((size_t)n_spec * dL);
  for (size_t q = 0; q < negc.size(); ++q) negc[q] = -spec_c[q];
  UP(net->negC64, double, negc.data(), negc.size());
  // y^(L-1) = W^(L)^T nu^(L) = -W^(L)^T c_k and c_k^T b^(L), per spec row
  const gcp_layer_desc& last = layers[L - 1];
  const int dl1 = net->dims[L - 1];
  std::vector<double> yl((size_t)n_spec * dl1, 0.0), cb(n_spec, 0.0);
  for (int k = 0; k < n_spec; ++k) {
    for (int q = 0; q < dL; ++q) {
      const double cv = spec_c[(size_t)k * dL + q];
      if (cv == 0.0) continue;   // sparse specs (unit rows) skip the zero columns
      cb[k] += cv * last.b[q];
      for (int j = 0; j < dl1; ++j) yl[(size_t)k * dl1 + j] -= cv * last.W[(size_t)q * dl1 + j];
    }
  }
  // a skip on the last layer adds S^T nu^(L) = -S^T c_k (S = I: -c_k at the
  // skip's offset) to y^(m); from the last hidden layer it folds into y^(L-1)
  if (const int sL = net->skip[L - 1]) {
    const int m = sL - 1, dm = net->dims[m];
    std::vector<double> sk((size_t)n_spec * dm, 0.0);
    for (int k = 0; k < n_spec; ++k)
      for (int q = 0; q < dL; ++q) {
        const double cv = spec_c[(size_t)k * dL + q];
        if (cv == 0.0) continue;
        if (!last.shortcut) {
          sk[(size_t)k * dm + net->skip_off + q] -= cv;
        } else {
          const double* Srow = last.shortcut->W + (size_t)q * dm;
          for (int j = 0; j < dm; ++j) sk[(size_t)k * dm + j] -= cv * Srow[j];
        }
      }
    if (m == L - 1) {
      for (size_t q = 0; q < yl.size(); ++q) yl[q] += sk[q];
    } else {
      UP(net->SK64, double, sk.data(), sk.size());
      auto skf = to_f32(sk.data(), sk.size());
      UP(net->SK32, float, skf.data(), skf.size());
    }
  }
  UP(net->YL64, double, yl.data(), yl.size());
  auto ylf = to_f32(yl.data(), yl.size());
  UP(net->YL32, float, ylf.data(), ylf.size());
  UP(net->cb64, double, cb.data(), n_spec);
  auto cbf = to_f32(cb.data(), n_spec);
  UP(net->cb32, float, cbf.data(), n_spec);
  UP(net->bL64, double, last.b, dL);
  int64_t off = 0;
  for (int i = 1; i < L; ++i) {
    const int di = net->dims[i];
    double *lo, *hi;
    float *lof, *hif;
    UP(lo, double, inter_lo + off, di);
    UP(hi, double, inter_hi + off, di);
    auto a = to_f32(inter_lo + off, di), b = to_f32(inter_hi + off, di);
    // float copies rounded outwards so that float classification never
    // treats an unstable neuron as stable
    for (int j = 0; j < di; ++j) {
      if ((double)a[j] > inter_lo[off + j]) a[j] = std::nextafter(a[j], -INFINITY);
      if ((double)b[j] < inter_hi[off + j]) b[j] = std::nextafter(b[j], INFINITY);
    }
    UP(lof, float, a.data(), di);
    UP(hif, float, b.data(), di);
    net->lo64.push_back(lo); net->hi64.push_back(hi); net->lo32.push_back(lof); net->hi32.push_back(hif);
    std::vector<double> iv(di, 0.0);
    std::vector<float> ivf(di, 0.f);
    for (int j = 0; j < di; ++j) {
      if (inter_lo[off + j] < 0 && inter_hi[off + j] > 0) iv[j] = 1.0 / (inter_hi[off + j] - inter_lo[off + j]);
      if (a[j] < 0.f && b[j] > 0.f) ivf[j] = 1.f / (b[j] - a[j]);
    }
    double* ivd;
    float* ivs;
    UP(ivd, double, iv.data(), di);
    UP(ivs, float, ivf.data(), di);
    net->invul64.push_back(ivd); net->invul32.push_back(ivs);
    std::vector<int32_t> un;
    for (int j = 0; j < di; ++j)
      if (inter_lo[off + j] < 0 && inter_hi[off + j] > 0) un.push_back(j);
    net->unstable.push_back(un);
    off += di;
  }
#undef UP
  int id = c.next_id++;
  c.nets[id] = std::move(net);
  *out_id = id;
  return GCP_OK;
}

// ------------------------------------------------------------------ cuts
gcp_status add_cuts(Ctx& c, int net_id, int n_cuts, const int64_t* row_ptr, const int16_t* layer, const int8_t* kind,
                    const int32_t* index, const double* coef, const double* d, int* cutset_id, int* first_cut) {
  auto it = c.nets.find(net_id);
  if (it == c.nets.end()) return c.fail(GCP_ENOTFOUND, "unknown net %d", net_id);
  if (!cutset_id || n_cuts < 0 || (n_cuts > 0 && (!row_ptr || !d))) return c.fail(GCP_EINVAL, "gcp_add_cuts: bad arguments");
  Net& net = *it->second;
  CutSet* cs = nullptr;
  if (*cutset_id < 0) {
    auto p = std::make_unique<CutSet>();
    p->net_id = net_id;
    p->ptr.push_back(0);
    int id = c.next_id++;
    cs = p.get();
    c.cutsets[id] = std::move(p);
    *cutset_id = id;
  } else {
    auto ci = c.cutsets.find(*cutset_id);
    if (ci == c.cutsets.end()) return c.fail(GCP_ENOTFOUND, "unknown cut set %d", *cutset_id);
    cs = ci->second.get();
    if (cs->net_id != net_id) return c.fail(GCP_EINVAL, "cut set %d belongs to net %d", *cutset_id, cs->net_id);
  }
  if (n_cuts > 0) {
    if (row_ptr[0] != 0) return c.fail(GCP_EINVAL, "row_ptr[0] must be 0");
    const int64_t nnz = row_ptr[n_cuts];
    if (nnz > 0 && (!layer || !kind || !index || !coef)) return c.fail(GCP_EINVAL, "null cut entry arrays");
    for (int k = 0; k < n_cuts; ++k) {
      if (row_ptr[k + 1] < row_ptr[k]) return c.fail(GCP_EINVAL, "row_ptr not monotone at cut %d", k);
      if (!std::isfinite(d[k])) return c.fail(GCP_EINVAL, "cut %d: non-finite d", k);
    }
    for (int64_t e = 0; e < nnz; ++e) {
      const int li = layer[e];
      if (li < 0 || li >= net.L) return c.fail(GCP_EINVAL, "entry %lld: layer %d out of range", (long long)e, li);
      if (kind[e] < 0 || kind[e] > 2) return c.fail(GCP_EINVAL, "entry %lld: bad kind", (long long)e);
      if (li == 0 && kind[e] != GCP_VAR_X) return c.fail(GCP_EINVAL, "entry %lld: input variables have kind X", (long long)e);
      if (index[e] < 0 || index[e] >= net.dims[li]) return c.fail(GCP_EINVAL, "entry %lld: index out of range", (long long)e);
      if (!std::isfinite(coef[e])) return c.fail(GCP_EINVAL, "entry %lld: non-finite coef", (long long)e);
    }
    if ((int64_t)cs->d.size() + n_cuts > 65535) return c.fail(GCP_EINVAL, "at most 65535 cuts per set");
    const int64_t base = cs->ptr.back();
    if (first_cut) *first_cut = (int)cs->d.size();
    for (int k = 0; k < n_cuts; ++k) {
      cs->d.push_back(d[k]);
      cs->ptr.push_back(base + row_ptr[k + 1]);
    }
    cs->layer.insert(cs->layer.end(), layer, layer + nnz);
    cs->kind.insert(cs->kind.end(), kind, kind + nnz);
    cs->index.insert(cs->index.end(), index, index + nnz);
    cs->coef.insert(cs->coef.end(), coef, coef + nnz);
  } else if (first_cut) {
    *first_cut = (int)cs->d.size();
  }
  return GCP_OK;
}

// Device copy of a cut set: CSR by cut for the gather, CSC by (layer, neuron, kind).
gcp_status build_cutdev(Ctx& c, const Net& net, const CutSet* cs, CutDev& out) {
  out.ctx = &c;
  const int L = net.L;
  out.N = cs ? (int)cs->d.size() : 0;
  out.nnz = cs ? (int64_t)cs->coef.size() : 0;
  std::vector<int64_t> poff(L + 1, 0);
  for (int i = 0; i < L; ++i) poff[i + 1] = poff[i] + net.dims[i] + 1;
  out.poff = poff;
  std::vector<int32_t> cut_of(out.nnz);
  for (int k = 0; k < out.N; ++k)
    for (int64_t e = cs->ptr[k]; e < cs->ptr[k + 1]; ++e) cut_of[e] = k;
  std::vector<int64_t> order(out.nnz);
  std::iota(order.begin(), order.end(), 0);
  if (out.nnz)
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
      if (cs->layer[a] != cs->layer[b]) return cs->layer[a] < cs->layer[b];
      if (cs->index[a] != cs->index[b]) return cs->index[a] < cs->index[b];
      return cs->kind[a] < cs->kind[b];   // runs of equal (neuron, kind): one segment each
    });
  std::vector<int32_t> cptr(poff[L], 0), ccut(out.nnz), ceid(out.nnz), cnrn(out.nnz), cpos(out.nnz);
  std::vector<int8_t> ckind(out.nnz);
  std::vector<double> ccoef(out.nnz);
  std::vector<int64_t> cnt(poff[L], 0);
  for (int64_t e = 0; e < out.nnz; ++e) cnt[poff[cs->layer[e]] + cs->index[e]]++;
  out.layer_nnz.assign(L, 0);
  for (int64_t e = 0; e < out.nnz; ++e) out.layer_nnz[cs->layer[e]]++;
  for (int i = 0; i < L; ++i) {
    int64_t run = 0;
    // entries of layer i start after all entries of layers < i
    for (int q = 0; q < i; ++q)
      for (int j = 0; j < net.dims[q]; ++j) run += cnt[poff[q] + j];
    for (int j = 0; j <= net.dims[i]; ++j) {
      cptr[poff[i] + j] = (int32_t)run;
      if (j < net.dims[i]) run += cnt[poff[i] + j];
    }
  }
  out.span4_max.assign(L, 0);
  for (int i = 0; i < L; ++i)
    for (int j0 = 0; j0 < net.dims[i]; j0 += 128) {
      const int j1 = std::min(j0 + 128, net.dims[i]);
      out.span4_max[i] = std::max(out.span4_max[i], cptr[poff[i] + j1] - cptr[poff[i] + j0]);
    }
  for (int64_t q = 0; q < out.nnz; ++q) {
    const int64_t e = order[q];
    ccut[q] = cut_of[e];
    ckind[q] = cs->kind[e];
    ccoef[q] = cs->coef[e];
    ceid[q] = (int32_t)e;
    cnrn[q] = cs->index[e];
    cpos[e] = (int32_t)q;
  }
  std::vector<int32_t> cp32(out.N + 1, 0);
  for (int k = 0; k <= out.N; ++k) cp32[k] = (int32_t)(cs ? cs->ptr[k] : 0);
  std::vector<double> dd = cs ? cs->d : std::vector<double>();
  gcp_status st = GCP_OK;
#define UPC(dst, T, host, n)                   \
  do {                                         \
    dst = upload<T>(c, host, n, &st);          \
    if (!dst) return st;                       \
    out.owned.push_back((void*)dst);           \
  } while (0)
  UPC(out.cut_ptr, int32_t, cp32.data(), cp32.size());
  UPC(out.d64, double, dd.data(), dd.size());
  auto df = to_f32(dd.data(), dd.size());
  UPC(out.d32, float, df.data(), df.size());
  UPC(out.csc_ptr, int32_t, cptr.data(), cptr.size());
  UPC(out.csc_cut, int32_t, ccut.data(), ccut.size());
  UPC(out.csc_kind, int8_t, ckind.data(), ckind.size());
  UPC(out.csc_coef64, double, ccoef.data(), ccoef.size());
  auto cf = to_f32(ccoef.data(), ccoef.size());
  UPC(out.csc_coef32, float, cf.data(), cf.size());
  UPC(out.csc_eid, int32_t, ceid.data(), ceid.size());
  UPC(out.csc_nrn, int32_t, cnrn.data(), cnrn.size());
  UPC(out.csr_pos, int32_t, cpos.data(), cpos.size());
#undef UPC
  return GCP_OK;
}

// ------------------------------------------------------------------ duals
// One batch for one or several queries on the same network. parts[q] = (cut
// set or nullptr, subdomains). Rows are query-major. With several parts the
// cut set is the union of the parts' sets (query q's cuts at offset o_q) and
// every subdomain may only move the multipliers of its own query's cuts; the
// others stay exactly 0 and contribute exact zeros, so a row's duals do not
// depend on what it is batched with.
gcp_status duals_create_parts(Ctx& c, int net_id, const std::vector<std::pair<const CutSet*, const gcp_subdomains*>>& parts,
                              int dual_prec, Batch** out) {
  auto it = c.nets.find(net_id);
  if (it == c.nets.end()) return c.fail(GCP_ENOTFOUND, "unknown net %d", net_id);
  if (!out || parts.empty()) return c.fail(GCP_EINVAL, "gcp_duals_create: bad arguments");
  if (dual_prec != GCP_FP64 && dual_prec != GCP_FP32) return c.fail(GCP_EINVAL, "dual_prec must be FP64 or FP32");
  Net& net = *it->second;
  std::vector<int32_t> sptr(1, 0), cut_lo, cut_hi;
  std::vector<int16_t> slay;
  std::vector<int32_t> sidx;
  std::vector<int8_t> ssgn;
  CutSet uni;
  uni.net_id = net_id;
  uni.ptr.push_back(0);
  int M = 0;
  for (const auto& part : parts) {
    const CutSet* cs = part.first;
    const gcp_subdomains* sub = part.second;
    if (!sub || sub->n_sub < 0) return c.fail(GCP_EINVAL, "gcp_duals_create: bad subdomains");
    if (cs && cs->net_id != net_id) return c.fail(GCP_EINVAL, "cut set of another net");
    const int S = sub->n_sub;
    if (S > 0 && !sub->split_ptr) return c.fail(GCP_EINVAL, "null split_ptr");
    if (S > 0 && sub->split_ptr[0] != 0) return c.fail(GCP_EINVAL, "split_ptr[0] must be 0");
    for (int s = 0; s < S; ++s) {
      const int n = sub->split_ptr[s + 1] - sub->split_ptr[s];
      if (n < 0 || n > kMaxSplits) return c.fail(GCP_EINVAL, "subdomain %d: 0..%d splits allowed", s, kMaxSplits);
      M = std::max(M, n);
    }
    const int64_t nsp = S > 0 ? sub->split_ptr[S] : 0;
    if (nsp > 0 && (!sub->split_layer || !sub->split_index || !sub->split_sign))
      return c.fail(GCP_EINVAL, "null split arrays");
    for (int s = 0; s < S; ++s)
      for (int q = sub->split_ptr[s]; q < sub->split_ptr[s + 1]; ++q) {
        const int li = sub->split_layer[q];
        if (li < 1 || li >= net.L) return c.fail(GCP_EINVAL, "split %d: layer %d not hidden", q, li);
        if (sub->split_index[q] < 0 || sub->split_index[q] >= net.dims[li] || sub->split_index[q] >= (1 << 23) ||
            li >= 128)
          return c.fail(GCP_EINVAL, "split %d: index out of range", q);
        if (sub->split_sign[q] != 1 && sub->split_sign[q] != -1) return c.fail(GCP_EINVAL, "split %d: sign must be +-1", q);
        for (int q2 = sub->split_ptr[s]; q2 < q; ++q2)
          if (sub->split_layer[q2] == li && sub->split_index[q2] == sub->split_index[q])
            return c.fail(GCP_EINVAL, "subdomain %d splits a neuron twice", s);
      }
    const int o = (int)uni.d.size(), nq = cs ? (int)cs->d.size() : 0;
    for (int s = 0; s < S; ++s) {
      sptr.push_back(sptr.back() + sub->split_ptr[s + 1] - sub->split_ptr[s]);
      cut_lo.push_back(o);
      cut_hi.push_back(o + nq);
    }
    if (nsp > 0) {
      slay.insert(slay.end(), sub->split_layer, sub->split_layer + nsp);
      sidx.insert(sidx.end(), sub->split_index, sub->split_index + nsp);
      ssgn.insert(ssgn.end(), sub->split_sign, sub->split_sign + nsp);
    }
    if (cs) {
      const int64_t base = uni.ptr.back();
      for (int k = 0; k < nq; ++k) uni.ptr.push_back(base + cs->ptr[k + 1]);
      uni.layer.insert(uni.layer.end(), cs->layer.begin(), cs->layer.end());
      uni.kind.insert(uni.kind.end(), cs->kind.begin(), cs->kind.end());
      uni.index.insert(uni.index.end(), cs->index.begin(), cs->index.end());
      uni.coef.insert(uni.coef.end(), cs->coef.begin(), cs->coef.end());
      uni.d.insert(uni.d.end(), cs->d.begin(), cs->d.end());
    }
  }
  if (uni.d.size() > 65535) return c.fail(GCP_EINVAL, "at most 65535 cuts per batch");
  const int S = (int)sptr.size() - 1;
  const int64_t nsp = sptr[S];
  gcp_subdomains all{S, sptr.data(), slay.data(), sidx.data(), ssgn.data()};
  const gcp_subdomains* sub = &all;
  const CutSet* cs = uni.d.empty() ? nullptr : &uni;
  auto b = std::make_unique<Batch>();
  b->ctx = &c;
  b->net = &net;
  b->net_id = net_id;
  b->S = S;
  b->K = net.K;
  b->R = (int64_t)S * net.K;
  b->M = M;
  b->fp64 = dual_prec == GCP_FP64;
  {
    const char* e = std::getenv("GCP_TC");
    b->tc = !(e && std::strcmp(e, "0") == 0);
  }
  gcp_status st = build_cutdev(c, net, cs, b->cuts);
  if (st) return st;
  b->N = b->cuts.N;
  b->nnz = b->cuts.nnz;
  b->nsp = nsp;
  b->parts = (int)parts.size();
#define UPB(dst, T, host, n)                   \
  do {                                         \
    dst = upload<T>(c, host, n, &st);          \
    if (!dst) return st;                       \
    b->owned.push_back((void*)dst);            \
  } while (0)
  UPB(b->sp_ptr, int32_t, sptr.data(), S + 1);
  UPB(b->sp_layer, int16_t, sub->split_layer, nsp);
  UPB(b->sp_index, int32_t, sub->split_index, nsp);
  UPB(b->sp_sign, int8_t, sub->split_sign, nsp);
  {
    const int Mt = std::max(M, 1);
    std::vector<int32_t> tab((size_t)S * Mt, -1);
    for (int s = 0; s < S; ++s)
      for (int q = sptr[s]; q < sptr[s + 1]; ++q)
        tab[(size_t)s * Mt + (q - sptr[s])] = split_code_of(sub->split_layer[q], sub->split_index[q], sub->split_sign[q]);
    UPB(b->sp_tab, int32_t, tab.data(), tab.size());
  }
  if (parts.size() > 1) {
    UPB(b->sub_cut_lo, int32_t, cut_lo.data(), S);
    UPB(b->sub_cut_hi, int32_t, cut_hi.data(), S);
  }
  const size_t es = b->fp64 ? 8 : 4;
  for (int i = 1; i < net.L; ++i) {
    void* p = c.alloc((size_t)b->R * net.dims[i] * es);
    if (!p) return c.fail(c.over_budget() ? GCP_EBUDGET : GCP_ENOMEM, "alpha allocation failed");
    b->owned.push_back(p);
    b->alpha.push_back(p);
  }
  b->beta = c.alloc((size_t)std::max(M, 1) * b->R * es);
  if (!b->beta) return c.fail(c.over_budget() ? GCP_EBUDGET : GCP_ENOMEM, "beta allocation failed");
  b->owned.push_back(b->beta);
  b->gamma = c.alloc((size_t)std::max(b->N, 1) * b->R * es);
  if (!b->gamma) return c.fail(c.over_budget() ? GCP_EBUDGET : GCP_ENOMEM, "gamma allocation failed");
  b->owned.push_back(b->gamma);
#undef UPB
  st = reset_duals(c, *b, true, true, true);
  if (st) return st;
  *out = b.get();
  c.batches[b.get()] = std::move(b);
  return GCP_OK;
}

gcp_status duals_create(Ctx& c, int net_id, int cutset_id, const gcp_subdomains* sub, int dual_prec, Batch** out) {
  const CutSet* cs = nullptr;
  if (cutset_id >= 0) {
    auto ci = c.cutsets.find(cutset_id);
    if (ci == c.cutsets.end()) return c.fail(GCP_ENOTFOUND, "unknown cut set %d", cutset_id);
    cs = ci->second.get();
  }
  return duals_create_parts(c, net_id, {{cs, sub}}, dual_prec, out);
}

gcp_status reset_duals(Ctx& c, Batch& b, bool a, bool be, bool g) {
  cudaStream_t st = c.stream;
  const Net& net = *b.net;
  const size_t es = b.fp64 ? 8 : 4;
  SplitsDev sp{b.sp_ptr, b.sp_layer, b.sp_index, b.sp_sign, b.nsp, b.sp_tab};
  if (a)
    for (int i = 1; i < net.L; ++i) {
      if (b.fp64)
        default_alpha<double>(st, b.R, b.K, net.dims[i], i, net.lo64[i - 1], net.hi64[i - 1], sp, (double*)b.alpha[i - 1]);
      else
        default_alpha<float>(st, b.R, b.K, net.dims[i], i, net.lo32[i - 1], net.hi32[i - 1], sp, (float*)b.alpha[i - 1]);
    }
  if (be) cudaMemsetAsync(b.beta, 0, (size_t)std::max(b.M, 1) * b.R * es, st);
  if (g) cudaMemsetAsync(b.gamma, 0, (size_t)std::max(b.N, 1) * b.R * es, st);
  {
    std::string e = reg_take_error();
    if (!e.empty()) return c.fail(GCP_EDEVICE, "reset duals: %s", e.c_str());
  }
  // Adam moments restart with the duals
  for (const char* nm : {"m_alpha", "v_alpha", "m_beta", "v_beta", "m_gamma", "v_gamma"}) {
    auto it = b.lazy.find(nm);
    if (it != b.lazy.end()) cudaMemsetAsync(it->second, 0, b.lazy_bytes[nm], st);
  }
  return c.cuda(cudaGetLastError(), "reset duals");
}

// ------------------------------------------------------------------ chain drivers
template <typename T>
struct TSel;
template <>
struct TSel<double> {
  static const double* lo(const Net& n, int i) { return n.lo64[i - 1]; }
  static const double* hi(const Net& n, int i) { return n.hi64[i - 1]; }
  static const double* inv(const Net& n, int i) { return n.invul64[i - 1]; }
  static const double* b(const Net& n, int i) { return n.b64[i - 1]; }
  static const double* xlo(const Net& n) { return n.xlo64; }
  static const double* xhi(const Net& n) { return n.xhi64; }
  static const double* YL(const Net& n) { return n.YL64; }
  static const double* cb(const Net& n) { return n.cb64; }
  static const double* coef(const CutDev& c) { return c.csc_coef64; }
  static const double* d(const CutDev& c) { return c.d64; }
};
template <>
struct TSel<float> {
  static const float* lo(const Net& n, int i) { return n.lo32[i - 1]; }
  static const float* hi(const Net& n, int i) { return n.hi32[i - 1]; }
  static const float* inv(const Net& n, int i) { return n.invul32[i - 1]; }
  static const float* b(const Net& n, int i) { return n.b32[i - 1]; }
  static const float* xlo(const Net& n) { return n.xlo32; }
  static const float* xhi(const Net& n) { return n.xhi32; }
  static const float* YL(const Net& n) { return n.YL32; }
  static const float* cb(const Net& n) { return n.cb32; }
  static const float* coef(const CutDev& c) { return c.csc_coef32; }
  static const float* d(const CutDev& c) { return c.d32; }
};
template <typename Top>
struct WSel;
template <>
struct WSel<double> {
  static const double* W(const Net& n, int i) { return n.W64[i - 1]; }
  static const double* WT(const Net& n, int i) { return n.WT64[i - 1]; }
};
template <>
struct WSel<float> {
  static const float* W(const Net& n, int i) { return n.W32[i - 1]; }
  static const float* WT(const Net& n, int i) { return n.WT32[i - 1]; }
};
template <>
struct WSel<__nv_bfloat16> {
  static const __nv_bfloat16* W(const Net& n, int i) { return n.W16[i - 1]; }
  static const __nv_bfloat16* WT(const Net& n, int i) { return n.WT16[i - 1]; }
};

template <typename T>
CutCSC<T> csc_of(const Batch& b, int layer) {
  const CutDev& c = b.cuts;
  return CutCSC<T>{c.csc_ptr + c.poff[layer], c.csc_cut, c.csc_kind, TSel<T>::coef(c), c.csc_eid, c.csc_nrn,
                   c.layer_nnz.empty() ? 0 : c.layer_nnz[layer], c.nnz,
                   c.span4_max.empty() ? 0 : c.span4_max[layer]};
}

int64_t Batch::dmax() const {
  int64_t m = 1;
  for (int i = 0; i < net->L; ++i) m = std::max<int64_t>(m, net->dims[i]);
  return m;
}
int Batch::n_partials() const {
  int p = 0;
  for (int i = 0; i < net->L; ++i) p += (net->dims[i] + kChunk - 1) / kChunk;
  return p;
}

// Tensor-core GEMMs per operand type (none for the float64 chain).
template <typename Top>
struct TcOps {
  static bool ok(int) { return false; }
  static bool bwd(cudaStream_t, const Net&, int, int64_t, const Top*, const float*, float*) { return false; }
  static bool fwd(cudaStream_t, const Net&, int, int64_t, const Top*, const float*, float*) { return false; }
};
template <>
struct TcOps<float> {
  static bool ok(int K) { return tc_available(K, false); }
  static bool bwd(cudaStream_t st, const Net& n, int i, int64_t R, const float* a, const float* alo, float* y) {
    const LayerGeom& g = n.geom[i - 1];
    return gemm_tc_tf32x3(st, R, g.d_in, g.d_out, a, n.WT32hi[i - 1], n.WT32lo[i - 1], y);
  }
  static bool fwd(cudaStream_t st, const Net& n, int i, int64_t R, const float* a, const float* alo, float* y) {
    const LayerGeom& g = n.geom[i - 1];
    return gemm_tc_tf32x3(st, R, g.d_out, g.d_in, a, n.W32hi[i - 1], n.W32lo[i - 1], y);
  }
};
template <>
struct TcOps<__nv_bfloat16> {
  static bool ok(int K) { return tc_available(K, true); }
  static bool bwd(cudaStream_t st, const Net& n, int i, int64_t R, const __nv_bfloat16* a, const float*, float* y) {
    const LayerGeom& g = n.geom[i - 1];
    return gemm_tc_bf16(st, R, g.d_in, g.d_out, a, n.WT16[i - 1], y);
  }
  static bool fwd(cudaStream_t st, const Net& n, int i, int64_t R, const __nv_bfloat16* a, const float*, float* y) {
    const LayerGeom& g = n.geom[i - 1];
    return gemm_tc_bf16(st, R, g.d_out, g.d_in, a, n.W16[i - 1], y);
  }
};

// Does the backward product through W^(i) (K = d_i) / the forward product
// through W^(i) (K = d_{i-1}) run on the tensor cores?
// (i: a layer, or the map index of a projection shortcut)
template <typename Top>
static bool tc_bwd(const Batch& b, int i) {
  const LayerGeom& g = b.net->geom[i - 1];
  return b.tc && g.kind == GCP_DENSE && TcOps<Top>::ok(g.d_out);
}
template <typename Top>
static bool tc_fwd(const Batch& b, int i) {
  const LayerGeom& g = b.net->geom[i - 1];
  return b.tc && i != b.net->L && g.kind == GCP_DENSE && TcOps<Top>::ok(g.d_in);
}

// Linear backward step y^(i-1) = W^(i)^T nu^(i) for all rows.
template <typename Top, typename T>
static void lin_backward(cudaStream_t st, const Batch& b, int i, const Top* nu, const float* nu_lo, T* y) {
  const Net& net = *b.net;
  const LayerGeom& g = net.geom[i - 1];
  if constexpr (!std::is_same<T, double>::value) {
    if (tc_bwd<Top>(b, i) && TcOps<Top>::bwd(st, net, i, b.R, nu, nu_lo, y)) return;
  }
  if constexpr (std::is_same<Top, __nv_bfloat16>::value) {
    if (g.kind != GCP_DENSE && b.tc &&
        conv_tc_bf16(st, b.R, g, 1, net.CT16[i - 1], net.ct_kp[i - 1], net.ct_np[i - 1], nu, y))
      return;
  }
  if (g.kind == GCP_DENSE) gemm_nt<Top, T>(st, b.R, g.d_in, g.d_out, nu, 0, WSel<Top>::WT(net, i), y);
  else conv_T<Top, T>(st, b.R, g, WSel<Top>::W(net, i), nu, y);
}
// The mixed-precision chain (bf16 operands, float accumulation) runs the
// backward product through W^(i) as one tensor-core product of three bf16
// terms concatenated along K (kTerms): [nu_hi | nu_lo | nu_hi] against
// [W_hi | W_hi | W_lo], i.e. nu_hi W_hi + nu_lo W_hi + nu_hi W_lo, whose
// operands keep about 16 significant bits each. A single bf16 rounding of nu
// or of W, passed down the chain, moves the bound by up to a few 1e-3 of
// max(|g|, 1) on networks whose bounds sit near zero. Products that have no
// tensor-core form take nu in float on the SIMT units.
template <typename Top>
static bool split_bwd(const Batch& b, int i) {
  if constexpr (!std::is_same<Top, __nv_bfloat16>::value) {
    return false;
  } else {
    const Net& n = *b.net;
    return b.tc && (n.geom[i - 1].kind == GCP_DENSE ? n.WT16x3[i - 1] != nullptr : n.CT16s[i - 1] != nullptr);
  }
}
// y = W^(i)^T nu in the mixed-precision chain, from the three-term operand
// nu2 [R, kTerms d_i] or from nu in float. false: a tensor-core launch was refused.
// The operand's term count a map's tensor-core product takes.
static int map_terms(const Net& n, int i) { return n.geom[i - 1].kind == GCP_DENSE ? kDenseTerms : kConvTerms; }

template <typename Top, typename T>
static bool lin_backward_mixed(cudaStream_t st, const Batch& b, int i, const Top* nu2, int terms, const T* full,
                               T* y) {
  if constexpr (std::is_same<Top, __nv_bfloat16>::value && std::is_same<T, float>::value) {
    const Net& net = *b.net;
    const LayerGeom& g = net.geom[i - 1];
    if (split_bwd<Top>(b, i) && nu2 && terms == map_terms(net, i)) {
      if (g.kind == GCP_DENSE)
        return gemm_tc_bf16(st, b.R, g.d_in, kDenseTerms * g.d_out, nu2, net.WT16x3[i - 1], y, 1.0 / kDenseTerms);
      return conv_tc_bf16(st, b.R, split_geom(g), 1, net.CT16s[i - 1], net.cts_kp[i - 1], net.cts_np[i - 1], nu2, y,
                          1.0 / kConvTerms, &net.CTs_b2[i - 1]);
    }
    if (g.kind == GCP_DENSE) gemm_nt<float, float>(st, b.R, g.d_in, g.d_out, full, 0, net.WT32[i - 1], y);
    else conv_T<float, float>(st, b.R, g, net.W32[i - 1], full, y);
    return true;
  }
  return false;
}
// Which of nu's forms layer i's relaxation writes in the mixed-precision
// chain: the three-term operand for tensor-core products (the layer's, or its
// projection shortcut's), float for SIMT products and identity skips.
template <typename Top>
static void mixed_forms(const Batch& b, int i, bool& split, bool& full, int& terms) {
  const Net& net = *b.net;
  const int sc = net.skip[i - 1] ? net.sc_map[i - 1] : 0;
  const bool ident = net.skip[i - 1] && !sc;
  const bool sp_i = split_bwd<Top>(b, i), sp_sc = sc && split_bwd<Top>(b, sc);
  // one operand layout serves the layer's product and its shortcut's; a
  // consumer that wants the other layout takes nu in float
  terms = sp_i ? map_terms(net, i) : (sp_sc ? map_terms(net, sc) : kDenseTerms);
  const bool use_i = sp_i && map_terms(net, i) == terms, use_sc = sp_sc && map_terms(net, sc) == terms;
  split = use_i || use_sc;
  full = !use_i || ident || (sc && !use_sc);
}

// Linear forward step nubar^(i) = W^(i) a for all rows.
template <typename Top, typename T>
static void lin_forward(cudaStream_t st, const Batch& b, int i, const Top* a, const float* a_lo, T* out) {
  const Net& net = *b.net;
  const LayerGeom& g = net.geom[i - 1];
  if constexpr (!std::is_same<T, double>::value) {
    if (tc_fwd<Top>(b, i) && TcOps<Top>::fwd(st, net, i, b.R, a, a_lo, out)) return;
  }
  if constexpr (std::is_same<Top, __nv_bfloat16>::value) {
    // a layer with fewer than 8 input channels (the input layer) fills at most
    // a quarter of an implicit-GEMM K block: float SIMT is faster there (CNN
    // input layer: 1.58 -> 1.36 ms per launch)
    if (g.kind != GCP_DENSE && b.tc && g.c_in >= 8 &&
        conv_tc_bf16(st, b.R, g, 0, net.CF16[i - 1], net.cf_kp[i - 1], net.cf_np[i - 1], a, out))
      return;
  }
  if (g.kind == GCP_DENSE) gemm_nt<Top, T>(st, b.R, g.d_out, g.d_in, a, 0, WSel<Top>::W(net, i), out);
  else conv_fwd<Top, T>(st, b.R, g, WSel<Top>::W(net, i), a, out);
}

// Skip connections in the backward pass (Theorem 3.1 with the shortcut S as
// one more linear map): once y^(i-1) = W^(i)^T nu^(i) is formed, S^T nu^(i) of
// a skip from xhat^(i-1) joins it; that of a skip from further back is parked
// until its y^(m) exists (nu^(i) itself for the identity, S^T nu^(i) in the
// chain's accumulation type for a projection); y^(i-1) then takes what was
// parked for it, or -S^T c_k when the last layer adds xhat^(i-1) (from L-1
// that is already folded into YL). In the mixed-precision chain (operand type
// narrower than T) an identity skip takes nu in T (nu_full), not the operand
// copy: an identity passes its term unaveraged into y^(m), so an operand
// rounding there would reach the bound at full size.
template <typename Top, typename T>
static gcp_status skip_backward(Ctx& c, Batch& b, cudaStream_t st, int i, const Top* nu, const Top* nu2,
                                int nu2_terms, const T* nu_full, T* y, const T* SK) {
  const Net& net = *b.net;
  const int L = net.L;
  const int64_t R = b.R;
  gcp_status s = GCP_OK;
  const int si = net.skip[i - 1], sc = net.sc_map[i - 1];
  if (si) {
    const int m = si - 1, dm = net.dims[m];
    if (sc) {
      T* dst = si == i ? (T*)b.ws("skip_tmp", (size_t)R * b.dmax() * sizeof(T), &s)
                       : (T*)b.ws("skipT" + std::to_string(m), (size_t)R * dm * sizeof(T), &s);
      if (!dst) return s;
      if (!std::is_same<Top, T>::value) {
        if (!lin_backward_mixed<Top, T>(st, b, sc, nu2, nu2_terms, nu_full, dst))
          return c.fail(GCP_EDEVICE, "projection of layer %d: tensor-core product refused", i);
      } else {
        lin_backward<Top, T>(st, b, sc, nu, nullptr, dst);
      }
      if (si == i) skip_add<T, T>(st, R, dm, dm, 0, dst, 0, y);
    } else if (nu_full && si == i) {
      skip_add<T, T>(st, R, dm, dm, 0, nu_full, 0, y);
    } else if (nu_full) {
      T* park = (T*)b.ws("skipT" + std::to_string(m), (size_t)R * dm * sizeof(T), &s);
      if (!park) return s;
      cudaMemcpyAsync(park, nu_full, (size_t)R * dm * sizeof(T), cudaMemcpyDeviceToDevice, st);
    } else if (si == i) {
      skip_add<Top, T>(st, R, dm, dm, 0, nu, 0, y);
    } else {
      Top* park = (Top*)b.ws("skip" + std::to_string(m), (size_t)R * dm * sizeof(Top), &s);
      if (!park) return s;
      cudaMemcpyAsync(park, nu, (size_t)R * dm * sizeof(Top), cudaMemcpyDeviceToDevice, st);
    }
  }
  const int k = net.consumer[i - 1], dm = net.dims[i - 1];
  if (k == L && i - 1 < L - 1) {
    skip_add<T, T>(st, R, dm, dm, 0, SK, b.K, y);
  } else if (k > i && k < L && (net.sc_map[k - 1] || !std::is_same<Top, T>::value)) {
    const T* park = (const T*)b.ws("skipT" + std::to_string(i - 1), (size_t)R * dm * sizeof(T), &s);
    if (!park) return s;
    skip_add<T, T>(st, R, dm, dm, 0, park, 0, y);
  } else if (k > i && k < L) {
    const Top* park = (const Top*)b.ws("skip" + std::to_string(i - 1), (size_t)R * dm * sizeof(Top), &s);
    if (!park) return s;
    skip_add<Top, T>(st, R, dm, dm, 0, park, 0, y);
  }
  return GCP_OK;
}

template <typename T>
static const T* spec_skip(const Net& n);
template <>
const double* spec_skip<double>(const Net& n) { return n.SK64; }
template <>
const float* spec_skip<float>(const Net& n) { return n.SK32; }

// The directly optimised ReLU duals theta (pi = theta [nuhat]_+) of the batch,
// layer i's block at R * (d_1 + .. + d_{i-1}); nullptr while the batch uses
// Lemma A.1's closed form.
template <typename T>
static T* theta_of(Batch& b, int i) {
  if (!b.theta_on) return nullptr;
  auto it = b.lazy.find("theta");
  if (it == b.lazy.end()) return nullptr;
  int64_t off = 0;
  for (int q = 1; q < i; ++q) off += b.R * b.net->dims[q];
  return (T*)it->second + off;
}

// Stored or recomputed nuhat for the adjoint. Storing costs R * (d_1 + ..
// + d_{L-1}) values; recomputing needs three buffers of the widest hidden
// layer and re-runs the evaluation from the top down to each layer (about
// L/2 times the evaluation's work). The adjoint recomputes when the memory
// budget cannot hold the stored copies and recomputing saves memory, or when
// GCP_NUHAT=recompute asks for it; not for networks with skip connections
// (their parked terms share the evaluation's buffers).
static bool want_recompute(const Ctx& c, const Batch& b, size_t es) {
  const Net& net = *b.net;
  for (int i = 0; i < net.L; ++i)
    if (net.skip[i]) return false;
  const char* e = std::getenv("GCP_NUHAT");
  if (e && std::strcmp(e, "recompute") == 0) return true;
  if (e && std::strcmp(e, "store") == 0) return false;
  int64_t sum = 0, mx = 0;
  for (int i = 1; i < net.L; ++i) {
    sum += net.dims[i];
    mx = std::max<int64_t>(mx, net.dims[i]);
  }
  if (!c.budget || 3 * mx >= sum) return false;
  return c.used + (uint64_t)b.R * sum * es > c.budget;
}

static int64_t max_hidden(const Net& net) {
  int64_t mx = 1;
  for (int i = 1; i < net.L; ++i) mx = std::max<int64_t>(mx, net.dims[i]);
  return mx;
}

// nuhat^(target) recomputed: the evaluation's layers from the top down to
// `target` (no objective), on buffers of its own; the duals of these layers
// are the ones the evaluation used (the adjoint steps them after this call).
template <typename T, typename Top>
static const T* recompute_nuhat(Ctx& c, Batch& b, cudaStream_t st, int target, gcp_status* s) {
  const Net& net = *b.net;
  const int L = net.L;
  const int64_t R = b.R, mh = max_hidden(net);
  Top* nu = (Top*)b.ws("rc_nu", (size_t)R * mh * sizeof(Top), s);
  T* y = nu ? (T*)b.ws("rc_y", (size_t)R * mh * sizeof(T), s) : nullptr;
  T* nh = y ? (T*)b.ws("rc_nuhat", (size_t)R * mh * sizeof(T), s) : nullptr;
  if (!nh) return nullptr;
  SplitsDev sp{b.sp_ptr, b.sp_layer, b.sp_index, b.sp_sign, b.nsp, b.sp_tab};
  for (int i = L - 1; i >= target; --i) {
    RelaxArgs<T, Top> a{};
    a.R = R; a.K = b.K; a.d = net.dims[i]; a.layer = i; a.M = b.M; a.N = b.N;
    a.y = (i == L - 1) ? TSel<T>::YL(net) : y;
    a.y_per_spec = (i == L - 1);
    a.lo = TSel<T>::lo(net, i); a.hi = TSel<T>::hi(net, i); a.bias = TSel<T>::b(net, i);
    a.inv_ul = TSel<T>::inv(net, i);
    a.alpha = (const T*)b.alpha[i - 1];
    a.beta = (const T*)b.beta;
    a.gamma = (const T*)b.gamma;
    a.sp = sp;
    a.csc = csc_of<T>(b, i);
    a.nu_out = nu;
    a.nuhat_out = nh;
    a.theta = theta_of<T>(b, i);
    if (!std::is_same<Top, T>::value && i > target) {
      bool sp = false, fu = false;
      mixed_forms<Top>(b, i, sp, fu, a.split_terms);
      a.nu_out = nullptr;
      if (sp && !(a.nu_split = (Top*)b.ws("rc_nu2", (size_t)R * kMaxTerms * mh * sizeof(Top), s))) return nullptr;
      if (fu && !(a.nu_full = (T*)b.ws("rc_nu_full", (size_t)R * mh * sizeof(T), s))) return nullptr;
    }
    relax_eval<T, Top>(st, a);
    if (i > target) {
      if (!std::is_same<Top, T>::value) {
        if (!lin_backward_mixed<Top, T>(st, b, i, a.nu_split, a.split_terms, a.nu_full, y)) {
          *s = c.fail(GCP_EDEVICE, "layer %d: tensor-core product refused", i);
          return nullptr;
        }
      } else {
        lin_backward<Top, T>(st, b, i, nu, nullptr, y);
      }
    }
  }
  return nh;
}

// Evaluate g for all rows at the batch's duals. with_adjoint_start: also write
// a0 = -seed*x* into the operand buffer and the input-layer cut entries into E.
// finalize = false leaves g itself out (ascent steps need only the gradient).
template <typename T, typename Top>
gcp_status run_eval(Ctx& c, Batch& b, cudaStream_t st, bool with_adjoint_start, const T* seed,
                    bool finalize = true, bool theta_init = false) {
  const Net& net = *b.net;
  const int L = net.L;
  const int64_t R = b.R;
  gcp_status s = GCP_OK;
  Top* nu = (Top*)b.ws("nu", (size_t)R * b.dmax() * sizeof(Top), &s);
  if (!nu) return s;
  T* y = (T*)b.ws("y", (size_t)R * b.dmax() * sizeof(T), &s);
  if (!y) return s;
  T* part = (T*)b.ws("obj_part", (size_t)b.n_partials() * R * sizeof(T), &s);
  if (!part) return s;
  T* g = (T*)b.ws("g", (size_t)std::max<int64_t>(R, 1) * sizeof(T), &s);
  if (!g) return s;
  float* lo = nullptr;   // no tf32 low plane: the tensor-core GEMM splits fp32 operands itself
  T* E = nullptr;
  if (with_adjoint_start && b.nnz) {
    E = (T*)b.ws("E", (size_t)b.nnz * R * sizeof(T), &s);
    if (!E) return s;
  }
  SplitsDev sp{b.sp_ptr, b.sp_layer, b.sp_index, b.sp_sign, b.nsp, b.sp_tab};
  if (with_adjoint_start && !b.recompute_decided) {
    b.recompute = want_recompute(c, b, sizeof(T));
    b.recompute_decided = true;
  }
  // nuhat per layer only where the adjoint will read it; otherwise one scratch row block
  const bool keep = (with_adjoint_start || b.keep_nuhat) && !b.recompute;
  int poff = 0;
  for (int i = L - 1; i >= 1; --i) {
    T* nuhat = keep ? (T*)b.ws("nuhat" + std::to_string(i), (size_t)R * net.dims[i] * sizeof(T), &s)
                    : (T*)b.ws("rc_nuhat", (size_t)R * max_hidden(net) * sizeof(T), &s);
    if (!nuhat) return s;
    RelaxArgs<T, Top> a{};
    a.R = R; a.K = b.K; a.d = net.dims[i]; a.layer = i; a.M = b.M; a.N = b.N;
    a.y = (i == L - 1) ? TSel<T>::YL(net) : y;
    a.y_per_spec = (i == L - 1);
    a.lo = TSel<T>::lo(net, i); a.hi = TSel<T>::hi(net, i); a.bias = TSel<T>::b(net, i);
    a.inv_ul = TSel<T>::inv(net, i);
    a.alpha = (const T*)b.alpha[i - 1];
    a.beta = (const T*)b.beta;
    a.gamma = (const T*)b.gamma;
    a.sp = sp;
    a.csc = csc_of<T>(b, i);
    a.nu_out = nu;
    a.nu_lo = (lo && tc_bwd<Top>(b, i)) ? lo : nullptr;
    a.nuhat_out = nuhat;
    a.obj_part = finalize ? part + (int64_t)poff * R : nullptr;   // ascent steps need no objective
    a.theta = theta_of<T>(b, i);
    a.theta_init = theta_init;
    if (!std::is_same<Top, T>::value) {
      bool sp = false, fu = false;
      mixed_forms<Top>(b, i, sp, fu, a.split_terms);
      a.nu_out = nullptr;
      if (sp && !(a.nu_split = (Top*)b.ws("nu2", (size_t)R * kMaxTerms * b.dmax() * sizeof(Top), &s))) return s;
      if (fu && !(a.nu_full = (T*)b.ws("nu_full", (size_t)R * b.dmax() * sizeof(T), &s))) return s;
    }
    relax_eval<T, Top>(st, a);
    poff += (net.dims[i] + kChunk - 1) / kChunk;
    if (!std::is_same<Top, T>::value) {
      if (!lin_backward_mixed<Top, T>(st, b, i, a.nu_split, a.split_terms, a.nu_full, y))
        return c.fail(GCP_EDEVICE, "layer %d: tensor-core product refused", i);
    } else {
      lin_backward<Top, T>(st, b, i, nu, a.nu_lo, y);
    }
    s = skip_backward<Top, T>(c, b, st, i, nu, a.nu_split, a.split_terms, a.nu_full, y, spec_skip<T>(net));
    if (s) return s;
  }
  ConcArgs<T, Top> ca{};
  ca.R = R; ca.K = b.K; ca.d0 = net.dims[0]; ca.N = b.N;
  ca.y0 = y;
  ca.x_lo = TSel<T>::xlo(net); ca.x_hi = TSel<T>::xhi(net);
  ca.gamma = (const T*)b.gamma;
  ca.seed = seed;
  ca.csc = csc_of<T>(b, 0);
  ca.a0_out = with_adjoint_start ? nu : nullptr;
  ca.a0_lo = (with_adjoint_start && lo && tc_fwd<Top>(b, 1)) ? lo : nullptr;
  ca.E = E;
  ca.obj_part = finalize ? part + (int64_t)poff * R : nullptr;
  concretize<T, Top>(st, ca);
  poff += (net.dims[0] + kChunk - 1) / kChunk;
  if (finalize) {
    FinalArgs<T> fa{R, b.K, b.N, poff, TSel<T>::cb(net), TSel<T>::d(b.cuts), (const T*)b.gamma, part, g};
    finalize_bound<T>(st, fa);
  }
  return launch_status(c, "eval");
}

// Reverse pass after run_eval(with_adjoint_start): gradients or an update step.
template <typename T, typename Top>
gcp_status run_adjoint(Ctx& c, Batch& b, cudaStream_t st, const StepArgs<T>& step, const T* seed, T* gal, T* gbe,
                       T* gga) {
  const Net& net = *b.net;
  const int L = net.L;
  const int64_t R = b.R;
  gcp_status s = GCP_OK;
  Top* abuf = (Top*)b.ws("nu", (size_t)R * b.dmax() * sizeof(Top), &s);
  T* y = (T*)b.ws("y", (size_t)R * b.dmax() * sizeof(T), &s);
  if (!abuf || !y) return s;
  T* E = b.nnz ? (T*)b.ws("E", (size_t)b.nnz * R * sizeof(T), &s) : nullptr;
  if (b.nnz && !E) return s;
  float* lo = nullptr;   // no tf32 low plane: the tensor-core GEMM splits fp32 operands itself
  T *ma = nullptr, *va = nullptr, *mb = nullptr, *vb = nullptr, *mg = nullptr, *vg = nullptr;
  int64_t nal = 0;
  for (int i = 1; i < L; ++i) nal += (int64_t)R * net.dims[i];
  if (step.mode == 2) {
    const size_t ab = (size_t)nal * sizeof(T), bb = (size_t)std::max(b.M, 1) * R * sizeof(T),
                 gb = (size_t)std::max(b.N, 1) * R * sizeof(T);
    bool fresh = b.lazy.find("m_alpha") == b.lazy.end();
    ma = (T*)b.ws("m_alpha", ab, &s); va = (T*)b.ws("v_alpha", ab, &s);
    mb = (T*)b.ws("m_beta", bb, &s); vb = (T*)b.ws("v_beta", bb, &s);
    mg = (T*)b.ws("m_gamma", gb, &s); vg = (T*)b.ws("v_gamma", gb, &s);
    if (!ma || !va || !mb || !vb || !mg || !vg) return s;
    if (fresh) {
      cudaMemsetAsync(ma, 0, ab, st); cudaMemsetAsync(va, 0, ab, st);
      cudaMemsetAsync(mb, 0, bb, st); cudaMemsetAsync(vb, 0, bb, st);
      cudaMemsetAsync(mg, 0, gb, st); cudaMemsetAsync(vg, 0, gb, st);
    }
  }
  SplitsDev sp{b.sp_ptr, b.sp_layer, b.sp_index, b.sp_sign, b.nsp, b.sp_tab};
  if (!gbe && b.M > 0) {   // ascent step: dg/dbeta goes through a workspace to the beta step
    gbe = (T*)b.ws("g_beta_step", (size_t)b.M * R * sizeof(T), &s);
    if (!gbe) return s;
  }
  // skips in the reverse pass: dg/dnu^(k) gains dg/dy^(m), the adjoint a^(m)
  // of the xhat^(m) that layer k adds; a^(m) is parked when a later layer needs it
  auto park_a = [&](int m) -> gcp_status {
    const int k = net.consumer[m];
    if (k <= m + 1 || k >= L) return GCP_OK;
    Top* park = (Top*)b.ws("skip" + std::to_string(m), (size_t)R * net.dims[m] * sizeof(Top), &s);
    if (!park) return s;
    cudaMemcpyAsync(park, abuf, (size_t)R * net.dims[m] * sizeof(Top), cudaMemcpyDeviceToDevice, st);
    return GCP_OK;
  };
  s = park_a(0);
  if (s) return s;
  int64_t aoff = 0;
  for (int i = 1; i < L; ++i) {
    lin_forward<Top, T>(st, b, i, abuf, (lo && tc_fwd<Top>(b, i)) ? lo : nullptr, y);
    if (const int si = net.skip[i - 1]) {
      const Top* src = abuf;
      if (si < i) {
        src = (const Top*)b.ws("skip" + std::to_string(si - 1), (size_t)R * net.dims[si - 1] * sizeof(Top), &s);
        if (!src) return s;
      }
      if (const int sc = net.sc_map[i - 1]) {   // + S a^(m) through the shortcut's own product
        T* tmp = (T*)b.ws("skip_tmp", (size_t)R * b.dmax() * sizeof(T), &s);
        if (!tmp) return s;
        lin_forward<Top, T>(st, b, sc, src, nullptr, tmp);
        skip_add<T, T>(st, R, net.dims[i], net.dims[i], 0, tmp, 0, y);
      } else {
        skip_add<Top, T>(st, R, net.dims[i], net.dims[i], 0, src, 0, y);
      }
    }
    const T* nuhat = b.recompute ? recompute_nuhat<T, Top>(c, b, st, i, &s)
                                 : (const T*)b.lazy["nuhat" + std::to_string(i)];
    if (!nuhat) return s;
    AdjArgs<T, Top> a{};
    a.R = R; a.K = b.K; a.d = net.dims[i]; a.layer = i; a.M = b.M; a.N = b.N;
    a.nubar = y; a.seed = seed;
    a.lo = TSel<T>::lo(net, i); a.hi = TSel<T>::hi(net, i); a.bias = TSel<T>::b(net, i);
    a.inv_ul = TSel<T>::inv(net, i);
    a.alpha = (T*)b.alpha[i - 1];
    a.gamma = (const T*)b.gamma;
    a.nuhat = nuhat;
    a.sp = sp;
    a.csc = csc_of<T>(b, i);
    a.a_out = (i < L - 1) ? abuf : nullptr;
    a.a_lo = (lo && i < L - 1 && tc_fwd<Top>(b, i + 1)) ? lo : nullptr;
    a.E = E;
    a.g_alpha = gal ? gal + aoff : nullptr;
    a.g_beta = gbe;
    if (ma) { a.m_alpha = ma + aoff; a.v_alpha = va + aoff; }
    a.st = step;
    if ((a.theta = theta_of<T>(b, i))) {
      a.g_theta = nullptr;
      if (step.mode == 2) {
        a.m_theta = (T*)b.lazy["m_theta"] + aoff;
        a.v_theta = (T*)b.lazy["v_theta"] + aoff;
      }
    }
    relax_adjoint<T, Top>(st, a);
    aoff += (int64_t)R * net.dims[i];
    if (i < L - 1) {
      s = park_a(i);
      if (s) return s;
    }
  }
  if (b.N > 0 || (b.M > 0 && step.mode != 0)) {
    GatherArgs<T> ga{R, b.N, b.cuts.cut_ptr, b.cuts.csr_pos, E, TSel<T>::d(b.cuts), seed, (T*)b.gamma, gga, mg, vg,
                     step, b.nnz, b.K, b.sub_cut_lo, b.sub_cut_hi,
                     b.M, b.sp_tab, (T*)b.beta, gbe, mb, vb};
    gather_gamma<T>(st, ga);
  }
  return launch_status(c, "adjoint");
}

// Float64 certification pass with outward rounding (rigorous lower bound).
template <typename Td>
gcp_status run_certify(Ctx& c, Batch& b, cudaStream_t st, double* out_dev) {
  const Net& net = *b.net;
  const int L = net.L;
  const int n_maps = (int)net.geom.size();   // the layers, then the projection shortcuts
  const int64_t R = b.R;
  gcp_status s = GCP_OK;
  double* nu = (double*)b.ws("c_nu", (size_t)R * b.dmax() * 8, &s);
  double* y = (double*)b.ws("c_y", (size_t)R * b.dmax() * 8, &s);
  float* ya = (float*)b.ws("c_yabs", (size_t)R * b.dmax() * 4, &s);
  double* part = (double*)b.ws("c_part", (size_t)b.n_partials() * R * 8, &s);
  if (!nu || !y || !ya || !part) return s;
  bool any_conv = false;
  for (int i = 0; i < n_maps; ++i) any_conv |= net.geom[i].kind != GCP_DENSE;
  float* nuabs = nullptr;
  if (any_conv) {
    nuabs = (float*)b.ws("c_nuabs", (size_t)R * b.dmax() * 4, &s);
    if (!nuabs) return s;
  }
  // slices of nu for the dense products on the tensor cores
  __nv_bfloat16* nu_sl = nullptr;
  int32_t* nu_ex = nullptr;
  float* sl_sums = nullptr;
  size_t sl_elems = 0, sum_elems = 0;
  for (int mi = 1; mi <= n_maps; ++mi) {
    const SliceB& sl = net.WTsl[mi - 1];
    if (mi == L || !b.tc || !sl.planes) continue;
    sl_elems = std::max(sl_elems, (size_t)sl.s * net.geom[mi - 1].d_out);
    sum_elems = std::max(sum_elems, (size_t)sl.s * net.geom[mi - 1].d_in);
  }
  if (sl_elems) {
    nu_sl = (__nv_bfloat16*)b.ws("c_nu_slices", (size_t)R * sl_elems * 2, &s);
    nu_ex = (int32_t*)b.ws("c_nu_exps", (size_t)R * 4, &s);
    sl_sums = (float*)b.ws("c_slice_sums", (size_t)R * sum_elems * 4, &s);
    if (!nu_sl || !nu_ex || !sl_sums) return s;
  }
  // yo = M^T nu for all rows through map mi (a layer or a shortcut) with
  // yao >= |M|^T |nu|; returns e with |yo - exact| <= e * yao: Higham's
  // gamma_K for the float64 dot products, the slice bound on the tensor cores
  auto product = [&](int mi, double* yo, float* yao) -> double {
    const LayerGeom& g = net.geom[mi - 1];
    const SliceB& sl = net.WTsl[mi - 1];
    if (g.kind == GCP_DENSE && b.tc && sl.planes &&
        gemm_f64_slices(st, R, g.d_in, g.d_out, nu, sl, nu_sl, nu_ex, sl_sums, yo, yao))
      return sl.cerr;
    if (g.kind == GCP_DENSE) gemm_nt_abs(st, R, g.d_in, g.d_out, nu, 0, net.WT64[mi - 1], yo, yao);
    else conv_T_abs(st, R, g, net.W64[mi - 1], net.Wabs32[mi - 1], nu, nuabs, yo, yao);
    return gamma_n_host(red_len(g));
  };
  // adding a term t with |t - exact| <= e_t * ta to y: |fl(y + t) - exact| <=
  // yerr ya + e_t ta + u (|y| + |t|) <= (max(yerr, e_t) + 2u) (ya + ta), and
  // ya grows by ta (|t| for an exact t)
  auto skip_err = [](double e, double e_t) {
    return std::nextafter(std::max(e, e_t) + std::ldexp(1.0, -52), INFINITY);
  };
  std::map<int, double> parked_err;       // error factor of the term parked for y^(m)
  SplitsDev sp{b.sp_ptr, b.sp_layer, b.sp_index, b.sp_sign, b.nsp, b.sp_tab};
  // y^(L-1) = W^(L)^T (-c_k), one row per spec row
  const LayerGeom& gl = net.geom[L - 1];
  const int dL = net.dims[L];
  gemm_nt_abs(st, b.K, gl.d_in, gl.d_out, net.negC64, 0, net.WT64[L - 1], y, ya);
  double yerr = gamma_n_host(red_len(gl));
  // a skip on the last layer: -c_k (identity, exact) or -S^T c_k (certified product)
  double* sk = nullptr;
  float* ska = nullptr;
  if (const int sL = net.skip[L - 1]) {
    const int m = sL - 1, dm = net.dims[m];
    if (const int sc = net.sc_map[L - 1]) {
      sk = (double*)b.ws("c_spec_skip", (size_t)b.K * dm * 8, &s);
      ska = (float*)b.ws("c_spec_skip_abs", (size_t)b.K * dm * 4, &s);
      if (!sk || !ska) return s;
      gemm_nt_abs(st, b.K, dm, dL, net.negC64, 0, net.WT64[sc - 1], sk, ska);
      parked_err[m] = gamma_n_host(dL);
      if (m == L - 1) {
        skip_add_cert(st, b.K, dm, dm, 0, sk, ska, 0, y, ya);
        yerr = skip_err(yerr, parked_err[m]);
      }
    } else if (m == L - 1) {
      skip_add_cert(st, b.K, dL, dm, net.skip_off, net.negC64, nullptr, 0, y, ya);
      yerr = skip_err(yerr, 0.0);
    }
  }
  int poff = 0;
  for (int i = L - 1; i >= 1; --i) {
    const int si = net.skip[i - 1], sc = net.sc_map[i - 1];
    CertArgs<Td> a{};
    a.R = R; a.K = b.K; a.d = net.dims[i]; a.layer = i; a.M = b.M; a.N = b.N;
    a.y = y; a.yabs = ya; a.y_per_spec = (i == L - 1);
    a.gamma_n = yerr;
    a.lo = net.lo64[i - 1]; a.hi = net.hi64[i - 1]; a.bias = net.b64[i - 1];
    a.alpha = (const Td*)b.alpha[i - 1];
    a.beta = (const Td*)b.beta;
    a.gamma = (const Td*)b.gamma;
    a.sp = sp;
    a.csc = csc_of<double>(b, i);
    a.nu_out = nu;
    const LayerGeom& g = net.geom[i - 1];
    const bool conv_here = g.kind != GCP_DENSE || (sc && net.geom[sc - 1].kind != GCP_DENSE);
    a.nuabs_out = conv_here ? nuabs : nullptr;
    a.obj_part = part + (int64_t)poff * R;
    a.theta = theta_of<Td>(b, i);
    certify_relax<Td>(st, a);
    poff += (net.dims[i] + kChunk - 1) / kChunk;
    yerr = product(i, y, ya);
    // skips, as in the chain's backward pass, with the error bound widened
    if (si) {
      const int m = si - 1, dm = net.dims[m];
      if (sc) {
        const std::string nm = si == i ? std::string("c_skip_tmp") : "c_skip" + std::to_string(m);
        double* ys = (double*)b.ws(nm, (size_t)R * b.dmax() * 8, &s);
        float* yas = (float*)b.ws(nm + "_abs", (size_t)R * b.dmax() * 4, &s);
        if (!ys || !yas) return s;
        const double e = product(sc, ys, yas);
        if (si == i) {
          skip_add_cert(st, R, dm, dm, 0, ys, yas, 0, y, ya);
          yerr = skip_err(yerr, e);
        } else {
          parked_err[m] = e;
        }
      } else if (si == i) {
        skip_add_cert(st, R, dm, dm, 0, nu, nullptr, 0, y, ya);
        yerr = skip_err(yerr, 0.0);
      } else {
        double* park = (double*)b.ws("c_skip" + std::to_string(m), (size_t)R * b.dmax() * 8, &s);
        if (!park) return s;
        cudaMemcpyAsync(park, nu, (size_t)R * dm * 8, cudaMemcpyDeviceToDevice, st);
        parked_err[m] = 0.0;
      }
    }
    const int k = net.consumer[i - 1], dm = net.dims[i - 1];
    if (k == L && i - 1 < L - 1) {
      if (sk) skip_add_cert(st, R, dm, dm, 0, sk, ska, b.K, y, ya);
      else skip_add_cert(st, R, dL, dm, net.skip_off, net.negC64, nullptr, b.K, y, ya);
      yerr = skip_err(yerr, sk ? parked_err[i - 1] : 0.0);
    } else if (k > i && k < L) {
      const std::string nm = "c_skip" + std::to_string(i - 1);
      const double* ys = (const double*)b.ws(nm, (size_t)R * b.dmax() * 8, &s);
      const float* yas = net.sc_map[k - 1] ? (const float*)b.ws(nm + "_abs", (size_t)R * b.dmax() * 4, &s) : nullptr;
      if (!ys || (net.sc_map[k - 1] && !yas)) return s;
      skip_add_cert(st, R, dm, dm, 0, ys, yas, 0, y, ya);
      yerr = skip_err(yerr, parked_err[i - 1]);
    }
  }
  certify_concretize<Td>(st, R, b.K, b.N, net.dims[0], y, ya, yerr, net.xlo64,
                         net.xhi64, (const Td*)b.gamma, csc_of<double>(b, 0), part + (int64_t)poff * R);
  poff += (net.dims[0] + kChunk - 1) / kChunk;
  certify_finalize<Td>(st, R, b.K, b.N, poff, net.C64, net.bL64, net.dims[L], b.cuts.d64, (const Td*)b.gamma, part,
                       out_dev);
  return launch_status(c, "certify");
}

template <typename T>
static StepArgs<T> make_step(const gcp_opt_params& p, int it) {
  StepArgs<T> s{};
  s.mode = p.optimizer == GCP_ADAM ? 2 : 1;
  const double f = std::pow(p.lr_decay, (double)it);
  s.lr_a = (T)(p.lr_alpha * f);
  s.lr_b = (T)(p.lr_beta * f);
  s.lr_g = (T)(p.lr_gamma * f);
  s.b1 = (T)0.9;
  s.b2 = (T)0.999;
  s.eps = (T)1e-8;
  s.c1 = (T)(1.0 - std::pow(0.9, it + 1));
  s.c2 = (T)(1.0 - std::pow(0.999, it + 1));
  s.ic1 = (T)(1.0 / (1.0 - std::pow(0.9, it + 1)));
  s.ic2 = (T)(1.0 / (1.0 - std::pow(0.999, it + 1)));
  return s;
}

template <typename T, typename Top>
gcp_status optimize_steps(Ctx& c, Batch& b, cudaStream_t st, const gcp_opt_params& p, bool theta_init) {
  for (int it = 0; it < p.iters; ++it) {
    // theta_init: the first evaluation sets theta from the closed form
    gcp_status s = run_eval<T, Top>(c, b, st, true, nullptr, false, theta_init && it == 0);
    if (s) return s;
    s = run_adjoint<T, Top>(c, b, st, make_step<T>(p, it), nullptr, nullptr, nullptr, nullptr);
    if (s) return s;
  }
  return GCP_OK;
}

gcp_status check_prec(Ctx& c, const Batch& b, int prec) {
  if (prec == GCP_FP64 && !b.fp64) return c.fail(GCP_EINVAL, "FP64 chain needs duals created with GCP_FP64");
  if ((prec == GCP_FP32 || prec == GCP_BF16) && b.fp64) return c.fail(GCP_EINVAL, "FP32/BF16 chain needs GCP_FP32 duals");
  if (prec < 0 || prec > 2) return c.fail(GCP_EINVAL, "unknown precision %d", prec);
  return GCP_OK;
}

// Copy the chain bound (T on device) to host doubles.
static gcp_status fetch_bound(Ctx& c, Batch& b, cudaStream_t st, double* out) {
  if (!out || b.R == 0) return GCP_OK;
  gcp_status s = GCP_OK;
  if (b.fp64) {
    cudaError_t e = cudaMemcpyAsync(out, b.lazy["g"], b.R * 8, cudaMemcpyDeviceToHost, st);
    if (e) return c.cuda(e, "copy bound");
  } else {
    double* tmp = (double*)b.ws("g64", b.R * 8, &s);
    if (!tmp) return s;
    cast_copy<float, double>(st, b.R, (const float*)b.lazy["g"], tmp);
    cudaError_t e = cudaMemcpyAsync(out, tmp, b.R * 8, cudaMemcpyDeviceToHost, st);
    if (e) return c.cuda(e, "copy bound");
  }
  return GCP_OK;
}

gcp_status eval_dispatch(Ctx& c, Batch& b, cudaStream_t st, int prec, bool adj_start, const void* seed,
                         bool theta_init) {
  if (prec == GCP_FP64) return run_eval<double, double>(c, b, st, adj_start, (const double*)seed, true, theta_init);
  if (prec == GCP_FP32) return run_eval<float, float>(c, b, st, adj_start, (const float*)seed, true, theta_init);
  return run_eval<float, __nv_bfloat16>(c, b, st, adj_start, (const float*)seed, true, theta_init);
}

gcp_status certify_dispatch(Ctx& c, Batch& b, cudaStream_t st, double* out_dev) {
  return b.fp64 ? run_certify<double>(c, b, st, out_dev) : run_certify<float>(c, b, st, out_dev);
}

gcp_status bound_batch(Ctx& c, Batch& b, int prec, int certify, double* out_bound, double* out_cert) {
  gcp_status s = check_prec(c, b, prec);
  if (s) return s;
  cudaStream_t st = c.stream;
  if (b.R == 0) return GCP_OK;
  s = eval_dispatch(c, b, st, prec, false, nullptr);
  if (s) return s;
  s = fetch_bound(c, b, st, out_bound);
  if (s) return s;
  if (certify) {
    double* cd = (double*)b.ws("cert", b.R * 8, &s);
    if (!cd) return s;
    s = certify_dispatch(c, b, st, cd);
    if (s) return s;
    if (out_cert) {
      cudaError_t e = cudaMemcpyAsync(out_cert, cd, b.R * 8, cudaMemcpyDeviceToHost, st);
      if (e) return c.cuda(e, "copy certified");
    }
  }
  return sync_check(c, st, "bound_batch");
}

template <typename T>
static gcp_status grad_impl(Ctx& c, Batch& b, int prec, double* out_bound, double* ga, double* gb, double* gg) {
  cudaStream_t st = c.stream;
  const Net& net = *b.net;
  gcp_status s = GCP_OK;
  int64_t nal = 0;
  for (int i = 1; i < net.L; ++i) nal += (int64_t)b.R * net.dims[i];
  T* gal = (T*)b.ws("g_alpha", (size_t)nal * sizeof(T), &s);
  T* gbe = (T*)b.ws("g_beta", (size_t)std::max(b.M, 1) * b.R * sizeof(T), &s);
  T* gga = (T*)b.ws("g_gamma", (size_t)std::max(b.N, 1) * b.R * sizeof(T), &s);
  if (!gal || !gbe || !gga) return s;
  cudaMemsetAsync(gbe, 0, (size_t)std::max(b.M, 1) * b.R * sizeof(T), st);
  s = eval_dispatch(c, b, st, prec, true, nullptr);
  if (s) return s;
  StepArgs<T> step{};
  step.mode = 0;
  if constexpr (std::is_same<T, double>::value) {
    s = run_adjoint<double, double>(c, b, st, step, nullptr, gal, gbe, gga);
  } else {
    s = prec == GCP_FP32 ? run_adjoint<float, float>(c, b, st, step, nullptr, gal, gbe, gga)
                         : run_adjoint<float, __nv_bfloat16>(c, b, st, step, nullptr, gal, gbe, gga);
  }
  if (s) return s;
  s = fetch_bound(c, b, st, out_bound);
  if (s) return s;
  // export layouts: alpha [R, sum d] (layer blocks), beta [R, M], gamma [R, N]
  std::vector<T> h;
  s = sync_check(c, st, "grad_batch");
  if (s) return s;
  cudaError_t e = cudaSuccess;
  if (ga) {
    h.resize(nal);
    e = cudaMemcpy(h.data(), gal, nal * sizeof(T), cudaMemcpyDeviceToHost);
    if (e) return c.cuda(e, "copy g_alpha");
    int64_t cols = 0, off = 0;
    for (int i = 1; i < net.L; ++i) cols += net.dims[i];
    int64_t coff = 0;
    for (int i = 1; i < net.L; ++i) {
      const int di = net.dims[i];
      for (int64_t r = 0; r < b.R; ++r)
        for (int j = 0; j < di; ++j) ga[r * cols + coff + j] = (double)h[off + r * di + j];
      off += b.R * di;
      coff += di;
    }
  }
  if (gb && b.M > 0) {
    h.resize((size_t)b.M * b.R);
    e = cudaMemcpy(h.data(), gbe, h.size() * sizeof(T), cudaMemcpyDeviceToHost);
    if (e) return c.cuda(e, "copy g_beta");
    for (size_t q = 0; q < h.size(); ++q) gb[q] = (double)h[q];
  }
  if (gg && b.N > 0) {
    h.resize((size_t)b.N * b.R);
    e = cudaMemcpy(h.data(), gga, h.size() * sizeof(T), cudaMemcpyDeviceToHost);
    if (e) return c.cuda(e, "copy g_gamma");
    for (size_t q = 0; q < h.size(); ++q) gg[q] = (double)h[q];
  }
  return GCP_OK;
}

gcp_status grad_batch(Ctx& c, Batch& b, int prec, double* out_bound, double* ga, double* gb, double* gg) {
  gcp_status s = check_prec(c, b, prec);
  if (s) return s;
  if (b.R == 0) return GCP_OK;
  return b.fp64 ? grad_impl<double>(c, b, prec, out_bound, ga, gb, gg) : grad_impl<float>(c, b, prec, out_bound, ga, gb, gg);
}

gcp_status optimize_on(Ctx& c, Batch& b, const gcp_opt_params& p, cudaStream_t st, double* cert_dev) {
  gcp_status s = check_prec(c, b, p.prec);
  if (s) return s;
  if (p.iters < 0 || (p.optimizer != GCP_PGA && p.optimizer != GCP_ADAM) || !(p.lr_decay > 0))
    return c.fail(GCP_EINVAL, "bad optimiser parameters");
  if (b.R == 0) return GCP_OK;
  // directly optimised pi (App. A's closing remark): theta continues from the
  // duals' own theta when they hold one, else it starts at the closed form;
  // its Adam moments start afresh in every call
  const bool theta_init = p.opt_pi && !b.theta_on;
  b.theta_on = false;
  if (p.opt_pi) {
    int64_t nal = 0;
    for (int i = 1; i < b.net->L; ++i) nal += b.R * b.net->dims[i];
    const size_t bytes = (size_t)std::max<int64_t>(nal, 1) * (b.fp64 ? 8 : 4);
    if (!b.ws("theta", bytes, &s)) return s;
    if (p.optimizer == GCP_ADAM) {
      void* m = b.ws("m_theta", bytes, &s);
      void* v = m ? b.ws("v_theta", bytes, &s) : nullptr;
      if (!v) return s;
      cudaMemsetAsync(m, 0, bytes, st);
      cudaMemsetAsync(v, 0, bytes, st);
    }
    b.theta_on = true;
  }
  if (p.prec == GCP_FP64) s = optimize_steps<double, double>(c, b, st, p, theta_init);
  else if (p.prec == GCP_FP32) s = optimize_steps<float, float>(c, b, st, p, theta_init);
  else s = optimize_steps<float, __nv_bfloat16>(c, b, st, p, theta_init);
  if (s) return s;
  s = eval_dispatch(c, b, st, p.prec, false, nullptr, theta_init && p.iters == 0);
  if (s) return s;
  if (p.certify && cert_dev) s = certify_dispatch(c, b, st, cert_dev);
  return s;
}

gcp_status branch_picks_from_last_eval(Ctx& c, Batch& b, cudaStream_t st, int32_t* picks_dev) {
  const Net& net = *b.net;
  if (b.fp64 || b.recompute) return c.fail(GCP_EINVAL, "branching score: needs float duals with stored nuhat");
  std::vector<ScoreLayer> ls;
  for (int i = 1; i < net.L; ++i) {
    auto it = b.lazy.find("nuhat" + std::to_string(i));
    if (it == b.lazy.end()) return c.fail(GCP_EINVAL, "branching score: layer %d's nuhat was not kept", i);
    ls.push_back(ScoreLayer{(const float*)it->second, net.lo32[i - 1], net.hi32[i - 1], net.dims[i], i});
  }
  if (ls.empty() || b.S == 0) return GCP_OK;
  gcp_status s = GCP_OK;
  ScoreLayer* ld = (ScoreLayer*)b.ws("score_layers", ls.size() * sizeof(ScoreLayer), &s);
  if (!ld) return s;
  cudaError_t e = cudaMemcpyAsync(ld, ls.data(), ls.size() * sizeof(ScoreLayer), cudaMemcpyHostToDevice, st);
  if (e) return c.cuda(e, "branching score layers");
  bab_branch_score(st, b.S, b.K, (int)ls.size(), ld, b.sp_tab, b.M, picks_dev);
  e = cudaStreamSynchronize(st);   // ls is read by the copy above
  if (e) return c.cuda(e, "branching score");
  return launch_status(c, "branching score");
}

gcp_status optimize_batch(Ctx& c, Batch& b, const gcp_opt_params* p, double* out_bound, double* out_cert,
                          double* out_err) {
  if (!p) return c.fail(GCP_EINVAL, "null params");
  cudaStream_t st = c.stream;
  gcp_status s = GCP_OK;
  double* cd = nullptr;
  if (p->certify && b.R > 0) {
    cd = (double*)b.ws("cert", b.R * 8, &s);
    if (!cd) return s;
  }
  s = optimize_on(c, b, *p, st, cd);
  if (s) return s;
  if (b.R == 0) return GCP_OK;
  s = fetch_bound(c, b, st, out_bound);
  if (s) return s;
  std::vector<double> cert;
  if (cd && (out_cert || out_err)) {
    cert.resize(b.R);
    cudaError_t e = cudaMemcpyAsync(cert.data(), cd, b.R * 8, cudaMemcpyDeviceToHost, st);
    if (e) return c.cuda(e, "copy certified");
  }
  std::vector<double> bnd;
  if (out_err && !out_bound) {
    bnd.resize(b.R);
    s = fetch_bound(c, b, st, bnd.data());
    if (s) return s;
  }
  s = sync_check(c, st, "optimize_batch");
  if (s) return s;
  if (cd) {
    if (out_cert) std::copy(cert.begin(), cert.end(), out_cert);
    if (out_err) {
      const double* gb = out_bound ? out_bound : bnd.data();
      for (int64_t r = 0; r < b.R; ++r) out_err[r] = std::fabs(gb[r] - cert[r]);
    }
  }
  return GCP_OK;
}

// ------------------------------------------------------------------ dual import / export
// theta (layer-major [R, d_i] blocks on the device) <-> host [R, sum d_i]
gcp_status duals_theta(Ctx& c, Batch& b, const double* theta_in, double* theta_out) {
  const Net& net = *b.net;
  int64_t cols = 0;
  for (int i = 1; i < net.L; ++i) cols += net.dims[i];
  const size_t es = b.fp64 ? 8 : 4, bytes = (size_t)std::max<int64_t>(cols * b.R, 1) * es;
  if (theta_in) {
    for (int64_t q = 0; q < cols * b.R; ++q)
      if (!std::isfinite(theta_in[q])) return c.fail(GCP_EINVAL, "theta: non-finite entry");
    gcp_status s = GCP_OK;
    char* d = (char*)b.ws("theta", bytes, &s);
    if (!d) return s;
    std::vector<char> h((size_t)cols * b.R * es);
    int64_t off = 0, coff = 0;
    for (int i = 1; i < net.L; ++i) {
      const int di = net.dims[i];
      for (int64_t r = 0; r < b.R; ++r)
        for (int j = 0; j < di; ++j) {
          const double v = theta_in[r * cols + coff + j];
          const size_t k = (size_t)(off + r * di + j);
          if (b.fp64) ((double*)h.data())[k] = v; else ((float*)h.data())[k] = (float)v;
        }
      off += b.R * di;
      coff += di;
    }
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (!e && !h.empty()) e = cudaMemcpy(d, h.data(), h.size(), cudaMemcpyHostToDevice);
    if (e) return c.cuda(e, "import theta");
    b.theta_on = true;
  }
  if (theta_out) {
    if (!b.theta_on) return c.fail(GCP_ENOTFOUND, "the duals use the closed-form pi (no theta)");
    std::vector<char> h((size_t)cols * b.R * es);
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (!e && !h.empty()) e = cudaMemcpy(h.data(), b.lazy["theta"], h.size(), cudaMemcpyDeviceToHost);
    if (e) return c.cuda(e, "export theta");
    int64_t off = 0, coff = 0;
    for (int i = 1; i < net.L; ++i) {
      const int di = net.dims[i];
      for (int64_t r = 0; r < b.R; ++r)
        for (int j = 0; j < di; ++j) {
          const size_t k = (size_t)(off + r * di + j);
          theta_out[r * cols + coff + j] = b.fp64 ? ((const double*)h.data())[k] : (double)((const float*)h.data())[k];
        }
      off += b.R * di;
      coff += di;
    }
  }
  return GCP_OK;
}

gcp_status duals_export(Ctx& c, Batch& b, double* alpha, double* beta, double* gamma) {
  const Net& net = *b.net;
  cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e) return c.cuda(e, "export sync");
  const size_t es = b.fp64 ? 8 : 4;
  std::vector<char> h;
  auto rd = [&](const char* p, size_t i) -> double {
    return b.fp64 ? ((const double*)p)[i] : (double)((const float*)p)[i];
  };
  if (alpha) {
    int64_t cols = 0;
    for (int i = 1; i < net.L; ++i) cols += net.dims[i];
    int64_t coff = 0;
    for (int i = 1; i < net.L; ++i) {
      const int di = net.dims[i];
      h.resize((size_t)b.R * di * es);
      e = cudaMemcpy(h.data(), b.alpha[i - 1], h.size(), cudaMemcpyDeviceToHost);
      if (e) return c.cuda(e, "export alpha");
      for (int64_t r = 0; r < b.R; ++r)
        for (int j = 0; j < di; ++j) alpha[r * cols + coff + j] = rd(h.data(), (size_t)r * di + j);
      coff += di;
    }
  }
  if (beta && b.M > 0) {
    h.resize((size_t)b.M * b.R * es);
    e = cudaMemcpy(h.data(), b.beta, h.size(), cudaMemcpyDeviceToHost);
    if (e) return c.cuda(e, "export beta");
    for (size_t q = 0; q < (size_t)b.M * b.R; ++q) beta[q] = rd(h.data(), q);
  }
  if (gamma && b.N > 0) {
    h.resize((size_t)b.N * b.R * es);
    e = cudaMemcpy(h.data(), b.gamma, h.size(), cudaMemcpyDeviceToHost);
    if (e) return c.cuda(e, "export gamma");
    for (size_t q = 0; q < (size_t)b.N * b.R; ++q) gamma[q] = rd(h.data(), q);
  }
  return GCP_OK;
}

gcp_status duals_import(Ctx& c, Batch& b, const double* alpha, const double* beta, const double* gamma) {
  const Net& net = *b.net;
  gcp_status s = reset_duals(c, b, !alpha, !beta, !gamma);
  if (s) return s;
  b.theta_on = false;                 // back to the closed-form pi
  cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e) return c.cuda(e, "import sync");
  const size_t es = b.fp64 ? 8 : 4;
  std::vector<char> h;
  auto wr = [&](char* p, size_t i, double v) {
    if (b.fp64) ((double*)p)[i] = v; else ((float*)p)[i] = (float)v;
  };
  if (alpha) {
    int64_t cols = 0;
    for (int i = 1; i < net.L; ++i) cols += net.dims[i];
    int64_t coff = 0;
    for (int i = 1; i < net.L; ++i) {
      const int di = net.dims[i];
      h.resize((size_t)b.R * di * es);
      for (int64_t r = 0; r < b.R; ++r)
        for (int j = 0; j < di; ++j) wr(h.data(), (size_t)r * di + j, alpha[r * cols + coff + j]);
      e = cudaMemcpy(b.alpha[i - 1], h.data(), h.size(), cudaMemcpyHostToDevice);
      if (e) return c.cuda(e, "import alpha");
      coff += di;
    }
  }
  if (beta && b.M > 0) {
    h.resize((size_t)b.M * b.R * es);
    for (size_t q = 0; q < (size_t)b.M * b.R; ++q) wr(h.data(), q, beta[q]);
    e = cudaMemcpy(b.beta, h.data(), h.size(), cudaMemcpyHostToDevice);
    if (e) return c.cuda(e, "import beta");
  }
  if (gamma && b.N > 0) {
    h.resize((size_t)b.N * b.R * es);
    for (size_t q = 0; q < (size_t)b.N * b.R; ++q) wr(h.data(), q, gamma[q]);
    e = cudaMemcpy(b.gamma, h.data(), h.size(), cudaMemcpyHostToDevice);
    if (e) return c.cuda(e, "import gamma");
  }
  return GCP_OK;
}

// Caller-owned device arrays of the device entry points take part in the launch
// checks for the duration of the call (registered with their documented sizes).
struct ForeignArrays {
  std::vector<uint64_t> regs;
  gcp_status add(Ctx& c, const void* p, size_t bytes, const char* what) {
    if (!p || bytes == 0) return GCP_OK;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      return c.fail(GCP_EINVAL, "%s is not a device pointer", what);
    }
    regs.push_back(reg_foreign(p, bytes));
    return GCP_OK;
  }
  ~ForeignArrays() {
    for (uint64_t t : regs) reg_unforeign(t);
  }
};

static int64_t alpha_cols(const Net& net) {
  int64_t cols = 0;
  for (int i = 1; i < net.L; ++i) cols += net.dims[i];
  return cols;
}

// Device-pointer variants (float duals in export layouts).
gcp_status load_device_duals(Ctx& c, Batch& b, cudaStream_t st, const float* alpha, const float* beta,
                             const float* gamma) {
  if (b.fp64) return c.fail(GCP_EINVAL, "device entry points need GCP_FP32 duals");
  const Net& net = *b.net;
  int64_t cols = 0;
  for (int i = 1; i < net.L; ++i) cols += net.dims[i];
  int64_t coff = 0;
  for (int i = 1; i < net.L; ++i) {
    const int di = net.dims[i];
    if (alpha && b.R > 0) {
      cudaError_t e = cudaMemcpy2DAsync(b.alpha[i - 1], di * 4, alpha + coff, cols * 4, di * 4, b.R,
                                        cudaMemcpyDeviceToDevice, st);
      if (e) return c.cuda(e, "alpha in");
    }
    coff += di;
  }
  cudaError_t e = cudaSuccess;
  if (beta && b.M > 0) e = cudaMemcpyAsync(b.beta, beta, (size_t)b.R * b.M * 4, cudaMemcpyDeviceToDevice, st);
  if (!e && gamma && b.N > 0) e = cudaMemcpyAsync(b.gamma, gamma, (size_t)b.R * b.N * 4, cudaMemcpyDeviceToDevice, st);
  if (e) return c.cuda(e, "load duals");
  return launch_status(c, "load duals");
}

gcp_status bound_device(Ctx& c, Batch& b, int prec, const float* alpha, const float* beta, const float* gamma,
                        float* out, cudaStream_t st) {
  gcp_status s = check_prec(c, b, prec);
  if (s) return s;
  if (prec == GCP_FP64) return c.fail(GCP_EINVAL, "device entry points run FP32 or BF16");
  ForeignArrays fa;
  const size_t R4 = (size_t)b.R * 4;
  if ((s = fa.add(c, alpha, R4 * alpha_cols(*b.net), "alpha")) || (s = fa.add(c, beta, R4 * b.M, "beta")) ||
      (s = fa.add(c, gamma, R4 * b.N, "gamma")) || (s = fa.add(c, out, R4, "out")))
    return s;
  s = load_device_duals(c, b, st, alpha, beta, gamma);
  if (s) return s;
  if (b.R == 0) return GCP_OK;
  s = eval_dispatch(c, b, st, prec, false, nullptr);
  if (s) return s;
  return c.cuda(cudaMemcpyAsync(out, b.lazy["g"], (size_t)b.R * 4, cudaMemcpyDeviceToDevice, st), "bound out");
}

gcp_status grad_device(Ctx& c, Batch& b, int prec, const float* alpha, const float* beta, const float* gamma,
                       const float* grad_out, float* g_alpha, float* g_beta, float* g_gamma, cudaStream_t st) {
  gcp_status s = check_prec(c, b, prec);
  if (s) return s;
  if (prec == GCP_FP64) return c.fail(GCP_EINVAL, "device entry points run FP32 or BF16");
  ForeignArrays fa;
  const size_t R4 = (size_t)b.R * 4, na = (size_t)alpha_cols(*b.net);
  if ((s = fa.add(c, alpha, R4 * na, "alpha")) || (s = fa.add(c, beta, R4 * b.M, "beta")) ||
      (s = fa.add(c, gamma, R4 * b.N, "gamma")) || (s = fa.add(c, grad_out, R4, "grad_out")) ||
      (s = fa.add(c, g_alpha, R4 * na, "g_alpha")) || (s = fa.add(c, g_beta, R4 * b.M, "g_beta")) ||
      (s = fa.add(c, g_gamma, R4 * b.N, "g_gamma")))
    return s;
  s = load_device_duals(c, b, st, alpha, beta, gamma);
  if (s) return s;
  if (b.R == 0) return GCP_OK;
  const Net& net = *b.net;
  int64_t nal = 0;
  for (int i = 1; i < net.L; ++i) nal += (int64_t)b.R * net.dims[i];
  float* gal = (float*)b.ws("g_alpha", (size_t)nal * 4, &s);
  float* gbe = (float*)b.ws("g_beta", (size_t)std::max(b.M, 1) * b.R * 4, &s);
  float* gga = (float*)b.ws("g_gamma", (size_t)std::max(b.N, 1) * b.R * 4, &s);
  if (!gal || !gbe || !gga) return s;
  cudaMemsetAsync(gbe, 0, (size_t)std::max(b.M, 1) * b.R * 4, st);
  s = eval_dispatch(c, b, st, prec, true, grad_out);
  if (s) return s;
  StepArgs<float> step{};
  step.mode = 0;
  s = prec == GCP_FP32 ? run_adjoint<float, float>(c, b, st, step, grad_out, gal, gbe, gga)
                       : run_adjoint<float, __nv_bfloat16>(c, b, st, step, grad_out, gal, gbe, gga);
  if (s) return s;
  int64_t cols = 0;
  for (int i = 1; i < net.L; ++i) cols += net.dims[i];
  int64_t coff = 0, off = 0;
  for (int i = 1; i < net.L; ++i) {
    const int di = net.dims[i];
    if (g_alpha) {
      cudaError_t e = cudaMemcpy2DAsync(g_alpha + coff, cols * 4, gal + off, di * 4, di * 4, b.R,
                                        cudaMemcpyDeviceToDevice, st);
      if (e) return c.cuda(e, "g_alpha out");
    }
    coff += di;
    off += (int64_t)b.R * di;
  }
  cudaError_t e = cudaSuccess;
  if (g_beta && b.M > 0) e = cudaMemcpyAsync(g_beta, gbe, (size_t)b.R * b.M * 4, cudaMemcpyDeviceToDevice, st);
  if (!e && g_gamma && b.N > 0) e = cudaMemcpyAsync(g_gamma, gga, (size_t)b.R * b.N * 4, cudaMemcpyDeviceToDevice, st);
  if (e) return c.cuda(e, "grad out");
  return launch_status(c, "grad out");
}

}  // namespace gcp

// ====================================================================== C ABI
using gcp::Ctx;

#define CTX_GUARD(ctx)                                   \
  if (!(ctx)) return GCP_EINVAL;                         \
  std::lock_guard<std::recursive_mutex> _lk((ctx)->mu);  \
  cudaSetDevice((ctx)->device);

extern "C" {

gcp_status gcp_create(gcp_ctx** out, int32_t device, uint64_t budget) {
  if (!out) return GCP_EINVAL;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return GCP_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return GCP_ECUDA;
  Ctx* c = new (std::nothrow) Ctx();
  if (!c) return GCP_ENOMEM;
  c->device = device;
  c->budget = budget;
  if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return GCP_ECUDA;
  }
  c->stream = c->own_stream;
  *out = reinterpret_cast<gcp_ctx*>(c);
  return GCP_OK;
}

gcp_status gcp_destroy(gcp_ctx* h) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  if (!c) return GCP_EINVAL;
  gcp::serve_shutdown(*c);
  {
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    c->batches.clear();
    c->cutsets.clear();
    c->nets.clear();
    c->trim();
    cudaStreamDestroy(c->own_stream);
  }
  delete c;
  return GCP_OK;
}

const char* gcp_last_error(const gcp_ctx* h) {
  const Ctx* c = reinterpret_cast<const Ctx*>(h);
  if (!c) return "null context";
  return c->err.c_str();
}

gcp_status gcp_set_stream(gcp_ctx* h, void* stream) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  CTX_GUARD(c);
  c->stream = stream ? (cudaStream_t)stream : c->own_stream;
  return GCP_OK;
}

gcp_status gcp_mem_used(const gcp_ctx* h, uint64_t* bytes) {
  const Ctx* c = reinterpret_cast<const Ctx*>(h);
  if (!c || !bytes) return GCP_EINVAL;
  *bytes = c->used;
  return GCP_OK;
}

gcp_status gcp_init_net(gcp_ctx* h, const gcp_layer_desc* layers, int32_t n_layers, const double* x_lo,
                        const double* x_hi, const double* spec_c, int32_t n_spec, const double* inter_lo,
                        const double* inter_hi, int32_t* net_id) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  CTX_GUARD(c);
  return gcp::init_net(*c, layers, n_layers, x_lo, x_hi, spec_c, n_spec, inter_lo, inter_hi, net_id);
}

gcp_status gcp_add_cuts(gcp_ctx* h, int32_t net_id, int32_t n_cuts, const int64_t* row_ptr, const int16_t* layer,
                        const int8_t* kind, const int32_t* index, const double* coef, const double* d,
                        int32_t* cutset_id, int32_t* first_cut) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  CTX_GUARD(c);
  return gcp::add_cuts(*c, net_id, n_cuts, row_ptr, layer, kind, index, coef, d, cutset_id, first_cut);
}

static gcp::Batch* find_batch(Ctx* c, void* duals) {
  auto it = c->batches.find((gcp::Batch*)duals);
  return it == c->batches.end() ? nullptr : it->second.get();
}

gcp_status gcp_duals_create(gcp_ctx* h, int32_t net_id, int32_t cutset_id, const gcp_subdomains* sub,
                            int32_t dual_prec, void** duals) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  CTX_GUARD(c);
  gcp::Batch* b = nullptr;
  gcp_status s;
  {
    // blocks come from (and go back to) the context's pool: a batch created
    // and freed every step reuses the previous one's memory
    gcp::AllocPool g;
    s = gcp::duals_create(*c, net_id, cutset_id, sub, dual_prec, &b);
  }
  if (s == GCP_OK) {
    b->pool_stream = c->stream;
    s = gcp::sync_check(*c, c->stream, "duals_create");
    if (s == GCP_OK) *duals = b;
  }
  return s;
}

gcp_status gcp_duals_create_multi(gcp_ctx* h, int32_t net_id, int32_t n_queries, const int32_t* cutset_ids,
                                  const gcp_subdomains* subs, int32_t dual_prec, void** duals) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  CTX_GUARD(c);
  if (n_queries < 1 || !cutset_ids || !subs || !duals) return c->fail(GCP_EINVAL, "gcp_duals_create_multi: bad arguments");
  std::vector<std::pair<const gcp::CutSet*, const gcp_subdomains*>> parts;
  for (int q = 0; q < n_queries; ++q) {
    const gcp::CutSet* cs = nullptr;
    if (cutset_ids[q] >= 0) {
      auto ci = c->cutsets.find(cutset_ids[q]);
      if (ci == c->cutsets.end()) return c->fail(GCP_ENOTFOUND, "unknown cut set %d", cutset_ids[q]);
      cs = ci->second.get();
    }
    parts.push_back({cs, &subs[q]});
  }
  gcp::Batch* b = nullptr;
  gcp_status s;
  {
    gcp::AllocPool g;
    s = gcp::duals_create_parts(*c, net_id, parts, dual_prec, &b);
  }
  if (s == GCP_OK) {
    b->pool_stream = c->stream;
    s = gcp::sync_check(*c, c->stream, "duals_create_multi");
    if (s == GCP_OK) *duals = b;
  }
  return s;
}

gcp_status gcp_duals_shape(gcp_ctx* h, void* duals, int64_t* rows, int64_t* n_alpha, int32_t* max_splits,
                           int32_t* n_cuts) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  CTX_GUARD(c);
  gcp::Batch* b = find_batch(c, duals);
  if (!b) return c->fail(GCP_ENOTFOUND, "unknown duals");
  int64_t na = 0;
  for (int i = 1; i < b->net->L; ++i) na += b->net->dims[i];
  if (rows) *rows = b->R;
  if (n_alpha) *n_alpha = na;
  if (max_splits) *max_splits = b->M;
  if (n_cuts) *n_cuts = b->N;
  return GCP_OK;
}

gcp_status gcp_duals_export(gcp_ctx* h, void* duals, double* a, double* be, double* g) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  CTX_GUARD(c);
  gcp::Batch* b = find_batch(c, duals);
  if (!b) return c->fail(GCP_ENOTFOUND, "unknown duals");
  return gcp::duals_export(*c, *b, a, be, g);
}

gcp_status gcp_duals_theta(gcp_ctx* h, void* duals, const double* theta_in, double* theta_out) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  CTX_GUARD(c);
  gcp::Batch* b = find_batch(c, duals);
  if (!b) return c->fail(GCP_ENOTFOUND, "unknown duals");
  return gcp::duals_theta(*c, *b, theta_in, theta_out);
}

gcp_status gcp_duals_import(gcp_ctx* h, void* duals, const double* a, const double* be, const double* g) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  CTX_GUARD(c);
  gcp::Batch* b = find_batch(c, duals);
  if (!b) return c->fail(GCP_ENOTFOUND, "unknown duals");
  return gcp::duals_import(*c, *b, a, be, g);
}

gcp_status gcp_duals_free(gcp_ctx* h, void* duals) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  CTX_GUARD(c);
  auto it = c->batches.find((gcp::Batch*)duals);
  if (it == c->batches.end()) return c->fail(GCP_ENOTFOUND, "unknown duals");
  cudaStreamSynchronize(c->stream);
  c->batches.erase(it);
  return GCP_OK;
}

gcp_status gcp_bound_batch(gcp_ctx* h, void* duals, int32_t prec, int32_t certify, double* out_bound,
                           double* out_cert) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  CTX_GUARD(c);
  gcp::Batch* b = find_batch(c, duals);
  if (!b) return c->fail(GCP_ENOTFOUND, "unknown duals");
  return gcp::bound_batch(*c, *b, prec, certify, out_bound, out_cert);
}

gcp_status gcp_grad_batch(gcp_ctx* h, void* duals, int32_t prec, double* out_bound, double* ga, double* gb,
                          double* gg) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  CTX_GUARD(c);
  gcp::Batch* b = find_batch(c, duals);
  if (!b) return c->fail(GCP_ENOTFOUND, "unknown duals");
  return gcp::grad_batch(*c, *b, prec, out_bound, ga, gb, gg);
}

gcp_status gcp_branch_picks(gcp_ctx* h, void* duals, int32_t prec, int32_t* layer, int32_t* index) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  CTX_GUARD(c);
  gcp::Batch* b = find_batch(c, duals);
  if (!b) return c->fail(GCP_ENOTFOUND, "unknown duals");
  if (!layer || !index) return c->fail(GCP_EINVAL, "gcp_branch_picks: null output");
  if (prec != GCP_FP32 && prec != GCP_BF16) return c->fail(GCP_EINVAL, "gcp_branch_picks: FP32 or BF16 chain");
  if (b->fp64) return c->fail(GCP_EINVAL, "gcp_branch_picks: needs GCP_FP32 duals");
  gcp_status s0 = gcp::check_prec(*c, *b, prec);
  if (s0) return s0;
  if (b->S == 0) return GCP_OK;
  gcp_status s = GCP_OK;
  int32_t* pd = (int32_t*)b->ws("picks", (size_t)b->S * 4, &s);
  if (!pd) return s;
  b->keep_nuhat = true;
  s = gcp::eval_dispatch(*c, *b, c->stream, prec, false, nullptr, false);
  b->keep_nuhat = false;
  if (s == GCP_OK) s = gcp::branch_picks_from_last_eval(*c, *b, c->stream, pd);
  if (s) return s;
  std::vector<int32_t> h_picks((size_t)b->S);
  cudaError_t e = cudaMemcpy(h_picks.data(), pd, (size_t)b->S * 4, cudaMemcpyDeviceToHost);
  if (e) return c->cuda(e, "gcp_branch_picks");
  for (int q = 0; q < b->S; ++q) {
    layer[q] = h_picks[q] < 0 ? -1 : (h_picks[q] >> 24);
    index[q] = h_picks[q] < 0 ? -1 : (h_picks[q] & 0xffffff);
  }
  return GCP_OK;
}

gcp_status gcp_optimize_batch(gcp_ctx* h, void* duals, const gcp_opt_params* p, double* out_bound,
                              double* out_cert, double* out_err) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  CTX_GUARD(c);
  gcp::Batch* b = find_batch(c, duals);
  if (!b) return c->fail(GCP_ENOTFOUND, "unknown duals");
  return gcp::optimize_batch(*c, *b, p, out_bound, out_cert, out_err);
}

gcp_status gcp_bound_device(gcp_ctx* h, void* duals, int32_t prec, const float* alpha, const float* beta,
                            const float* gamma, float* out, void* stream) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  CTX_GUARD(c);
  gcp::Batch* b = find_batch(c, duals);
  if (!b) return c->fail(GCP_ENOTFOUND, "unknown duals");
  return gcp::bound_device(*c, *b, prec, alpha, beta, gamma, out, stream ? (cudaStream_t)stream : c->stream);
}

gcp_status gcp_grad_device(gcp_ctx* h, void* duals, int32_t prec, const float* alpha, const float* beta,
                           const float* gamma, const float* grad_out, float* g_alpha, float* g_beta, float* g_gamma,
                           void* stream) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  CTX_GUARD(c);
  gcp::Batch* b = find_batch(c, duals);
  if (!b) return c->fail(GCP_ENOTFOUND, "unknown duals");
  return gcp::grad_device(*c, *b, prec, alpha, beta, gamma, grad_out, g_alpha, g_beta, g_gamma,
                          stream ? (cudaStream_t)stream : c->stream);
}

}  // extern "C"

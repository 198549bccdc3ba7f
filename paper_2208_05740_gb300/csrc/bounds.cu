// Root intermediate bounds by the library's own bound propagation.
//
// The method needs sound pre-activation bounds l, u of every hidden neuron
// (Sec. 2; they classify the neurons and bound the relaxations). Here they
// come from the same machinery, layer by layer: the bounds of hidden layer 1
// are the interval image of the box under the first linear map (outward
// rounded on the host); for a hidden layer i > 1 the network truncated after
// the linear map of layer i, with the spec rows +e_j and -e_j over its
// pre-activations, is bounded with the layers below already bounded, and the
// certified FP64 values give lo_j = g(+e_j) and hi_j = -g(-e_j). At the
// default slopes this is CROWN; with ascent steps on the slopes of each such
// row it is alpha-CROWN. Every value is a certified (outward-rounded) bound,
// so the result is sound whatever precision the chain runs in. A residual
// layer keeps its skip in the truncated network: the last layer's skip then
// adds the rows' own slice of xhat^(m) (identity) or the same rows of its
// projection S.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gcp_ctx.h"

namespace gcp {
namespace {

constexpr int kBoundRows = 512;   // neurons of a layer bounded per batch (spec rows = 2x)

// Cutting planes for the root bounds, CSR by cut as in gcp_add_cuts.
struct CutRows {
  int n = 0;
  const int64_t* ptr = nullptr;
  const int16_t* layer = nullptr;
  const int8_t* kind = nullptr;
  const int32_t* index = nullptr;
  const double* coef = nullptr;
  const double* d = nullptr;
};

double round_down(double x) { return std::nextafter(x, -INFINITY); }
double round_up(double x) { return std::nextafter(x, INFINITY); }

// rows j0 .. j0+nj-1 of a layer's linear map as a dense [nj, d_in] matrix
// (a convolution's rows materialised) and their biases (0 without b)
void dense_rows(const gcp_layer_desc& d, int j0, int nj, std::vector<double>& W, std::vector<double>& b) {
  W.assign((size_t)nj * d.d_in, 0.0);
  b.resize(nj);
  for (int q = 0; q < nj; ++q) {
    const int j = j0 + q;
    b[q] = d.b ? d.b[j] : 0.0;
    double* row = W.data() + (size_t)q * d.d_in;
    if (d.kind == GCP_DENSE) {
      std::copy(d.W + (size_t)j * d.d_in, d.W + (size_t)(j + 1) * d.d_in, row);
      continue;
    }
    const int hw = d.h_out * d.w_out, o = j / hw, oh = (j % hw) / d.w_out, ow = j % d.w_out;
    for (int ci = 0; ci < d.c_in; ++ci)
      for (int kh = 0; kh < d.k; ++kh) {
        const int ih = oh * d.stride - d.pad + kh;
        if (ih < 0 || ih >= d.h_in) continue;
        for (int kw = 0; kw < d.k; ++kw) {
          const int iw = ow * d.stride - d.pad + kw;
          if (iw < 0 || iw >= d.w_in) continue;
          row[((size_t)ci * d.h_in + ih) * d.w_in + iw] += d.W[(((size_t)o * d.c_in + ci) * d.k + kh) * d.k + kw];
        }
      }
  }
}

}  // namespace

gcp_status intermediate_bounds(Ctx& c, const gcp_layer_desc* layers, int L, const double* x_lo, const double* x_hi,
                               const gcp_opt_params* p, double* out_lo, double* out_hi, const CutRows* cuts = nullptr) {
  if (!layers || L < 2 || !x_lo || !x_hi || !out_lo || !out_hi)
    return c.fail(GCP_EINVAL, "gcp_intermediate_bounds: null argument or no hidden layer");
  for (int i = 0; i < L; ++i)
    if (!layers[i].W || !layers[i].b || layers[i].d_in <= 0 || layers[i].d_out <= 0 ||
        (i > 0 && layers[i].d_in != layers[i - 1].d_out))
      return c.fail(GCP_EINVAL, "gcp_intermediate_bounds: layer %d: bad shape or null weights", i + 1);
  {
    const gcp_layer_desc& d = layers[0];
    const gcp_layer_desc* sc = d.shortcut;
    if (d.skip != 0 && (d.skip != 1 || (sc ? (sc->d_in != d.d_in || sc->d_out != d.d_out || !sc->W)
                                           : d.d_in != d.d_out)))
      return c.fail(GCP_EINVAL, "gcp_intermediate_bounds: layer 1 can only add the input (skip 1) through the "
                    "identity (d_in = d_out) or a shortcut of its shape");
  }
  if (p && (p->iters < 0 || p->prec < GCP_FP32 || p->prec > GCP_BF16))
    return c.fail(GCP_EINVAL, "gcp_intermediate_bounds: iters >= 0 and prec FP32 or BF16");
  int64_t total = 0;
  for (int i = 0; i + 1 < L; ++i) total += layers[i].d_out;
  std::vector<double> blo(total), bhi(total);   // the outputs stay untouched on error
  std::vector<double> W, b;
  // hidden layer 1: interval image of the box, each product and sum rounded outwards
  {
    const gcp_layer_desc& d = layers[0];
    std::vector<double> S, bs;
    for (int j0 = 0; j0 < d.d_out; j0 += kBoundRows) {
      const int nj = std::min(kBoundRows, d.d_out - j0);
      dense_rows(d, j0, nj, W, b);
      if (d.skip == 1 && d.shortcut) dense_rows(*d.shortcut, j0, nj, S, bs);
      for (int q = 0; q < nj; ++q) {
        double lo = b[q], hi = b[q];
        auto add_row = [&](const double* row) {
          for (int k = 0; k < d.d_in; ++k) {
            const double w = row[k];
            if (w == 0.0) continue;
            const double a = w * x_lo[k], e = w * x_hi[k];
            lo = round_down(lo + round_down(std::min(a, e)));
            hi = round_up(hi + round_up(std::max(a, e)));
          }
        };
        add_row(W.data() + (size_t)q * d.d_in);
        if (d.skip == 1 && d.shortcut) {         // x^(1) = W x + b + S x
          add_row(S.data() + (size_t)q * d.d_in);
        } else if (d.skip == 1) {                // x^(1) = W x + b + x
          lo = round_down(lo + x_lo[j0 + q]);
          hi = round_up(hi + x_hi[j0 + q]);
        }
        if (!std::isfinite(lo) || !std::isfinite(hi)) return c.fail(GCP_EINVAL, "layer 1 bounds not finite");
        blo[j0 + q] = lo;
        bhi[j0 + q] = hi;
      }
    }
  }
  // hidden layers 2 .. L-1 through the bound propagation
  int64_t off = layers[0].d_out;
  std::vector<int32_t> ptr{0, 0}, idx{0};
  std::vector<int16_t> lay{0};
  std::vector<int8_t> sgn{0};
  const gcp_subdomains sub{1, ptr.data(), lay.data(), idx.data(), sgn.data()};
  // each cut's deepest layer: it constrains the truncated networks of the layers below it
  std::vector<int> cut_top;
  if (cuts && cuts->n > 0) {
    if (!cuts->ptr || !cuts->d || cuts->ptr[0] != 0) return c.fail(GCP_EINVAL, "cut arrays");
    cut_top.assign(cuts->n, 0);
    for (int k = 0; k < cuts->n; ++k) {
      if (cuts->ptr[k + 1] < cuts->ptr[k]) return c.fail(GCP_EINVAL, "cut %d: row_ptr decreases", k);
      for (int64_t e = cuts->ptr[k]; e < cuts->ptr[k + 1]; ++e) {
        if (cuts->layer[e] < 0 || cuts->layer[e] >= L) return c.fail(GCP_EINVAL, "cut %d: layer out of range", k);
        cut_top[k] = std::max<int>(cut_top[k], cuts->layer[e]);
      }
    }
  }
  std::vector<double> S, bs;
  for (int i = 2; i < L; ++i) {
    const gcp_layer_desc& d = layers[i - 1];
    for (int j0 = 0; j0 < d.d_out; j0 += kBoundRows) {
      const int nj = std::min(kBoundRows, d.d_out - j0);
      dense_rows(d, j0, nj, W, b);
      gcp_layer_desc sc{};                  // the same rows of a projection shortcut
      if (d.skip && d.shortcut) {
        dense_rows(*d.shortcut, j0, nj, S, bs);
        sc.kind = GCP_DENSE;
        sc.d_in = d.shortcut->d_in;
        sc.d_out = nj;
        sc.W = S.data();
      }
      std::vector<gcp_layer_desc> net(layers, layers + (i - 1));
      gcp_layer_desc last{};
      last.kind = GCP_DENSE;
      last.d_in = d.d_in;
      last.d_out = nj;
      last.W = W.data();
      last.b = b.data();
      last.skip = d.skip;
      last.shortcut = (d.skip && d.shortcut) ? &sc : nullptr;
      net.push_back(last);
      std::vector<double> spec((size_t)2 * nj * nj, 0.0);
      for (int q = 0; q < nj; ++q) {
        spec[(size_t)q * nj + q] = 1.0;
        spec[(size_t)(nj + q) * nj + q] = -1.0;
      }
      int nid = -1;
      gcp_status s = init_net(c, net.data(), i, x_lo, x_hi, spec.data(), 2 * nj, blo.data(), bhi.data(), &nid,
                              (d.skip && !d.shortcut) ? j0 : 0);
      if (s) return s;
      // the cuts over layers 0 .. i-1 constrain this truncated network
      int cs_id = -1;
      if (!cut_top.empty()) {
        std::vector<int64_t> ptr{0};
        std::vector<int16_t> lay;
        std::vector<int8_t> knd;
        std::vector<int32_t> idx;
        std::vector<double> cf, dd;
        for (int k = 0; k < cuts->n; ++k) {
          if (cut_top[k] > i - 1) continue;
          for (int64_t e = cuts->ptr[k]; e < cuts->ptr[k + 1]; ++e) {
            lay.push_back(cuts->layer[e]);
            knd.push_back(cuts->kind[e]);
            idx.push_back(cuts->index[e]);
            cf.push_back(cuts->coef[e]);
          }
          ptr.push_back((int64_t)lay.size());
          dd.push_back(cuts->d[k]);
        }
        if (!dd.empty()) {
          int first = 0;
          s = add_cuts(c, nid, (int)dd.size(), ptr.data(), lay.data(), knd.data(), idx.data(), cf.data(), dd.data(),
                       &cs_id, &first);
          if (s) {
            c.nets.erase(nid);
            return s;
          }
        }
      }
      Batch* bt = nullptr;
      s = duals_create(c, nid, cs_id, &sub, GCP_FP32, &bt);
      std::vector<double> cert((size_t)2 * nj);
      if (s == GCP_OK) {
        if (p) {
          gcp_opt_params q = *p;
          q.certify = 1;
          s = optimize_batch(c, *bt, &q, nullptr, cert.data(), nullptr);
        } else {
          s = bound_batch(c, *bt, GCP_FP32, 1, nullptr, cert.data());
        }
      }
      if (bt) {
        cudaStreamSynchronize(c.stream);
        c.batches.erase(bt);
      }
      if (cs_id >= 0) c.cutsets.erase(cs_id);
      c.nets.erase(nid);
      if (s) return s;
      for (int q = 0; q < nj; ++q) {
        const double lo = cert[q], hi = -cert[nj + q];
        if (!std::isfinite(lo) || !std::isfinite(hi) || lo > hi)
          return c.fail(GCP_EDEVICE, "layer %d neuron %d: bounds [%g, %g]", i, j0 + q, lo, hi);
        blo[off + j0 + q] = lo;
        bhi[off + j0 + q] = hi;
      }
    }
    off += d.d_out;
  }
  std::copy(blo.begin(), blo.end(), out_lo);
  std::copy(bhi.begin(), bhi.end(), out_hi);
  return GCP_OK;
}

}  // namespace gcp

extern "C" gcp_status gcp_intermediate_bounds(gcp_ctx* h, const gcp_layer_desc* layers, int32_t n_layers,
                                              const double* x_lo, const double* x_hi, const gcp_opt_params* p,
                                              double* inter_lo, double* inter_hi) {
  gcp::Ctx* c = reinterpret_cast<gcp::Ctx*>(h);
  if (!c) return GCP_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  cudaSetDevice(c->device);
  return gcp::intermediate_bounds(*c, layers, n_layers, x_lo, x_hi, p, inter_lo, inter_hi);
}

extern "C" gcp_status gcp_intermediate_bounds_cuts(gcp_ctx* h, const gcp_layer_desc* layers, int32_t n_layers,
                                                   const double* x_lo, const double* x_hi, const gcp_opt_params* p,
                                                   int32_t n_cuts, const int64_t* row_ptr, const int16_t* layer,
                                                   const int8_t* kind, const int32_t* index, const double* coef,
                                                   const double* d, double* inter_lo, double* inter_hi) {
  gcp::Ctx* c = reinterpret_cast<gcp::Ctx*>(h);
  if (!c) return GCP_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  cudaSetDevice(c->device);
  if (n_cuts < 0 || (n_cuts > 0 && (!row_ptr || !layer || !kind || !index || !coef || !d)))
    return c->fail(GCP_EINVAL, "gcp_intermediate_bounds_cuts: bad cut arrays");
  gcp::CutRows cr{n_cuts, row_ptr, layer, kind, index, coef, d};
  return gcp::intermediate_bounds(*c, layers, n_layers, x_lo, x_hi, p, inter_lo, inter_hi, &cr);
}

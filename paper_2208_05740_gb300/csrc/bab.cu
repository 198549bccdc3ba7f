// Branch and bound over ReLU splits with the library's bounding (Sec. 3.2).
//
// A property (every spec row c_k of the network positive over the input box)
// is verified by splitting the input region's ReLU phases: a subdomain whose
// certified bounds are all positive is done; any other is split on one more
// unstable neuron into its x >= 0 and x <= 0 children (App. B), which start
// from the parent's duals. Each round bounds up to `batch` pending subdomains
// in one batch (ascent steps, then the FP64 certification); when more are
// pending, the easiest ones, with the largest lower bounds, go first (the
// order the paper uses so that cuts arriving later meet the hard domains).
// The branching neuron of a subdomain is chosen from its duals at the end of
// its round: the largest intercept cost w_j * sum_k [nuhat_j]_+ over its
// unsplit root-unstable neurons (BaBSR's score; kernel bab_branch_score),
// or, by request or where every score is zero, its not yet split
// root-unstable neuron with the largest relaxation intercept -l u / (u - l).
//
// Label by label (the same section): every spec row (target label) is
// bounded at the root, and the rows not yet positive get a branch and bound
// of their own, the easiest first -- the root bound closest to zero -- so that
// harder labels come later (when cuts from a MIP solver are stronger). Each
// label runs on a one-row view of the network that shares its device data.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <memory>
#include <vector>

#include "gcp_ctx.h"

namespace gcp {
namespace {

// One round's duals kept on the device for the children of its subdomains
// (alpha row-major [rows, na], beta [rows, M], gamma [rows, N]); its blocks go
// back to the context's pool once the last child has been bounded (after that
// round's stream synchronisation).
struct ParentStore {
  Ctx* c = nullptr;
  float* alpha = nullptr;
  float* beta = nullptr;
  float* gamma = nullptr;
  int64_t rows = 0;
  int M = 0;
  ~ParentStore() {
    if (!c) return;
    c->recycle(alpha);
    c->recycle(beta);
    c->recycle(gamma);
  }
};

struct Domain {
  std::vector<int16_t> lay;
  std::vector<int32_t> idx;
  std::vector<int8_t> sgn;
  double margin = -INFINITY;    // priority: the parent's smallest certified bound
  std::shared_ptr<ParentStore> par;   // the parent's duals (null: defaults)
  int64_t prow = 0;                   // the parent's first row in it
};

}  // namespace


gcp_status bab_verify(Ctx& c, int net_id, int cutset_id, const gcp_bab_params& bp, gcp_bab_result& res) {
  const auto t0 = std::chrono::steady_clock::now();
  auto it = c.nets.find(net_id);
  if (it == c.nets.end()) return c.fail(GCP_ENOTFOUND, "unknown network %d", net_id);
  if (bp.batch < 1 || bp.max_rounds < 1 || bp.max_domains < 1 || bp.p.iters < 0)
    return c.fail(GCP_EINVAL, "gcp_bab_verify: batch, max_rounds, max_domains >= 1 and iters >= 0");
  const Net& net = *it->second;
  const int K = net.K;
  int64_t na = 0;
  for (int i = 1; i < net.L; ++i) na += net.dims[i];
  // root-unstable neurons by decreasing intercept -l u / (u - l)
  struct Cand {
    double score;
    int16_t layer;
    int32_t index;
  };
  std::vector<Cand> cand;
  {
    std::vector<double> lo, hi;
    for (int i = 1; i < net.L; ++i) {
      const int di = net.dims[i];
      lo.resize(di);
      hi.resize(di);
      cudaMemcpy(lo.data(), net.lo64[i - 1], di * 8, cudaMemcpyDeviceToHost);
      cudaMemcpy(hi.data(), net.hi64[i - 1], di * 8, cudaMemcpyDeviceToHost);
      for (int j = 0; j < di; ++j)
        if (lo[j] < 0 && hi[j] > 0) cand.push_back({-lo[j] * hi[j] / (hi[j] - lo[j]), (int16_t)i, j});
    }
    std::stable_sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) { return a.score > b.score; });
  }
  gcp_opt_params p = bp.p;
  p.certify = 1;
  std::vector<Domain> pending(1);
  res = gcp_bab_result{};
  res.min_bound = INFINITY;
  bool undecided = false;   // a subdomain with every candidate split and a non-positive bound
  while (!pending.empty()) {
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (res.rounds >= bp.max_rounds || (int64_t)pending.size() > bp.max_domains ||
        (bp.timeout_s > 0 && el > bp.timeout_s))
      break;
    // the easiest domains first
    const size_t n = std::min<size_t>(pending.size(), (size_t)bp.batch);
    std::stable_sort(pending.begin(), pending.end(),
                     [](const Domain& a, const Domain& b) { return a.margin > b.margin; });
    std::vector<Domain> cur(std::make_move_iterator(pending.begin()), std::make_move_iterator(pending.begin() + n));
    pending.erase(pending.begin(), pending.begin() + n);
    std::vector<int32_t> ptr{0};
    std::vector<int16_t> lay;
    std::vector<int32_t> idx;
    std::vector<int8_t> sgn;
    for (const Domain& d : cur) {
      lay.insert(lay.end(), d.lay.begin(), d.lay.end());
      idx.insert(idx.end(), d.idx.begin(), d.idx.end());
      sgn.insert(sgn.end(), d.sgn.begin(), d.sgn.end());
      ptr.push_back((int32_t)lay.size());
    }
    lay.push_back(0);   // keep the arrays non-empty
    idx.push_back(0);
    sgn.push_back(0);
    const gcp_subdomains sub{(int32_t)n, ptr.data(), lay.data(), idx.data(), sgn.data()};
    Batch* b = nullptr;
    gcp_status s;
    {
      AllocPool g;   // every round's batch reuses the previous round's memory
      s = duals_create(c, net_id, cutset_id, &sub, GCP_FP32, &b);
    }
    if (s) return s;
    b->pool_stream = c.stream;
    const int64_t R = b->R;
    const int M = b->M, N = b->N;
    const int L1 = net.L - 1;
    // warm start: each child's rows from its parent's rows on the device (new split slots 0)
    bool warm = false;
    for (const Domain& d : cur) warm |= (bool)d.par;
    if (warm && L1 > 0) {
      std::vector<WarmSrc> src((size_t)R);
      for (size_t q = 0; q < n; ++q) {
        const Domain& d = cur[q];
        for (int k = 0; k < K; ++k) {
          WarmSrc& w = src[q * K + k];
          w = WarmSrc{};
          if (!d.par) continue;
          const int64_t pr = d.prow + k;
          if (pr < 0 || pr >= d.par->rows) {
            cudaStreamSynchronize(c.stream);
            c.batches.erase(b);
            return c.fail(GCP_EINVAL, "branch and bound: parent row %lld outside its store", (long long)pr);
          }
          w.alpha = d.par->alpha + pr * na;
          w.beta = d.par->M > 0 ? d.par->beta + pr * d.par->M : nullptr;
          w.gamma = N > 0 ? d.par->gamma + pr * N : nullptr;
          w.np = std::min<int>((int)d.lay.size() - 1, d.par->M);
        }
      }
      std::vector<int> dims(L1);
      std::vector<float*> aptr(L1);
      for (int l = 0; l < L1; ++l) {
        dims[l] = net.dims[l + 1];
        aptr[l] = (float*)b->alpha[l];
      }
      WarmSrc* src_d = (WarmSrc*)b->ws("bab_src", src.size() * sizeof(WarmSrc), &s);
      int* dims_d = src_d ? (int*)b->ws("bab_dims", dims.size() * sizeof(int), &s) : nullptr;
      float** aptr_d = dims_d ? (float**)b->ws("bab_aptr", aptr.size() * sizeof(float*), &s) : nullptr;
      if (aptr_d) {
        cudaMemcpyAsync(src_d, src.data(), src.size() * sizeof(WarmSrc), cudaMemcpyHostToDevice, c.stream);
        cudaMemcpyAsync(dims_d, dims.data(), dims.size() * sizeof(int), cudaMemcpyHostToDevice, c.stream);
        cudaMemcpyAsync(aptr_d, aptr.data(), aptr.size() * sizeof(float*), cudaMemcpyHostToDevice, c.stream);
        bab_warm_start(c.stream, R, L1, dims_d, aptr_d, na, (float*)b->beta, M, (float*)b->gamma, N, src_d);
        if (!reg_take_error().empty()) s = c.fail(GCP_EDEVICE, "branch and bound: warm start launch check");
      }
    }
    std::vector<double> cert((size_t)R);
    // branching by the duals: the round's last evaluation keeps nuhat for the score
    const bool by_duals = bp.branching == 0 && p.prec != GCP_FP64 && !b->fp64;
    b->keep_nuhat = by_duals;
    if (s == GCP_OK) s = optimize_batch(c, *b, &p, nullptr, cert.data(), nullptr);
    std::vector<int32_t> picks;
    if (s == GCP_OK && by_duals && !b->recompute) {
      int32_t* pd = (int32_t*)b->ws("bab_picks", n * 4, &s);
      if (pd) s = branch_picks_from_last_eval(c, *b, c.stream, pd);
      if (s == GCP_OK) {
        picks.resize(n);
        s = c.cuda(cudaMemcpy(picks.data(), pd, n * 4, cudaMemcpyDeviceToHost), "branch and bound: picks");
      }
    }
    // the subdomains that branch keep their rows of this round's duals on the
    // device for their children (only those rows, gathered by runs of
    // consecutive branching subdomains); if the store cannot be allocated the
    // children start from the default duals instead
    std::shared_ptr<ParentStore> store;
    std::vector<int64_t> store_slot(n, -1);   // first store row of subdomain q
    if (s == GCP_OK) {
      int64_t nb = 0;
      for (size_t q = 0; q < n; ++q) {
        bool br = false;
        for (int k = 0; k < K; ++k) br |= !(cert[q * K + k] > 0);
        if (br) store_slot[q] = (nb++) * K;
      }
      if (nb > 0) {
        const int64_t rows = nb * K;
        auto st_ = std::make_shared<ParentStore>();
        st_->c = &c;
        st_->rows = rows;
        st_->M = M;
        {
          AllocPool g;
          st_->alpha = (float*)c.alloc((size_t)rows * std::max<int64_t>(na, 1) * 4);
          st_->beta = (float*)c.alloc((size_t)rows * std::max(M, 1) * 4);
          st_->gamma = (float*)c.alloc((size_t)rows * std::max(N, 1) * 4);
        }
        if (st_->alpha && st_->beta && st_->gamma) {
          store = st_;
          for (size_t q0 = 0; q0 < n && s == GCP_OK;) {
            if (store_slot[q0] < 0) {
              ++q0;
              continue;
            }
            size_t q1 = q0 + 1;   // a run of consecutive branching subdomains
            while (q1 < n && store_slot[q1] >= 0) ++q1;
            const int64_t src = (int64_t)q0 * K, dst = store_slot[q0], cnt = (int64_t)(q1 - q0) * K;
            int64_t off = 0;
            for (int l = 0; l < L1 && s == GCP_OK; ++l) {
              const int d = net.dims[l + 1];
              const cudaError_t e =
                  cudaMemcpy2DAsync(store->alpha + dst * na + off, (size_t)na * 4, (float*)b->alpha[l] + src * d,
                                    (size_t)d * 4, (size_t)d * 4, (size_t)cnt, cudaMemcpyDeviceToDevice, c.stream);
              if (e) s = c.cuda(e, "branch and bound: store alpha");
              off += d;
            }
            if (s == GCP_OK && M > 0)
              s = c.cuda(cudaMemcpyAsync(store->beta + dst * M, (float*)b->beta + src * M, (size_t)cnt * M * 4,
                                         cudaMemcpyDeviceToDevice, c.stream), "branch and bound: store beta");
            if (s == GCP_OK && N > 0)
              s = c.cuda(cudaMemcpyAsync(store->gamma + dst * N, (float*)b->gamma + src * N, (size_t)cnt * N * 4,
                                         cudaMemcpyDeviceToDevice, c.stream), "branch and bound: store gamma");
            q0 = q1;
          }
        }
        // else: st_ gives back what it got; store stays null (default duals)
      }
    }
    cudaStreamSynchronize(c.stream);
    c.batches.erase(b);
    if (s) return s;
    res.rounds += 1;
    res.domains_bounded += (int64_t)n;
    for (size_t q = 0; q < n; ++q) {
      Domain& d = cur[q];
      double m = INFINITY;
      for (int k = 0; k < K; ++k) m = std::min(m, cert[q * K + k]);
      if (m > 0) {   // a verified leaf
        res.domains_verified += 1;
        res.min_bound = std::min(res.min_bound, m);
        continue;
      }
      // branch: the duals' pick (never a neuron already split here), else
      // the first candidate of the static order not split in this domain
      const Cand* pick = nullptr;
      Cand dual_pick{};
      if (!picks.empty() && picks[q] >= 0) {
        dual_pick = Cand{0.0, (int16_t)(picks[q] >> 24), picks[q] & 0xffffff};
        pick = &dual_pick;
      }
      for (size_t ci = 0; ci < cand.size() && !pick; ++ci) {
        const Cand& cd = cand[ci];
        bool dup = false;
        for (size_t e = 0; e < d.lay.size() && !dup; ++e) dup = d.lay[e] == cd.layer && d.idx[e] == cd.index;
        if (!dup) pick = &cd;
      }
      if (!pick) {   // every root-unstable neuron is split: nothing left to refine
        undecided = true;
        res.min_bound = std::min(res.min_bound, m);
        continue;
      }
      for (int side = 0; side < 2; ++side) {
        Domain ch;
        ch.lay = d.lay;
        ch.idx = d.idx;
        ch.sgn = d.sgn;
        ch.lay.push_back(pick->layer);
        ch.idx.push_back(pick->index);
        ch.sgn.push_back(side == 0 ? 1 : -1);
        ch.margin = m;
        ch.par = store;
        ch.prow = store ? store_slot[q] : 0;
        pending.push_back(std::move(ch));
      }
    }
    if (undecided) break;
  }
  for (const Domain& d : pending) res.min_bound = std::min(res.min_bound, d.margin);
  res.domains_left = (int64_t)pending.size();
  res.verified = (!undecided && pending.empty()) ? 1 : 0;
  res.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return GCP_OK;
}

namespace {

// A one-spec-row view of a network: the same device weights and bounds, the
// spec-derived arrays offset to row k; it owns nothing.
int label_view(Ctx& c, const Net& net, int k) {
  auto v = std::make_unique<Net>(net);
  v->owned.clear();
  const int dL = net.dims[net.L], dl1 = net.dims[net.L - 1];
  v->K = 1;
  v->C64 = net.C64 + (size_t)k * dL;
  v->negC64 = net.negC64 + (size_t)k * dL;
  v->YL64 = net.YL64 + (size_t)k * dl1;
  v->YL32 = net.YL32 + (size_t)k * dl1;
  v->cb64 = net.cb64 + k;
  v->cb32 = net.cb32 + k;
  if (net.skip[net.L - 1]) {
    const int dm = net.dims[net.skip[net.L - 1] - 1];
    if (net.SK64) v->SK64 = net.SK64 + (size_t)k * dm;
    if (net.SK32) v->SK32 = net.SK32 + (size_t)k * dm;
  }
  const int id = c.next_id++;
  c.nets[id] = std::move(v);
  return id;
}

}  // namespace

gcp_status bab_verify_labels(Ctx& c, int net_id, int cutset_id, const gcp_bab_params& bp, bool stop_at_failure,
                             int32_t* order, int32_t* label_verified, gcp_bab_result& res) {
  const auto t0 = std::chrono::steady_clock::now();
  auto it = c.nets.find(net_id);
  if (it == c.nets.end()) return c.fail(GCP_ENOTFOUND, "unknown network %d", net_id);
  if (cutset_id >= 0 && c.cutsets.find(cutset_id) == c.cutsets.end())
    return c.fail(GCP_ENOTFOUND, "unknown cut set %d", cutset_id);
  const Net& net = *it->second;
  const int K = net.K;
  // root bounds of every label: one subdomain, no splits
  std::vector<double> root(K);
  {
    std::vector<int32_t> ptr{0, 0};
    std::vector<int16_t> lay{0};
    std::vector<int32_t> idx{0};
    std::vector<int8_t> sgn{0};
    const gcp_subdomains sub{1, ptr.data(), lay.data(), idx.data(), sgn.data()};
    Batch* b = nullptr;
    gcp_status s = duals_create(c, net_id, cutset_id, &sub, GCP_FP32, &b);
    gcp_opt_params p = bp.p;
    p.certify = 1;
    if (s == GCP_OK) s = optimize_batch(c, *b, &p, nullptr, root.data(), nullptr);
    if (b) {
      cudaStreamSynchronize(c.stream);
      c.batches.erase(b);
    }
    if (s) return s;
  }
  // positive labels are done; the others by closeness of their root bound to zero
  std::vector<int> lab(K);
  for (int k = 0; k < K; ++k) lab[k] = k;
  std::stable_sort(lab.begin(), lab.end(), [&](int a, int b) {
    const bool pa = root[a] > 0, pb = root[b] > 0;
    if (pa != pb) return pa;
    return pa ? false : root[a] > root[b];
  });
  res = gcp_bab_result{};
  res.rounds = 1;
  res.domains_bounded = 1;
  res.min_bound = INFINITY;
  bool all = true, failed = false;
  for (int q = 0; q < K; ++q) {
    const int k = lab[q];
    order[q] = k;
    if (root[k] > 0) {
      label_verified[k] = 1;
      res.min_bound = std::min(res.min_bound, root[k]);
      continue;
    }
    if (failed && stop_at_failure) {
      label_verified[k] = -1;
      all = false;
      continue;
    }
    const int vid = label_view(c, net, k);
    int vcs = -1;
    if (cutset_id >= 0) {
      auto cs = std::make_unique<CutSet>(*c.cutsets[cutset_id]);
      cs->net_id = vid;
      vcs = c.next_id++;
      c.cutsets[vcs] = std::move(cs);
    }
    gcp_bab_result r{};
    const gcp_status s = bab_verify(c, vid, vcs, bp, r);
    if (vcs >= 0) c.cutsets.erase(vcs);
    c.nets.erase(vid);
    if (s) return s;
    label_verified[k] = r.verified;
    all = all && r.verified;
    failed = failed || !r.verified;
    res.rounds += r.rounds;
    res.domains_bounded += r.domains_bounded;
    res.domains_verified += r.domains_verified;
    res.domains_left += r.domains_left;
    res.min_bound = std::min(res.min_bound, r.min_bound);
  }
  res.verified = all ? 1 : 0;
  res.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return GCP_OK;
}

}  // namespace gcp

extern "C" gcp_status gcp_bab_verify_labels(gcp_ctx* h, int32_t net_id, int32_t cutset_id, const gcp_bab_params* bp,
                                            int32_t stop_at_failure, int32_t* label_order, int32_t* label_verified,
                                            gcp_bab_result* res) {
  gcp::Ctx* c = reinterpret_cast<gcp::Ctx*>(h);
  if (!c || !bp || !res || !label_order || !label_verified) return GCP_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  cudaSetDevice(c->device);
  auto it = c->nets.find(net_id);
  if (it == c->nets.end()) return c->fail(GCP_ENOTFOUND, "unknown network %d", net_id);
  const int K = it->second->K;
  std::vector<int32_t> ord(K), ver(K);
  gcp_bab_result r{};
  const gcp_status s = gcp::bab_verify_labels(*c, net_id, cutset_id, *bp, stop_at_failure != 0, ord.data(), ver.data(), r);
  if (s == GCP_OK) {
    std::copy(ord.begin(), ord.end(), label_order);
    std::copy(ver.begin(), ver.end(), label_verified);
    *res = r;
  }
  return s;
}

extern "C" gcp_status gcp_bab_verify(gcp_ctx* h, int32_t net_id, int32_t cutset_id, const gcp_bab_params* bp,
                                     gcp_bab_result* res) {
  gcp::Ctx* c = reinterpret_cast<gcp::Ctx*>(h);
  if (!c || !bp || !res) return GCP_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  cudaSetDevice(c->device);
  gcp_bab_result r{};
  const gcp_status s = gcp::bab_verify(*c, net_id, cutset_id, *bp, r);
  if (s == GCP_OK) *res = r;
  return s;
}

// Serving loop: continuous batching of verification requests.
//
// A request is a branch-and-bound query (App. B): a set of subdomains of one
// network with one cut set, optimised and certified for a number of rounds;
// after each round every subdomain is replaced by one child (one more split
// on a root-unstable neuron, chosen by the request's seed, on a random side)
// whose duals are warm-started from the parent. The paper runs this loop for
// one property with cuts arriving from a MIP solver (Sec. 3.2); here many
// such queries share one GPU.
//
// The scheduler thread admits submitted requests while fewer than
// max_inflight run and their device memory fits the context's budget. Every
// round, the active requests are grouped by network; each group becomes one
// merged batch (several queries, one cut set per query) evaluated by shared
// launches on that network's stream, and the groups of different networks
// run concurrently from worker threads. Requests submitted meanwhile join at
// the next round. Between rounds each request's duals stay on the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <random>
#include <thread>
#include <tuple>
#include <vector>

#include "gcp_ctx.h"

namespace gcp {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int net_id = 0, cutset_id = -1, rounds = 1, done = 0;
  gcp_opt_params p{};
  std::mt19937_64 rng;
  // current subdomains (host)
  std::vector<int32_t> ptr;
  std::vector<int16_t> layer;
  std::vector<int32_t> index;
  std::vector<int8_t> sign;
  int S = 0, K = 0, N = 0, Mcap = 0;
  int64_t R = 0, na = 0;
  // resident duals between rounds (float32, device): alpha [R, na], beta [R, Mcap], gamma [R, N]
  float* alpha = nullptr;
  float* beta = nullptr;
  float* gamma = nullptr;
  size_t resident_bytes = 0, estimate = 0;
  // results of the last round
  std::vector<double> certified;
  double min_cert = 0, max_err = 0, max_rel_err = 0;
  // keep_final: the last round's duals, copied to the host when it finishes
  bool keep_final = false;
  std::vector<float> fin_alpha, fin_beta, fin_gamma;
  gcp_status status = GCP_PENDING;
  Clock::time_point t_submit, t_done;
};

struct Serve {
  Ctx* ctx = nullptr;
  int max_inflight = 1;
  std::thread thr;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<std::unique_ptr<Request>> pending;
  std::vector<std::unique_ptr<Request>> active;
  std::map<uint64_t, std::unique_ptr<Request>> finished;
  std::map<uint64_t, std::unique_ptr<Request>> kept;   // taken keep_final results, for gcp_serve_final
  std::map<int, cudaStream_t> streams;   // one per network
  size_t reserved = 0;                   // device bytes promised to admitted requests
};

namespace {

// Device bytes a request needs: its resident duals plus its share of a
// merged batch (chain, adjoint, Adam and certification workspace per row).
size_t estimate_bytes(const Net& net, int64_t R, int N, int64_t nnz, int Mcap) {
  int64_t sum_d = 0, dmax = 1, P = 0;
  for (int i = 0; i < net.L; ++i) {
    if (i > 0) sum_d += net.dims[i];
    dmax = std::max<int64_t>(dmax, net.dims[i]);
    P += (net.dims[i] + kChunk - 1) / kChunk;
  }
  // certification by exact slices: bf16 slices of nu and the fp32 slice sums
  int smax = 0;
  for (const SliceB& sl : net.WTsl) smax = std::max(smax, sl.s);
  // skips from further back than the layer's input park nu, S^T nu, a (fp32)
  // and the certification's term and its magnitude bound, of their source's
  // width; projections add one product buffer of each kind
  // (the mixed-precision chain adds nu's three-term bf16 operand and its
  // float form, 10 bytes per neuron of the widest layer)
  int64_t parked = 0;
  bool proj = false;
  for (int m = 0; m < net.L; ++m)
    if (net.consumer[m] > m + 1 && net.consumer[m] < net.L) parked += net.dims[m];
  for (int i = 0; i < net.L; ++i) proj |= net.sc_map[i] != 0;
  const double per_row = 4.0 * (5 * sum_d + 5 * dmax + nnz + 3 * N + 3 * Mcap) + 8.0 * (2 * dmax + P) +
                         4.0 * (dmax + P) + 6.0 * smax * dmax + 24.0 * parked + (proj ? 28.0 * dmax : 0.0) +
                         10.0 * dmax;
  const double resident = 4.0 * (sum_d + Mcap + N);
  return (size_t)(R * (per_row + resident)) + (size_t(16) << 20);
}

void free_resident(Ctx& c, Request& q) {
  c.release(q.alpha);
  c.release(q.beta);
  c.release(q.gamma);
  q.alpha = q.beta = q.gamma = nullptr;
}

// One more split per subdomain: a root-unstable neuron not yet split in it,
// chosen uniformly by the request's generator, on a random side.
void branch(const Net& net, Request& q) {
  std::vector<int32_t> ptr(1, 0);
  std::vector<int16_t> lay;
  std::vector<int32_t> idx;
  std::vector<int8_t> sgn;
  int64_t total = 0;
  for (int i = 1; i < net.L; ++i) total += (int64_t)net.unstable[i - 1].size();
  for (int s = 0; s < q.S; ++s) {
    const int a = q.ptr[s], b = q.ptr[s + 1];
    for (int e = a; e < b; ++e) {
      lay.push_back(q.layer[e]);
      idx.push_back(q.index[e]);
      sgn.push_back(q.sign[e]);
    }
    if (b - a < q.Mcap && total > b - a) {
      for (int tries = 0; tries < 64; ++tries) {
        int64_t u = (int64_t)(q.rng() % (uint64_t)total);
        int li = 1;
        while (u >= (int64_t)net.unstable[li - 1].size()) { u -= net.unstable[li - 1].size(); ++li; }
        const int j = net.unstable[li - 1][u];
        bool dup = false;
        for (int e = a; e < b && !dup; ++e) dup = q.layer[e] == li && q.index[e] == j;
        if (dup) continue;
        lay.push_back((int16_t)li);
        idx.push_back(j);
        sgn.push_back((q.rng() & 1) ? 1 : -1);
        break;
      }
    }
    ptr.push_back((int32_t)lay.size());
  }
  q.ptr.swap(ptr);
  q.layer.swap(lay);
  q.index.swap(idx);
  q.sign.swap(sgn);
}

// One round for the requests of one network: merged batch, warm start,
// optimise + certify on the network's stream, results and duals back.
void run_group(Serve& sv, int net_id, cudaStream_t st, std::vector<Request*> group) {
  Ctx& c = *sv.ctx;
  AllocPool pooled;   // the merged batch's blocks come from and go back to the pool
  const Net* netp = nullptr;
  Batch* b = nullptr;
  gcp_status status = GCP_OK;
  std::vector<gcp_subdomains> subs(group.size());
  std::vector<std::pair<const CutSet*, const gcp_subdomains*>> parts;
  {
    std::lock_guard<std::recursive_mutex> lk(c.mu);
    cudaSetDevice(c.device);
    for (size_t g = 0; g < group.size(); ++g) {
      Request& q = *group[g];
      subs[g] = gcp_subdomains{q.S, q.ptr.data(), q.layer.data(), q.index.data(), q.sign.data()};
      const CutSet* cs = nullptr;
      auto ci = c.cutsets.find(q.cutset_id);
      if (q.cutset_id >= 0 && ci != c.cutsets.end()) cs = ci->second.get();
      parts.push_back({cs, &subs[g]});
    }
    netp = c.nets.at(net_id).get();
    status = duals_create_parts(c, net_id, parts, GCP_FP32, &b);
    if (status == GCP_OK) status = c.cuda(cudaStreamSynchronize(c.stream), "serve batch");
    if (b) b->pool_stream = st;
  }
  cudaSetDevice(c.device);
  const Net& net = *netp;
  double* cert = nullptr;
  std::vector<double> h_bound, h_cert;
  if (status == GCP_OK) {
    // warm start: copy each request's resident duals into its rows
    int64_t r0 = 0, cut0 = 0;
    for (Request* q : group) {
      if (q->done > 0) {
        int64_t coff = 0;
        for (int i = 1; i < net.L; ++i) {
          const int di = net.dims[i];
          cudaMemcpy2DAsync((float*)b->alpha[i - 1] + r0 * di, di * 4, q->alpha + coff, q->na * 4, di * 4, q->R,
                            cudaMemcpyDeviceToDevice, st);
          coff += di;
        }
        const int mc = std::min(q->Mcap, b->M);
        if (mc > 0)
          cudaMemcpy2DAsync((float*)b->beta + r0 * b->M, b->M * 4, q->beta, q->Mcap * 4, mc * 4, q->R,
                            cudaMemcpyDeviceToDevice, st);
        if (q->N > 0)
          cudaMemcpy2DAsync((float*)b->gamma + r0 * b->N + cut0, b->N * 4, q->gamma, q->N * 4, q->N * 4, q->R,
                            cudaMemcpyDeviceToDevice, st);
      }
      r0 += q->R;
      cut0 += q->N;
    }
    gcp_status s2 = GCP_OK;
    cert = (double*)b->ws("serve_cert", (size_t)std::max<int64_t>(b->R, 1) * 8, &s2);
    gcp_opt_params p = group[0]->p;
    p.certify = 1;
    status = cert ? optimize_on(c, *b, p, st, cert) : s2;
    if (status == GCP_OK) {
      h_bound.resize(b->R);
      h_cert.resize(b->R);
      double* gb = (double*)b->ws("serve_bound", (size_t)std::max<int64_t>(b->R, 1) * 8, &s2);
      if (!gb) status = s2;
      else {
        cast_copy<float, double>(st, b->R, (const float*)b->lazy["g"], gb);
        cudaMemcpyAsync(h_bound.data(), gb, b->R * 8, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(h_cert.data(), cert, b->R * 8, cudaMemcpyDeviceToHost, st);
        // duals back to the requests
        r0 = 0;
        cut0 = 0;
        for (Request* q : group) {
          int64_t coff = 0;
          for (int i = 1; i < net.L; ++i) {
            const int di = net.dims[i];
            cudaMemcpy2DAsync(q->alpha + coff, q->na * 4, (float*)b->alpha[i - 1] + r0 * di, di * 4, di * 4, q->R,
                              cudaMemcpyDeviceToDevice, st);
            coff += di;
          }
          const int mc = std::min(q->Mcap, b->M);
          if (mc > 0)
            cudaMemcpy2DAsync(q->beta, q->Mcap * 4, (float*)b->beta + r0 * b->M, b->M * 4, mc * 4, q->R,
                              cudaMemcpyDeviceToDevice, st);
          if (q->N > 0)
            cudaMemcpy2DAsync(q->gamma, q->N * 4, (float*)b->gamma + r0 * b->N + cut0, b->N * 4, q->N * 4, q->R,
                              cudaMemcpyDeviceToDevice, st);
          r0 += q->R;
          cut0 += q->N;
        }
        status = sync_check(c, st, "serve round");
      }
    }
  }
  {
    std::lock_guard<std::recursive_mutex> lk(c.mu);
    if (b) {
      cudaStreamSynchronize(st);
      c.batches.erase(b);
    }
  }
  int64_t r0 = 0;
  for (Request* q : group) {
    if (status != GCP_OK) {
      q->status = status;
      q->done = q->rounds;
      continue;
    }
    q->certified.assign(h_cert.begin() + r0, h_cert.begin() + r0 + q->R);
    q->min_cert = q->R ? *std::min_element(q->certified.begin(), q->certified.end()) : 0.0;
    q->max_err = 0;
    q->max_rel_err = 0;
    for (int64_t r = 0; r < q->R; ++r) {
      const double e = std::fabs(h_bound[r0 + r] - h_cert[r0 + r]);
      q->max_err = std::max(q->max_err, e);
      q->max_rel_err = std::max(q->max_rel_err, e / std::max(1.0, std::fabs(h_cert[r0 + r])));
    }
    r0 += q->R;
    q->done += 1;
    if (q->done < q->rounds) branch(net, *q);
    else q->status = GCP_OK;
  }
}

void scheduler(Serve* sv) {
  Ctx& c = *sv->ctx;
  cudaSetDevice(c.device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv.wait(lk, [&] { return sv->stop || !sv->pending.empty() || !sv->active.empty(); });
      if (sv->stop && sv->pending.empty() && sv->active.empty()) break;
      // admission: slots and device memory
      while (!sv->pending.empty() && (int)sv->active.size() < sv->max_inflight) {
        Request& q = *sv->pending.front();
        if (c.budget && sv->reserved + q.estimate > c.budget && !sv->active.empty()) break;
        const size_t ab = (size_t)q.R * q.na * 4, bb = (size_t)q.R * std::max(q.Mcap, 1) * 4,
                     gb = (size_t)q.R * std::max(q.N, 1) * 4;
        q.alpha = (float*)c.alloc(ab);
        q.beta = (float*)c.alloc(bb);
        q.gamma = (float*)c.alloc(gb);
        if (!q.alpha || !q.beta || !q.gamma) {
          free_resident(c, q);
          if (!sv->active.empty()) break;       // wait for memory to free up
          q.status = GCP_EBUDGET;               // cannot run even alone
          q.t_done = Clock::now();
          sv->finished[q.ticket] = std::move(sv->pending.front());
          sv->pending.pop_front();
          sv->done_cv.notify_all();
          continue;
        }
        cudaMemsetAsync(q.beta, 0, bb, c.stream);
        cudaMemsetAsync(q.gamma, 0, gb, c.stream);
        cudaStreamSynchronize(c.stream);
        q.resident_bytes = ab + bb + gb;
        sv->reserved += q.estimate;
        if (!sv->streams.count(q.net_id)) {
          cudaStream_t s = nullptr;
          cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
          sv->streams[q.net_id] = s;
        }
        sv->active.push_back(std::move(sv->pending.front()));
        sv->pending.pop_front();
      }
    }
    // one round for every active request: one merged batch per network and
    // optimiser schedule, groups of different networks run concurrently
    std::map<std::tuple<int, int, int, int, double, double, double, double>, std::vector<Request*>> groups;
    for (auto& q : sv->active) {
      const gcp_opt_params& p = q->p;
      groups[std::make_tuple(q->net_id, p.iters, p.optimizer, p.prec, p.lr_alpha, p.lr_beta, p.lr_gamma, p.lr_decay)]
          .push_back(q.get());
    }
    std::vector<std::thread> workers;
    for (auto& g : groups) {
      const int net_id = std::get<0>(g.first);
      workers.emplace_back(run_group, std::ref(*sv), net_id, sv->streams[net_id], g.second);
    }
    for (auto& t : workers) t.join();
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      for (auto it = sv->active.begin(); it != sv->active.end();) {
        Request& q = **it;
        if (q.done >= q.rounds) {
          if (q.keep_final && q.status == GCP_OK) {
            // the round's stream was synchronised: the resident duals are final
            q.fin_alpha.resize((size_t)q.R * q.na);
            q.fin_beta.resize((size_t)q.R * q.Mcap);
            q.fin_gamma.resize((size_t)q.R * q.N);
            cudaError_t e = cudaSuccess;
            if (!q.fin_alpha.empty())
              e = cudaMemcpy(q.fin_alpha.data(), q.alpha, q.fin_alpha.size() * 4, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && !q.fin_beta.empty())
              e = cudaMemcpy(q.fin_beta.data(), q.beta, q.fin_beta.size() * 4, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && !q.fin_gamma.empty())
              e = cudaMemcpy(q.fin_gamma.data(), q.gamma, q.fin_gamma.size() * 4, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) q.status = GCP_ECUDA;
          }
          free_resident(c, q);
          sv->reserved -= std::min(sv->reserved, q.estimate);
          q.t_done = Clock::now();
          sv->finished[q.ticket] = std::move(*it);
          it = sv->active.erase(it);
        } else {
          ++it;
        }
      }
      sv->done_cv.notify_all();
    }
  }
}

// A taken result is forgotten, unless its request keeps its final state for
// gcp_serve_final.
void take_finished(Serve& sv, std::map<uint64_t, std::unique_ptr<Request>>::iterator it) {
  if (it->second->keep_final) sv.kept[it->first] = std::move(it->second);
  sv.finished.erase(it);
}

gcp_status fill_result(Request& q, gcp_result* res) {
  res->status = q.status;
  res->rows = (int32_t)q.certified.size();
  if (res->certified) std::copy(q.certified.begin(), q.certified.end(), res->certified);
  res->min_certified = q.min_cert;
  res->max_err_vs_fp64 = q.max_err;
  res->max_rel_err_vs_fp64 = q.max_rel_err;
  res->latency_ms = std::chrono::duration<double, std::milli>(q.t_done - q.t_submit).count();
  return GCP_OK;
}

}  // namespace

void serve_shutdown(Ctx& c) {
  Serve* sv = c.serve;
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  if (sv->thr.joinable()) sv->thr.join();
  for (auto& kv : sv->streams) cudaStreamDestroy(kv.second);
  for (auto& q : sv->active) free_resident(c, *q);
  delete sv;
  c.serve = nullptr;
  c.trim();
}

}  // namespace gcp

using gcp::Ctx;

extern "C" {

gcp_status gcp_serve_start(gcp_ctx* h, int32_t max_inflight) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  if (!c || max_inflight < 1) return GCP_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  if (c->serve) return c->fail(GCP_EINVAL, "serving loop already running");
  auto* sv = new gcp::Serve();
  sv->ctx = c;
  sv->max_inflight = max_inflight;
  c->serve = sv;
  sv->thr = std::thread(gcp::scheduler, sv);
  return GCP_OK;
}

gcp_status gcp_serve_submit(gcp_ctx* h, const gcp_request* req, uint64_t* ticket) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  if (!c || !req || !ticket) return GCP_EINVAL;
  std::unique_ptr<gcp::Request> q(new gcp::Request());
  {
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    if (!c->serve) return c->fail(GCP_EINVAL, "serving loop not started");
    auto ni = c->nets.find(req->net_id);
    if (ni == c->nets.end()) return c->fail(GCP_ENOTFOUND, "unknown net %d", req->net_id);
    const gcp::Net& net = *ni->second;
    int N = 0;
    int64_t nnz = 0;
    if (req->cutset_id >= 0) {
      auto ci = c->cutsets.find(req->cutset_id);
      if (ci == c->cutsets.end()) return c->fail(GCP_ENOTFOUND, "unknown cut set %d", req->cutset_id);
      if (ci->second->net_id != req->net_id) return c->fail(GCP_EINVAL, "cut set of another net");
      N = (int)ci->second->d.size();
      nnz = (int64_t)ci->second->coef.size();
    }
    const gcp_subdomains& sd = req->sub;
    if (sd.n_sub < 0 || (sd.n_sub > 0 && !sd.split_ptr) || req->rounds < 1 || req->p.prec == GCP_FP64)
      return c->fail(GCP_EINVAL, "bad request (subdomains, rounds >= 1, FP32/BF16 chain)");
    int M = 0;
    for (int s = 0; s < sd.n_sub; ++s) M = std::max(M, sd.split_ptr[s + 1] - sd.split_ptr[s]);
    if (M + req->rounds - 1 > gcp::kMaxSplits) return c->fail(GCP_EINVAL, "too many splits after the rounds");
    const int64_t nsp = sd.n_sub ? sd.split_ptr[sd.n_sub] : 0;
    q->ptr.assign(sd.split_ptr, sd.split_ptr + sd.n_sub + 1);
    if (sd.n_sub == 0) q->ptr.assign(1, 0);
    if (nsp > 0) {
      if (!sd.split_layer || !sd.split_index || !sd.split_sign) return c->fail(GCP_EINVAL, "null split arrays");
      q->layer.assign(sd.split_layer, sd.split_layer + nsp);
      q->index.assign(sd.split_index, sd.split_index + nsp);
      q->sign.assign(sd.split_sign, sd.split_sign + nsp);
    }
    q->net_id = req->net_id;
    q->cutset_id = req->cutset_id;
    q->rounds = req->rounds;
    q->p = req->p;
    q->rng.seed(req->seed);
    q->keep_final = req->keep_final != 0;
    q->S = sd.n_sub;
    q->K = net.K;
    q->R = (int64_t)q->S * q->K;
    q->N = N;
    q->Mcap = std::max(1, M + req->rounds - 1);
    for (int i = 1; i < net.L; ++i) q->na += net.dims[i];
    q->estimate = gcp::estimate_bytes(net, q->R, N, nnz, q->Mcap);
    if (q->p.opt_pi) q->estimate += (size_t)(12.0 * (double)q->R * (double)q->na);   // theta and its Adam moments
    if (c->budget && q->estimate > c->budget) return c->fail(GCP_EBUDGET, "request needs about %zu bytes", q->estimate);
  }
  gcp::Serve* sv = c->serve;
  q->t_submit = gcp::Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    q->ticket = sv->next_ticket++;
    *ticket = q->ticket;
    sv->pending.push_back(std::move(q));
  }
  sv->cv.notify_all();
  return GCP_OK;
}

gcp_status gcp_serve_poll(gcp_ctx* h, uint64_t ticket, gcp_result* res) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  if (!c || !res || !c->serve) return GCP_EINVAL;
  gcp::Serve* sv = c->serve;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->finished.find(ticket);
  if (it == sv->finished.end()) {
    for (auto& q : sv->pending)
      if (q->ticket == ticket) return GCP_PENDING;
    for (auto& q : sv->active)
      if (q->ticket == ticket) return GCP_PENDING;
    return GCP_ENOTFOUND;
  }
  gcp::fill_result(*it->second, res);
  gcp::take_finished(*sv, it);
  return GCP_OK;
}

gcp_status gcp_serve_wait(gcp_ctx* h, uint64_t ticket, int32_t timeout_ms, gcp_result* res) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  if (!c || !res || !c->serve) return GCP_EINVAL;
  gcp::Serve* sv = c->serve;
  std::unique_lock<std::mutex> lk(sv->mu);
  const bool ok = sv->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                       [&] { return sv->finished.count(ticket) > 0; });
  if (!ok) {
    bool known = false;
    for (auto& q : sv->pending) known = known || q->ticket == ticket;
    for (auto& q : sv->active) known = known || q->ticket == ticket;
    return known ? GCP_ETIMEOUT : GCP_ENOTFOUND;
  }
  auto it = sv->finished.find(ticket);
  gcp::fill_result(*it->second, res);
  gcp::take_finished(*sv, it);
  return GCP_OK;
}

gcp_status gcp_serve_final(gcp_ctx* h, uint64_t ticket, gcp_final* out) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  if (!c || !out || !c->serve) return GCP_EINVAL;
  gcp::Serve* sv = c->serve;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->kept.find(ticket);
  if (it == sv->kept.end()) return GCP_ENOTFOUND;
  gcp::Request& q = *it->second;
  if (q.status != GCP_OK) return GCP_EINVAL;
  out->n_sub = q.S;
  out->rows = (int32_t)q.R;
  out->n_alpha = (int32_t)q.na;
  out->max_splits = q.Mcap;
  out->n_cuts = q.N;
  out->n_split_entries = (int64_t)q.layer.size();
  if (!out->split_ptr || !out->split_layer || !out->split_index || !out->split_sign || !out->alpha ||
      !out->beta || !out->gamma)
    return GCP_OK;
  std::copy(q.ptr.begin(), q.ptr.end(), out->split_ptr);
  std::copy(q.layer.begin(), q.layer.end(), out->split_layer);
  std::copy(q.index.begin(), q.index.end(), out->split_index);
  std::copy(q.sign.begin(), q.sign.end(), out->split_sign);
  std::copy(q.fin_alpha.begin(), q.fin_alpha.end(), out->alpha);
  std::copy(q.fin_beta.begin(), q.fin_beta.end(), out->beta);
  std::copy(q.fin_gamma.begin(), q.fin_gamma.end(), out->gamma);
  sv->kept.erase(it);
  return GCP_OK;
}

gcp_status gcp_serve_stop(gcp_ctx* h) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  if (!c) return GCP_EINVAL;
  gcp::serve_shutdown(*c);
  return GCP_OK;
}

}  // extern "C"

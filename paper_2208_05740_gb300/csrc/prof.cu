// Launch accounting: every kernel launch of the library is counted; launches
// of the kernels selected by name prefix are bracketed by CUDA events on their
// own stream and accumulate device time plus their algorithmic flops and bytes
// (the minimum a launch must compute and move, from its shapes).
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "gcp_internal.cuh"

namespace gcp {
namespace {
struct Pending {
  std::string name;
  cudaEvent_t a, b;
  double flops, bytes;
};
struct Agg {
  int64_t launches = 0, timed = 0;
  double ms = 0, flops = 0, bytes = 0;
};
std::mutex g_mu;
bool g_on = false;
std::string g_sel;
std::vector<Pending> g_pend;
std::vector<cudaEvent_t> g_pool;
std::map<std::string, Agg> g_agg;
std::string g_rep;   // idempotent kernels whose launches are issued twice

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void drain_locked() {
  for (auto& p : g_pend) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      Agg& a = g_agg[p.name];
      a.ms += ms;
      a.timed += 1;
    }
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pend.clear();
}
}  // namespace

int prof_begin(cudaStream_t st, const char* name, double flops, double bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return -1;
  Agg& a = g_agg[name];
  a.launches += 1;
  a.flops += flops;
  a.bytes += bytes;
  if (g_sel.empty() || (g_sel != "*" && strncmp(name, g_sel.c_str(), g_sel.size()) != 0)) return -1;
  Pending p{name, take_event(), take_event(), flops, bytes};
  cudaEventRecord(p.a, st);
  g_pend.push_back(p);
  return (int)g_pend.size() - 1;
}

void prof_end(cudaStream_t st, int token) {
  if (token < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (token < (int)g_pend.size()) cudaEventRecord(g_pend[token].b, st);
}

bool smem_opt_in(const void* kern, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> done;
  if (bytes <= 48 * 1024) return true;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  size_t& have = done[{dev, kern}];
  if (have >= bytes) return true;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  have = bytes;
  return true;
}

int prof_repeats(const char* name) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on || g_rep.empty()) return 1;
  return strncmp(name, g_rep.c_str(), g_rep.size()) == 0 ? 2 : 1;
}

}  // namespace gcp

using namespace gcp;

extern "C" {

gcp_status gcp_profile_start(const char* kernel_prefix) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  g_agg.clear();
  g_sel = kernel_prefix ? kernel_prefix : "";
  g_on = true;
  return GCP_OK;
}

gcp_status gcp_profile_stop(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  g_on = false;
  g_rep.clear();
  return GCP_OK;
}

gcp_status gcp_profile_repeat(const char* kernel_prefix) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_rep = kernel_prefix ? kernel_prefix : "";
  return GCP_OK;
}

gcp_status gcp_profile_query(const char* name, int64_t* launches, double* total_ms, double* flops, double* bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  Agg t;
  for (auto& kv : g_agg) {
    if (name && kv.first != name) continue;
    t.launches += kv.second.launches;
    t.ms += kv.second.ms;
    t.flops += kv.second.flops;
    t.bytes += kv.second.bytes;
  }
  if (launches) *launches = t.launches;
  if (total_ms) *total_ms = t.ms;
  if (flops) *flops = t.flops;
  if (bytes) *bytes = t.bytes;
  return GCP_OK;
}

gcp_status gcp_profile_report(char* buf, int64_t cap) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  if (!buf || cap <= 0) return GCP_EINVAL;
  std::string s;
  char line[256];
  for (auto& kv : g_agg) {
    snprintf(line, sizeof line, "%s %lld %lld %.6f %.6e %.6e\n", kv.first.c_str(), (long long)kv.second.launches,
             (long long)kv.second.timed, kv.second.ms, kv.second.flops, kv.second.bytes);
    s += line;
  }
  strncpy(buf, s.c_str(), (size_t)cap - 1);
  buf[cap - 1] = 0;
  return (int64_t)s.size() < cap ? GCP_OK : GCP_EINVAL;
}

}  // extern "C"

// ---------------------------------------------------------------- launch validation
namespace gcp {
namespace {
struct RegKey {
  int dev;
  uintptr_t base;
  bool operator<(const RegKey& o) const { return dev != o.dev ? dev < o.dev : base < o.base; }
};
struct Foreign {
  int dev;
  uintptr_t base;
  size_t bytes;
};
std::mutex g_reg_mu;
std::map<RegKey, size_t> g_reg;                 // the library's allocations (disjoint per device)
std::map<uint64_t, Foreign> g_foreign;          // caller arrays of calls in flight, by token
uint64_t g_next_token = 1;
thread_local std::string t_reg_err;             // the calling thread's first problem

int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return d;
}

bool covers(uintptr_t base, size_t bytes, uintptr_t a, double need, size_t& have) {
  if (a < base || a - base > bytes) return false;
  have = bytes - (a - base);
  return (double)have >= need;
}
}  // namespace

void reg_alloc(const void* p, size_t bytes) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_reg_mu);
  g_reg[RegKey{dev, (uintptr_t)p}] = bytes;
}

void reg_free(const void* p) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_reg_mu);
  g_reg.erase(RegKey{dev, (uintptr_t)p});
}

uint64_t reg_foreign(const void* p, size_t bytes) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_reg_mu);
  const uint64_t t = g_next_token++;
  g_foreign[t] = Foreign{dev, (uintptr_t)p, bytes};
  return t;
}

void reg_unforeign(uint64_t token) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  g_foreign.erase(token);
}

bool reg_check(const void* p, double bytes, const char* what) {
  if (bytes <= 0) return true;
  const int dev = current_device();
  const uintptr_t a = (uintptr_t)p;
  bool ok = false;
  size_t have = 0;
  {
    std::lock_guard<std::mutex> lk(g_reg_mu);
    if (p) {
      auto it = g_reg.upper_bound(RegKey{dev, a});
      if (it != g_reg.begin()) {
        --it;
        if (it->first.dev == dev) ok = covers(it->first.base, it->second, a, bytes, have);
      }
      for (auto f = g_foreign.begin(); !ok && f != g_foreign.end(); ++f)
        if (f->second.dev == dev) ok = covers(f->second.base, f->second.bytes, a, bytes, have);
    }
  }
  if (!ok && t_reg_err.empty()) {
    char buf[256];
    snprintf(buf, sizeof buf, "launch check failed: %s at %p needs %.0f bytes, allocation has %zu", what, p, bytes,
             have);
    t_reg_err = buf;
  }
  return ok;
}

std::string reg_take_error() {
  std::string e;
  e.swap(t_reg_err);
  return e;
}
}  // namespace gcp

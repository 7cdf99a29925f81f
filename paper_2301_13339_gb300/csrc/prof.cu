// Optional per-launch timing: when enabled, every instrumented launch is
// bracketed by two CUDA events recorded on its stream; qtt_profile_read
// synchronises and sums the elapsed times per kernel name.
#include "qtt_internal.cuh"
#include <cstring>
#include <map>
#include <mutex>
#include <string>

namespace qtt {

struct ProfRec {
  const char* name;
  cudaEvent_t a, b;
};
static bool g_prof_on = false;
static std::mutex g_prof_mu;
static std::vector<ProfRec> g_recs;
static std::vector<cudaEvent_t> g_pool;
// algorithmic work recorded by the launch sites: name -> (flop, bytes)
static std::map<std::string, std::pair<double, double>> g_work;

static cudaEvent_t ev_get() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

bool prof_enabled() { return g_prof_on; }

void prof_add_work(const char* name, double flops, double bytes) {
  if (!g_prof_on) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  auto& w = g_work[name];
  w.first += flops;
  w.second += bytes;
}

ProfScope::ProfScope(const char* name, cudaStream_t s) : name_(name), s_(s), active_(g_prof_on) {
  if (!active_) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  a_ = ev_get();
  b_ = ev_get();
  cudaEventRecord((cudaEvent_t)a_, s_);
}

ProfScope::~ProfScope() {
  if (!active_) return;
  cudaEventRecord((cudaEvent_t)b_, s_);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_recs.push_back({name_, (cudaEvent_t)a_, (cudaEvent_t)b_});
}

}  // namespace qtt

using namespace qtt;

extern "C" {

void qtt_profile_enable(int on) { g_prof_on = (on != 0); }

int qtt_profile_read(char* names, int name_stride, double* ms, int* counts, int cap) {
  cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  std::map<std::string, std::pair<double, int>> agg;
  for (auto& r : g_recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      auto& v = agg[r.name];
      v.first += t;
      v.second += 1;
    }
  }
  int n = 0;
  for (auto& kv : agg) {
    if (n >= cap) break;
    if (names) {
      strncpy(names + (size_t)n * name_stride, kv.first.c_str(), name_stride - 1);
      names[(size_t)n * name_stride + name_stride - 1] = 0;
    }
    if (ms) ms[n] = kv.second.first;
    if (counts) counts[n] = kv.second.second;
    ++n;
  }
  return n;
}

int qtt_profile_work(const char* name, double* flops, double* bytes) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  auto it = g_work.find(name ? name : "");
  if (it == g_work.end()) return 0;
  if (flops) *flops = it->second.first;
  if (bytes) *bytes = it->second.second;
  return 1;
}

void qtt_profile_reset(void) {
  cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_work.clear();
  for (auto& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
}

}  // extern "C"

// Launch counter and optional per-phase CUDA-event timing.
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "c2_internal.cuh"

namespace c2 {

std::atomic<long long> g_launches{0};

namespace {

struct Rec {
  const char* name;
  cudaEvent_t a, b;
  long long launches;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

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

}  // namespace

Prof::Prof(cudaStream_t st, const char* name) : st_(st), name_(name), idx_(-1), launches0_(0) {
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_on) return;
  Rec r{name, take_event(), take_event(), 0};
  cudaEventRecord(r.a, st_);
  launches0_ = g_launches.load();
  idx_ = (int)g_recs.size();
  g_recs.push_back(r);
}

void Prof::end() {
  std::lock_guard<std::mutex> g(g_mu);
  if (idx_ < 0 || idx_ >= (int)g_recs.size()) return;
  cudaEventRecord(g_recs[idx_].b, st_);
  g_recs[idx_].launches = g_launches.load() - launches0_;
  idx_ = -1;
}

}  // namespace c2

using namespace c2;

extern "C" {

int64_t c2_kernel_launches(void) { return (int64_t)g_launches.load(); }

void c2_profile_enable(int on) {
  std::lock_guard<std::mutex> g(g_mu);
  g_on = on != 0;
}

size_t c2_profile_report(char* buf, size_t len) {
  std::lock_guard<std::mutex> g(g_mu);
  const bool consume = buf != nullptr;
  struct Agg {
    double ms = 0;
    long long calls = 0, launches = 0;
  };
  std::map<std::string, Agg> agg;
  std::vector<std::string> order;
  for (Rec& r : g_recs) {
    float ms = 0.f;
    cudaEventSynchronize(r.b);
    cudaEventElapsedTime(&ms, r.a, r.b);
    if (!agg.count(r.name)) order.push_back(r.name);
    Agg& x = agg[r.name];
    x.ms += ms;
    x.calls += 1;
    x.launches += r.launches;
    if (consume) {
      g_pool.push_back(r.a);
      g_pool.push_back(r.b);
    }
  }
  if (consume) g_recs.clear();
  std::string out = "{";
  for (size_t i = 0; i < order.size(); ++i) {
    const Agg& x = agg[order[i]];
    char tmp[256];
    snprintf(tmp, sizeof tmp, "%s\"%s\": {\"ms\": %.6f, \"calls\": %lld, \"launches\": %lld}",
             i ? ", " : "", order[i].c_str(), x.ms, x.calls, x.launches);
    out += tmp;
  }
  out += "}";
  if (buf && len) {
    size_t n = out.size() < len - 1 ? out.size() : len - 1;
    memcpy(buf, out.data(), n);
    buf[n] = 0;
  }
  return out.size() + 1;
}

}  // extern "C"

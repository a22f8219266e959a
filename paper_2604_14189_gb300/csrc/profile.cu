// Optional per-launch event timing of the time-step kernels (benchmarks).
#include <atomic>
#include <mutex>
#include <vector>

#include "sweep_internal.cuh"

namespace sweep {
namespace {

struct Rec {
  int kernel;
  cudaEvent_t a, b;
};

std::mutex g_mu;
std::atomic<int> g_mask{0};  // bit k: record kernel class k
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void release_all() {
  for (auto& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
}

}  // namespace


void* profile_begin(int kernel, cudaStream_t st) {
  // checked before taking the lock: launches from several host threads do
  // not serialise on it while profiling is off
  if (kernel < 0 || kernel >= 31 || !((g_mask.load(std::memory_order_relaxed) >> kernel) & 1))
    return nullptr;
  if (t_capturing) return nullptr;  // calls recorded into a graph are not timed
  std::lock_guard<std::mutex> lk(g_mu);
  Rec r{kernel, take_event(), take_event()};
  if (!r.a || !r.b) return nullptr;
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  return reinterpret_cast<void*>(g_recs.size());
}

void profile_end(void* token, cudaStream_t st) {
  if (!token) return;
  std::lock_guard<std::mutex> lk(g_mu);
  const size_t i = reinterpret_cast<size_t>(token) - 1;
  if (i < g_recs.size()) cudaEventRecord(g_recs[i].b, st);
}

}  // namespace sweep

extern "C" int sweep_profile_enable(int mask) {
  std::lock_guard<std::mutex> lk(sweep::g_mu);
  sweep::release_all();
  sweep::g_mask.store(mask);
  return SWEEP_OK;
}

extern "C" int sweep_profile_read(int kernel, double* ms, long long* launches) {
  if (kernel < 0 || kernel >= SWEEP_K_COUNT || !ms || !launches) return SWEEP_EINVAL;
  std::lock_guard<std::mutex> lk(sweep::g_mu);
  double t = 0.0;
  long long n = 0;
  for (auto& r : sweep::g_recs) {
    if (r.kernel != kernel) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return SWEEP_ECUDA;
    float e = 0.f;
    if (cudaEventElapsedTime(&e, r.a, r.b) != cudaSuccess) return SWEEP_ECUDA;
    t += e;
    ++n;
  }
  *ms = t;
  *launches = n;
  return SWEEP_OK;
}

// Launch counter and per-class event timing (see profile.h).
#include <atomic>
#include <mutex>
#include <vector>

#include "ebv.h"
#include "profile.h"

namespace ebv {
namespace prof {

namespace {
std::atomic<long long> g_launches{0};
std::atomic<bool> g_enabled{false};
std::mutex g_mu;
struct Rec {
  cudaEvent_t a, b;
  int cls;
  double work;
  bool closed;
};
std::vector<Rec> g_recs;        // records since the last read
std::vector<cudaEvent_t> g_pool;  // reusable events
thread_local int t_open = -1;     // index of the open record of this thread

cudaEvent_t take() {
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

bool enabled() { return g_enabled.load(std::memory_order_relaxed); }

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void begin(cudaStream_t s, int cls) {
  if (!enabled()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Rec r{take(), take(), cls, 0.0, false};
  cudaEventRecord(r.a, s);
  g_recs.push_back(r);
  t_open = (int)g_recs.size() - 1;
}

void end(cudaStream_t s, int cls, double work) {
  if (!enabled()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (t_open < 0 || t_open >= (int)g_recs.size()) return;
  Rec &r = g_recs[t_open];
  if (r.cls != cls || r.closed) return;
  cudaEventRecord(r.b, s);
  r.work = work;
  r.closed = true;
  t_open = -1;
}

}  // namespace prof
}  // namespace ebv

using namespace ebv::prof;

extern "C" {

EBV_API int64_t ebv_debug_launch_count(void) { return g_launches.load(); }

EBV_API void ebv_debug_profile(int32_t enable) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_enabled.store(enable != 0);
}

EBV_API int32_t ebv_debug_profile_read(double *ms_by_class, double *work_by_class, int64_t *count_by_class) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (int c = 0; c < kNumClasses; ++c) {
    ms_by_class[c] = 0.0;
    work_by_class[c] = 0.0;
    count_by_class[c] = 0;
  }
  int32_t st = 0;
  for (Rec &r : g_recs) {
    if (r.closed) {
      if (cudaEventSynchronize(r.b) != cudaSuccess) st = EBV_ERR_CUDA;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess && r.cls >= 0 && r.cls < kNumClasses) {
        ms_by_class[r.cls] += ms;
        work_by_class[r.cls] += r.work;
        count_by_class[r.cls] += 1;
      }
    }
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  return st;
}

}  // extern "C"

// Launch counting and opt-in per-kernel-kind CUDA-event timing.
//
// Every launcher of the library calls count_launch(); when profiling is on, a ProfScope
// records one event before and one after the launch on the launching stream, so the
// elapsed time of each launch is measured on the device in stream order.
#include <atomic>
#include <mutex>
#include <vector>

#include "shot_internal.cuh"

namespace shot {

namespace {
struct Rec {
  int kind;
  cudaEvent_t b, e;
};
std::atomic<long long> g_launches{0};
std::atomic<int> g_on{0};
std::mutex g_mu;
std::vector<cudaEvent_t> g_pool;
std::vector<Rec> g_recs;

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

void count_launch(int n) { g_launches += n; }

bool profiling_on() { return g_on.load() != 0; }

ProfScope::ProfScope(int kind, cudaStream_t st) : kind_(kind), st_(st) {
  if (!g_on.load()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  b_ = take_event();
  e_ = take_event();
  if (b_) cudaEventRecord(b_, st_);
}

ProfScope::~ProfScope() {
  if (!b_) return;
  cudaEventRecord(e_, st_);
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back({kind_, b_, e_});
}

}  // namespace shot

extern "C" {

int shot_launch_count(long long* n) {
  if (!n) return SHOT_ERR_INVALID_ARG;
  *n = shot::g_launches.load();
  return SHOT_OK;
}

int shot_profile_enable(int on) {
  shot::g_on = on ? 1 : 0;
  return SHOT_OK;
}

int shot_profile_read(double* ms, long long* launches, int nkinds) {
  using namespace shot;
  if (nkinds < 0 || (nkinds > 0 && (!ms || !launches))) return SHOT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  for (int k = 0; k < nkinds; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (const Rec& r : g_recs) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(r.e);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.b, r.e);
    if (e != cudaSuccess) return cuda_status(e, "shot_profile_read");
    if (r.kind < nkinds) {
      ms[r.kind] += t;
      launches[r.kind] += 1;
    }
    g_pool.push_back(r.b);
    g_pool.push_back(r.e);
  }
  g_recs.clear();
  return SHOT_OK;
}

}  // extern "C"

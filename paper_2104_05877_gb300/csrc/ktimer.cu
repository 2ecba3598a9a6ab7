// Per-kernel CUDA-event timing for measurement runs: when enabled, the launch sites of the hot
// kernels record an event before and after each launch on the launching stream; totals are
// read back per kernel name.  Disabled (the default) it costs one branch per launch.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace skel {

namespace {

struct Record {
  const char* name;
  cudaEvent_t start, stop;
};

std::mutex g_mu;
bool g_enabled = false;
std::vector<Record> g_records;
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

}  // namespace

bool kernel_timing_enabled() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_enabled;
}

KernelTimer::KernelTimer(const char* name, cudaStream_t st) : name_(name), st_(st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_enabled || name == nullptr) return;     // a null name: this launch is not timed
  start_ = static_cast<void*>(take_event());
  stop_ = static_cast<void*>(take_event());
  if (start_ && stop_) cudaEventRecord(static_cast<cudaEvent_t>(start_), st_);
}

KernelTimer::~KernelTimer() {
  if (!start_ || !stop_) return;
  cudaEventRecord(static_cast<cudaEvent_t>(stop_), st_);
  std::lock_guard<std::mutex> lk(g_mu);
  g_records.push_back({name_, static_cast<cudaEvent_t>(start_), static_cast<cudaEvent_t>(stop_)});
}

}  // namespace skel

using namespace skel;

extern "C" {

skel_status skel_debug_kernel_timing(int enable) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (Record& r : g_records) {
    g_pool.push_back(r.start);
    g_pool.push_back(r.stop);
  }
  g_records.clear();
  g_enabled = enable != 0;
  return SKEL_OK;
}

skel_status skel_debug_kernel_time(const char* kernel, double* total_ms, int64_t* launches) {
  if (kernel == nullptr || total_ms == nullptr || launches == nullptr) return SKEL_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  double tot = 0.0;
  int64_t cnt = 0;
  for (const Record& r : g_records) {
    if (std::strcmp(r.name, kernel) != 0) continue;
    if (cudaEventSynchronize(r.stop) != cudaSuccess) return SKEL_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.start, r.stop) != cudaSuccess) return SKEL_ERR_CUDA;
    tot += ms;
    ++cnt;
  }
  *total_ms = tot;
  *launches = cnt;
  return SKEL_OK;
}

}  // extern "C"

// Optional kernel instrumentation: CUDA events on the launching stream.
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace q4c {
namespace {
struct Record {
  std::string name;
  cudaEvent_t e0, e1;
};
std::atomic<int> g_enabled{0};
std::mutex g_mu;
std::vector<Record> g_records;
}  // namespace

KernelScope::KernelScope(const char* name, cudaStream_t s) : name_(name), s_(s) {
  if (!g_enabled.load()) return;
  if (cudaEventCreate(&e0_) != cudaSuccess) { e0_ = nullptr; return; }
  cudaEventRecord(e0_, s_);
}

KernelScope::~KernelScope() {
  if (!e0_) return;
  cudaEvent_t e1 = nullptr;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0_); return; }
  cudaEventRecord(e1, s_);
  std::lock_guard<std::mutex> lk(g_mu);
  g_records.push_back({name_, e0_, e1});
}
}  // namespace q4c

using namespace q4c;

extern "C" q4c_status q4c_profile(int32_t enable) {
  g_enabled.store(enable ? 1 : 0);
  return Q4C_OK;
}

extern "C" q4c_status q4c_profile_read(const char* prefix, double* ms, int64_t* launches) {
  Q4C_CHECK_ARG(ms && launches, "q4c_profile_read: NULL output");
  const size_t np = prefix ? std::strlen(prefix) : 0;
  double tot = 0.0;
  int64_t n = 0;
  std::lock_guard<std::mutex> lk(g_mu);
  std::vector<Record> keep;
  for (Record& r : g_records) {
    if (np && r.name.compare(0, np, prefix) != 0) {
      keep.push_back(r);
      continue;
    }
    float t = 0.f;
    Q4C_CUDA(cudaEventSynchronize(r.e1));
    Q4C_CUDA(cudaEventElapsedTime(&t, r.e0, r.e1));
    tot += t;
    ++n;
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  g_records.swap(keep);
  *ms = tot;
  *launches = n;
  return Q4C_OK;
}

// pd_prof.cu -- tracing of libpd's own kernel launches with CUDA events
// (pd_prof_enable / pd_prof_read).
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "pd.h"
#include "pd_internal.h"

namespace pd {
namespace {

struct Rec {
  const char* name;
  cudaEvent_t a, b;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;

void clear_locked() {
  for (Rec& r : g_recs) {
    if (r.a) cudaEventDestroy(r.a);
    if (r.b) cudaEventDestroy(r.b);
  }
  g_recs.clear();
}

}  // namespace

bool prof_enabled() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_on;
}

ProfScope::ProfScope(cudaStream_t st, const char* name) : st_(st), idx_(-1) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  // (launches recorded into a graph are not traced: their events would
  // belong to the graph, not to a stream)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  Rec r{name, nullptr, nullptr};
  if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  idx_ = (int)g_recs.size() - 1;
}

ProfScope::~ProfScope() {
  if (idx_ < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (idx_ < (int)g_recs.size()) cudaEventRecord(g_recs[idx_].b, st_);
}

}  // namespace pd

extern "C" int pd_prof_enable(int on) {
  std::lock_guard<std::mutex> lk(pd::g_mu);
  if (on) pd::clear_locked();
  pd::g_on = on != 0;
  return PD_OK;
}

extern "C" int pd_prof_read(int cap, const char** names, int64_t* launches, double* total_ms) {
  std::lock_guard<std::mutex> lk(pd::g_mu);
  std::vector<const char*> nm;
  std::vector<int64_t> cnt;
  std::vector<double> ms;
  for (const pd::Rec& r : pd::g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return PD_ECUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return PD_ECUDA;
    size_t q = 0;
    while (q < nm.size() && strcmp(nm[q], r.name) != 0) ++q;
    if (q == nm.size()) {
      nm.push_back(r.name);
      cnt.push_back(0);
      ms.push_back(0.0);
    }
    cnt[q] += 1;
    ms[q] += t;
  }
  for (size_t q = 0; q < nm.size() && (int)q < cap; ++q) {
    if (names) names[q] = nm[q];
    if (launches) launches[q] = cnt[q];
    if (total_ms) total_ms[q] = ms[q];
  }
  return (int)nm.size();
}

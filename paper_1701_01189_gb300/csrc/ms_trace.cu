// ms_trace.cu -- stage timing: CUDA events around the pre-scan, scan and
// post-scan kernels of every multisplit while enabled (the per-stage timing of
// the paper's Table 4, taken on the launching stream).
#include <mutex>
#include <vector>

#include "ms.h"
#include "ms_host.h"

namespace ms {

namespace {
struct Quad {
  cudaEvent_t ev[4];
};
std::mutex g_mu;
bool g_on = false;
std::vector<Quad> g_used, g_free;
}  // namespace

int trace_begin(cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_on) return -1;
  Quad q;
  if (!g_free.empty()) {
    q = g_free.back();
    g_free.pop_back();
  } else {
    for (auto& e : q.ev)
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
  }
  g_used.push_back(q);
  const int slot = (int)g_used.size() - 1;
  cudaEventRecord(g_used[slot].ev[0], s);
  return slot;
}

void trace_mark(int slot, int stage, cudaStream_t s) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lock(g_mu);
  if (slot < (int)g_used.size()) cudaEventRecord(g_used[slot].ev[stage], s);
}

void trace_release() {
  std::lock_guard<std::mutex> lock(g_mu);
  g_on = false;
  for (auto* v : {&g_used, &g_free})
    for (auto& q : *v)
      for (auto& e : q.ev) cudaEventDestroy(e);
  g_used.clear();
  g_free.clear();
}

}  // namespace ms

using namespace ms;

extern "C" ms_status ms_stage_timing(int enable) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (enable) {
    for (auto& q : g_used) g_free.push_back(q);
    g_used.clear();
  }
  g_on = enable != 0;
  return MS_OK;
}

extern "C" ms_status ms_stage_times(double* prescan_ms, double* scan_ms, double* postscan_ms, uint64_t* launches) {
  std::lock_guard<std::mutex> lock(g_mu);
  double acc[3] = {0, 0, 0};
  for (auto& q : g_used) {
    if (cudaEventSynchronize(q.ev[3]) != cudaSuccess) return MS_ERR_CUDA;
    for (int k = 0; k < 3; ++k) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, q.ev[k], q.ev[k + 1]) != cudaSuccess) return MS_ERR_CUDA;
      acc[k] += t;
    }
  }
  if (prescan_ms) *prescan_ms = acc[0];
  if (scan_ms) *scan_ms = acc[1];
  if (postscan_ms) *postscan_ms = acc[2];
  if (launches) *launches = g_used.size();
  return MS_OK;
}

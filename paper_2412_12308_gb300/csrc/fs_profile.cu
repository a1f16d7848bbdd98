// fs_profile.cu -- optional per-launch CUDA-event timing of the library's
// kernels, and optional NVTX ranges per pass (env FS_NVTX=1) for timeline
// tools; the NVTX v3 calls are no-ops unless a tool is attached.
#include <nvtx3/nvToolsExt.h>

#include <cstdlib>
#include <mutex>
#include <vector>

#include "fs_host.h"
#include "fs_kernels.cuh"

namespace fs {

namespace {
struct Rec {
  int cls;
  cudaEvent_t a, b;
};
std::mutex g_mu;
std::vector<Rec *> g_recs;
std::atomic<bool> g_on{false};
}  // namespace

bool prof_on() { return g_on.load(std::memory_order_relaxed); }

bool nvtx_on() {
  static const bool on = [] {
    const char *v = getenv("FS_NVTX");
    return v && v[0] == '1';
  }();
  return on;
}
void nvtx_push(int cls) {
  static const char *names[PC_N] = {"fs row R2C", "fs column", "fs row C2R", "fs factor", "fs small", "fs batch"};
  nvtxRangePushA(cls >= 0 && cls < PC_N ? names[cls] : "fs");
}
void nvtx_pop() { nvtxRangePop(); }

void prof_begin(int cls, cudaStream_t s, void **tok) {
  Rec *r = new Rec{cls, nullptr, nullptr};
  if (cudaEventCreate(&r->a) != cudaSuccess || cudaEventCreate(&r->b) != cudaSuccess) {
    delete r;
    *tok = nullptr;
    return;
  }
  cudaEventRecord(r->a, s);
  *tok = r;
}

void prof_end(void *tok, cudaStream_t s) {
  Rec *r = static_cast<Rec *>(tok);
  cudaEventRecord(r->b, s);
  std::lock_guard<std::mutex> g(g_mu);
  g_recs.push_back(r);
}

static void clear_locked() {
  for (Rec *r : g_recs) {
    cudaEventDestroy(r->a);
    cudaEventDestroy(r->b);
    delete r;
  }
  g_recs.clear();
}

}  // namespace fs

using namespace fs;

extern "C" fs_status fs_profile_enable(int on) {
  std::lock_guard<std::mutex> g(g_mu);
  g_on.store(on != 0);
  if (!on) clear_locked();
  return FS_OK;
}

extern "C" int fs_profile_report(uint64_t *counts, double *total_ms, int cap) {
  std::lock_guard<std::mutex> g(g_mu);
  const int n = cap < PC_N ? cap : PC_N;
  for (int i = 0; i < n; ++i) {
    if (counts) counts[i] = 0;
    if (total_ms) total_ms[i] = 0.0;
  }
  for (Rec *r : g_recs) {
    if (cudaEventSynchronize(r->b) != cudaSuccess) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r->a, r->b) != cudaSuccess) continue;
    if (r->cls < n) {
      if (counts) counts[r->cls] += 1;
      if (total_ms) total_ms[r->cls] += ms;
    }
  }
  return n;
}

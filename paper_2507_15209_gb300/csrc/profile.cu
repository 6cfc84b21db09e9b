// Stage timers: a CUDA event pair around every kernel group when profiling is on, read back
// (after a synchronisation) as total milliseconds, kernel launches and calls per stage.
#include <mutex>
#include <unordered_map>

#include "zeta_internal.h"

namespace zk {

int ensure_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> done;
  if (bytes <= 48 * 1024) return ZETA_OK;
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find(kernel);
  if (it != done.end() && it->second >= bytes) return ZETA_OK;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes)) != cudaSuccess)
    return ZETA_ECUDA;
  done[kernel] = bytes;
  return ZETA_OK;
}
namespace {

cudaEvent_t take_event(Profiler& p) {
  if (!p.pool.empty()) {
    cudaEvent_t e = p.pool.back();
    p.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

const char* kNames[ST_COUNT] = {"assign",    "sort",      "r2c",       "alm_z",     "alm_y",     "alm_x",
                                "gram_node", "gram_gamma", "gram_particles", "mass", "reduce", "adj_points",
                                "adj_fft",   "adj_other"};

}  // namespace

StageScope::StageScope(const zeta_ctx* c, int stage, int nkernels, cudaStream_t s)
    : c_(c), stage_(stage), nk_(nkernels), s_(s) {
  Profiler& p = c_->prof;
  p.launches[stage_] += nk_;
  p.calls[stage_] += 1;
  if (!p.on || c_->capturing) return;
  a_ = take_event(p);
  if (a_) cudaEventRecord(a_, s_);
}

StageScope::~StageScope() {
  Profiler& p = c_->prof;
  if (!p.on || !a_ || c_->capturing) return;
  cudaEvent_t b = take_event(p);
  if (!b) {
    p.pool.push_back(a_);
    return;
  }
  cudaEventRecord(b, s_);
  p.pending.push_back({stage_, nk_, a_, b});
}

void profile_release(const zeta_ctx* c) {
  Profiler& p = c->prof;
  for (auto& r : p.pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : p.pool) cudaEventDestroy(e);
  p.pending.clear();
  p.pool.clear();
}

}  // namespace zk

extern "C" {

int zeta_profile_enable(zeta_ctx* c, int enable) {
  if (!c) return ZETA_EINVAL;
  zk::Profiler& p = c->prof;
  for (auto& r : p.pending) {
    cudaEventSynchronize(r.b);
    p.pool.push_back(r.a);
    p.pool.push_back(r.b);
  }
  p.pending.clear();
  for (int i = 0; i < zk::ST_COUNT; ++i) {
    p.ms[i] = 0.0;
    p.launches[i] = 0;
    p.calls[i] = 0;
  }
  p.on = enable != 0;
  return ZETA_OK;
}

int zeta_profile_read(zeta_ctx* c, double* ms, int64_t* launches, int64_t* calls, int nslots) {
  if (!c || nslots < 0) return ZETA_EINVAL;
  zk::Profiler& p = c->prof;
  for (auto& r : p.pending) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return ZETA_ECUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return ZETA_ECUDA;
    p.ms[r.stage] += t;
    p.pool.push_back(r.a);
    p.pool.push_back(r.b);
  }
  p.pending.clear();
  for (int i = 0; i < nslots && i < zk::ST_COUNT; ++i) {
    if (ms) ms[i] = p.ms[i];
    if (launches) launches[i] = p.launches[i];
    if (calls) calls[i] = p.calls[i];
  }
  return zk::ST_COUNT;
}

const char* zeta_profile_stage_name(int i) {
  if (i < 0 || i >= zk::ST_COUNT) return "";
  return zk::kNames[i];
}

}  // extern "C"

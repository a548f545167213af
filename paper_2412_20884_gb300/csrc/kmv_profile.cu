// Kernel timing: CUDA events recorded on the caller's stream around each launch
// of the main product kernels, summed on request.  Instrumentation only; the
// computation is unchanged whether it is on or off.
#include "kmv_internal.cuh"

namespace kmv {

namespace {
cudaEvent_t prof_event(kmv_handle h) {
  if (!h->prof_pool.empty()) {
    cudaEvent_t e = h->prof_pool.back();
    h->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
}  // namespace

ProfScope::ProfScope(kmv_handle h_, int kind_, cudaStream_t st_) : h(h_), kind(kind_), st(st_) {
  if (!h->prof || h->capturing || kind < 0 || kind > 1) return;
  cudaEvent_t e0 = prof_event(h);
  e1 = prof_event(h);
  if (!e0 || !e1) {
    if (e0) h->prof_pool.push_back(e0);
    if (e1) h->prof_pool.push_back(e1);
    e1 = nullptr;
    return;
  }
  cudaEventRecord(e0, st);
  h->prof_rec[kind].push_back({e0, e1});
}

ProfScope::~ProfScope() {
  if (e1) cudaEventRecord(e1, st);
}

}  // namespace kmv

using namespace kmv;

extern "C" kmv_status kmv_profile_enable(kmv_handle h, int32_t on) {
  if (!h) return KMV_EINVAL;
  h->prof = on != 0;
  for (int k = 0; k < 2; ++k) {
    for (auto& pr : h->prof_rec[k]) {
      h->prof_pool.push_back(pr.first);
      h->prof_pool.push_back(pr.second);
    }
    h->prof_rec[k].clear();
  }
  return KMV_OK;
}

extern "C" kmv_status kmv_profile_read(kmv_handle h, int32_t kind, double* total_ms, int64_t* launches) {
  if (!h || kind < 0 || kind > 1 || !total_ms || !launches) return KMV_EINVAL;
  if (cudaSetDevice(h->device) != cudaSuccess) return KMV_ECUDA;
  double tot = 0.0;
  int64_t n = 0;
  kmv_status status = KMV_OK;
  for (auto& pr : h->prof_rec[kind]) {
    float ms = 0.f;
    if (cudaEventSynchronize(pr.second) != cudaSuccess || cudaEventElapsedTime(&ms, pr.first, pr.second) != cudaSuccess) {
      cudaGetLastError();
      status = KMV_ECUDA;
    } else {
      tot += ms;
      ++n;
    }
    h->prof_pool.push_back(pr.first);
    h->prof_pool.push_back(pr.second);
  }
  h->prof_rec[kind].clear();
  *total_ms = tot;
  *launches = n;
  return status;
}

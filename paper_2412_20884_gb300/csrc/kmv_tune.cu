// Tile choices of the tensor-core kernels and the autotuner that picks them
// per call shape (kmv_set_tiles, kmv_get_tiles, kmv_autotune).
//
// The autotuner times each candidate with CUDA events around one public call
// (kmv_forward with m columns, kmv_backward with m columns and no grad_V) on a
// bounded sample of the caller's shape, and records the fastest under the
// shape key (kernel kind, d, m, size class of the largest instance).  The
// candidates vary what the kernels leave open: the exp split between the MUFU
// and the FMA-pipe polynomial, the depth of the operand ring, and how finely
// the work plan cuts the J range (work items per SM).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kmv_internal.cuh"
#include "tc_common.cuh"

namespace kmv {
namespace {

constexpr int64_t kTuneRows = 65536;

// Deterministic synthetic values in [-1, 1) (a 32-bit integer hash).
__global__ void tune_fill_kernel(float* v, int64_t n, uint32_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t x = (uint32_t)i * 2654435761u ^ seed;
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  v[i] = (float)(x >> 8) * (2.0f / 16777216.0f) - 1.0f;
}

bool tiles_valid(int kind, const kmv_tiles& t) {
  if (kind < 0 || kind >= kTilesKinds) return false;
  if (t.stages != 0 && (t.stages < 2 || t.stages > 8)) return false;
  if (t.items_per_sm < 1 || t.items_per_sm > 64) return false;
  if (t.exp_split < 0 || t.exp_split > 64) return false;
  return true;
}

TcTiles to_tc(const kmv_tiles& t) {
  TcTiles r;
  r.stages = t.stages;
  r.items_per_sm = t.items_per_sm;
  r.exp_split = t.exp_split <= 0 ? 0 : (t.exp_split <= 5 ? 4 : 8);
  return r;
}

void read_cache(TcState* S, const char* path) {
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[256];
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#') continue;
    TcTuned e{};
    if (std::sscanf(line, "%d %d %d %d %d %d %d %lf", &e.kind, &e.d, &e.m, &e.nlog2, &e.t.stages,
                    &e.t.items_per_sm, &e.t.exp_split, &e.ms) != 8)
      continue;
    kmv_tiles chk{e.t.stages, e.t.items_per_sm, e.t.exp_split};
    if (!tiles_valid(e.kind, chk)) continue;
    bool have = false;
    for (const TcTuned& o : S->tuned)
      have = have || (o.kind == e.kind && o.d == e.d && o.m == e.m && o.nlog2 == e.nlog2);
    if (!have) S->tuned.push_back(e);
  }
  std::fclose(f);
}

bool write_cache(const TcState* S, const char* path) {
  FILE* f = std::fopen(path, "w");
  if (!f) return false;
  std::fprintf(f, "# kmv tiles: kind d m nlog2 stages items_per_sm exp_split ms\n");
  for (const TcTuned& e : S->tuned)
    std::fprintf(f, "%d %d %d %d %d %d %d %.6f\n", e.kind, e.d, e.m, e.nlog2, e.t.stages, e.t.items_per_sm,
                 e.t.exp_split, e.ms);
  return std::fclose(f) == 0;
}

}  // namespace
}  // namespace kmv

using namespace kmv;

extern "C" {

kmv_status kmv_set_tiles(kmv_handle h, int32_t kernel, const kmv_tiles* t) {
  if (!h || !t) return KMV_EINVAL;
  if (!tiles_valid(kernel, *t)) {
    h->last_error = "kmv_set_tiles: unknown kernel or value out of range";
    return KMV_EINVAL;
  }
  tc_state(h)->tiles[kernel] = to_tc(*t);
  return KMV_OK;
}

kmv_status kmv_get_tiles(kmv_handle h, int32_t kernel, kmv_tiles* t) {
  if (!h || !t) return KMV_EINVAL;
  if (kernel < 0 || kernel >= kTilesKinds) {
    h->last_error = "kmv_get_tiles: unknown kernel";
    return KMV_EINVAL;
  }
  const TcTiles& c = tc_state(h)->tiles[kernel];
  t->stages = c.stages;
  t->items_per_sm = c.items_per_sm;
  t->exp_split = c.exp_split;
  return KMV_OK;
}

kmv_status kmv_autotune(kmv_handle h, const kmv_points* pts, int32_t chains, const double* theta, int32_t m,
                        const char* cache_path, void* stream) {
  if (!h) return KMV_EINVAL;
  if (!pts || !pts->offsets || !theta || m < 1 || chains < 1 || pts->n_inst < 1 || pts->d < 1) {
    h->last_error = "kmv_autotune: bad argument";
    return KMV_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    h->last_error = "kmv_autotune: the stream is being captured";
    return KMV_EINVAL;
  }
  if (cudaSetDevice(h->device) != cudaSuccess) return KMV_ECUDA;
  TcState* S = tc_state(h);
  if (cache_path) read_cache(S, cache_path);

  // the shape key, from the caller's layout
  int b_max = 0;
  int64_t n_max = 0;
  for (int b = 0; b < pts->n_inst; ++b) {
    const int64_t nb = pts->offsets[b + 1] - pts->offsets[b];
    if (nb < 0) {
      h->last_error = "kmv_autotune: offsets must be non-decreasing";
      return KMV_EINVAL;
    }
    if (nb > n_max) {
      n_max = nb;
      b_max = b;
    }
  }
  if (n_max == 0) return KMV_OK;
  int nlog2 = 0;
  while ((int64_t(1) << (nlog2 + 1)) <= n_max) ++nlog2;
  const int d = pts->d;
  const int k = pts->ard ? d : 1;
  int n_coef = 0;
  if (pts->cheb > 0) {
    n_coef = cheb_n_coef(pts->cheb, d);
    if (n_coef < 0) {
      h->last_error = "kmv_autotune: Chebyshev order out of range";
      return KMV_EINVAL;
    }
  }
  const int n_theta = pts->cheb > 0 ? n_coef + k + 1 : k + 2;
  const int fwd_kind = m <= 2 ? kTilesForwardFma : kTilesForward;

  // the timing sample: the first rows of the largest instance, one chain
  const int64_t n_sub = std::min(n_max, kTuneRows);
  const int64_t off_sub[2] = {0, n_sub};
  kmv_points sub = *pts;
  sub.n_inst = 1;
  sub.offsets = off_sub;
  sub.x = pts->x + pts->offsets[b_max] * d;
  const double* th_sub = theta + (int64_t)b_max * chains * n_theta;

  float *V = nullptr, *G = nullptr, *Y = nullptr;
  double* gth = nullptr;
  const size_t vb = sizeof(float) * (size_t)n_sub * m;
  if (cudaMalloc(&V, vb) != cudaSuccess || cudaMalloc(&G, vb) != cudaSuccess || cudaMalloc(&Y, vb) != cudaSuccess ||
      cudaMalloc(&gth, sizeof(double) * n_theta) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(V);
    cudaFree(G);
    cudaFree(Y);
    cudaFree(gth);
    h->last_error = "kmv_autotune: scratch allocation failed";
    return KMV_ENOMEM;
  }
  const int64_t nv = (int64_t)n_sub * m;
  tune_fill_kernel<<<(unsigned)((nv + 255) / 256), 256, 0, st>>>(V, nv, 0x9e3779b9u);
  tune_fill_kernel<<<(unsigned)((nv + 255) / 256), 256, 0, st>>>(G, nv, 0x85ebca6bu);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);

  // candidates are timed with the tuned table set aside, so the defaults apply
  std::vector<TcTuned> saved;
  saved.swap(S->tuned);
  const TcTiles defaults[kTilesKinds] = {S->tiles[0], S->tiles[1], S->tiles[2]};
  kmv_status status = KMV_OK;
  std::vector<TcTuned> found;

  auto time_call = [&](int kind, float* best_ms) -> kmv_status {
    auto run = [&]() -> kmv_status {
      if (kind == kTilesAdjoint) return kmv_backward(h, &sub, 1, th_sub, V, G, m, gth, nullptr, KMV_BF16_HILO, st);
      return kmv_forward(h, &sub, 1, th_sub, V, m, nullptr, Y, nullptr, KMV_BF16_HILO, st);
    };
    kmv_status s = run();  // warm-up (and plan / workspace set-up)
    if (s != KMV_OK) return s;
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, st);
      s = run();
      cudaEventRecord(e1, st);
      if (s != KMV_OK) return s;
      if (cudaEventSynchronize(e1) != cudaSuccess) return KMV_ECUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, ms);
    }
    *best_ms = best;
    return KMV_OK;
  };

  for (int kind : {fwd_kind, (int)kTilesAdjoint}) {
    bool have = false;
    for (const TcTuned& e : saved) have = have || (e.kind == kind && e.d == d && e.m == m && e.nlog2 == nlog2);
    if (have) continue;
    std::vector<TcTiles> cand;
    for (int split : (kind == kTilesAdjoint ? std::vector<int>{0} : std::vector<int>{0, 8, 4}))
      for (int stages : {0, 4})
        for (int ipsm : {3, 6, 12}) {
          TcTiles t;
          t.stages = stages;
          t.items_per_sm = ipsm;
          t.exp_split = split;
          cand.push_back(t);
        }
    TcTuned best{kind, d, m, nlog2, defaults[kind], 1e30};
    for (const TcTiles& t : cand) {
      S->tiles[kind] = t;
      float ms = 0.f;
      const kmv_status s = time_call(kind, &ms);
      if (s == KMV_EUNSUPPORTED) break;
      if (s != KMV_OK) {
        status = s;
        break;
      }
      if (ms < best.ms) {
        best.t = t;
        best.ms = ms;
      }
    }
    S->tiles[kind] = defaults[kind];
    if (status != KMV_OK) break;
    if (best.ms < 1e29) found.push_back(best);
  }
  for (int q = 0; q < kTilesKinds; ++q) S->tiles[q] = defaults[q];
  saved.insert(saved.end(), found.begin(), found.end());
  S->tuned.swap(saved);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(V);
  cudaFree(G);
  cudaFree(Y);
  cudaFree(gth);
  if (status != KMV_OK) return status;
  if (cache_path && !write_cache(S, cache_path)) {
    h->last_error = "kmv_autotune: could not write the cache file";
    return KMV_EINVAL;
  }
  return KMV_OK;
}

}  // extern "C"

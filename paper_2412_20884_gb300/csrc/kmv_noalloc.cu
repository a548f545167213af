// kmv_backward_noalloc: the FP32 adjoint with its scratch in a fixed device
// array, for callers that cannot allocate device memory.
//
// Who needs this: code that hands all of the device memory to its own pool
// or arena (a framework's caching allocator, a fixed budget per process) and
// must not take memory behind the pool's back, and latency-critical loops that
// cannot afford the device-wide synchronisation that cudaMalloc and cudaFree
// can imply.  It needs no handle either: kmv_create allocates, this entry
// point does not.
//
// Scratch: the static array below, kNoAllocScratchBytes (4 MiB) per device
// that loads the library, held until the process exits.  Host code may not
// pass the array's name to a kernel (in host code it is only a stand-in for
// the symbol); the device address comes from cudaGetSymbolAddress, looked up
// once per device, with that device current, on the first call there.
#include <atomic>
#include <cstring>

#include "kmv_internal.cuh"
#include "simt_common.cuh"

namespace kmv {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// device address of the array per device, looked up on the first call there
// (two threads making that first call at once both store the same address)
std::atomic<unsigned char*> g_scratch_addr[kMaxDevices];

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Fills inst_item0 / item_inst / item_row0 from the offsets already copied
// into the scratch.  One block: thread 0 forms the prefix over instances
// once, then the block fills the items of every instance.
__global__ void noalloc_items_kernel(int n_inst, const int64_t* offsets, int32_t* inst_item0,
                                     int32_t* item_inst, int64_t* item_row0) {
  if (threadIdx.x == 0) {
    int32_t acc = 0;
    for (int b = 0; b < n_inst; ++b) {
      inst_item0[b] = acc;
      acc += (int32_t)((offsets[b + 1] - offsets[b] + kTile - 1) / kTile);
    }
    inst_item0[n_inst] = acc;
  }
  __syncthreads();
  for (int b = 0; b < n_inst; ++b) {
    const int32_t first = inst_item0[b], tiles = inst_item0[b + 1] - first;
    for (int32_t t = threadIdx.x; t < tiles; t += blockDim.x) {
      item_inst[first + t] = b;
      item_row0[first + t] = offsets[b] + (int64_t)t * kTile;
    }
  }
}

}  // namespace
}  // namespace kmv

using namespace kmv;

extern "C" kmv_status kmv_backward_noalloc(const kmv_points* pts, int32_t chains, const double* theta,
                                           const float* V, const float* G, int32_t m, double* grad_theta,
                                           float* grad_V, void* stream) {
  // the same rules as every entry point with a handle (points_error), then this one's own
  if (points_error(pts, chains) != nullptr || m < 1 || !theta || !V || !G || !grad_theta) return KMV_EINVAL;
  if (pts->cheb != 0) return KMV_EUNSUPPORTED;   // the amplitudes would need scratch per point
  int64_t n_items = 0;
  for (int b = 0; b < pts->n_inst; ++b) n_items += (pts->offsets[b + 1] - pts->offsets[b] + kTile - 1) / kTile;
  const int64_t n_total = pts->offsets[pts->n_inst];
  const int n_theta = 2 + (pts->ard ? pts->d : 1);
  const int mp = backward_mp(m);
  const int n_z = (m + mp - 1) / mp;

  // scratch layout; a call that does not fit is rejected before any work
  const size_t o_off = 0;
  const size_t o_ii = o_off + align256(sizeof(int64_t) * (pts->n_inst + 1));
  const size_t o_inst = o_ii + align256(sizeof(int32_t) * (pts->n_inst + 1));
  const size_t o_row0 = o_inst + align256(sizeof(int32_t) * (size_t)(n_items > 0 ? n_items : 1));
  const size_t o_part = o_row0 + align256(sizeof(int64_t) * (size_t)(n_items > 0 ? n_items : 1));
  const double part_bytes = (double)sizeof(double) * (double)(n_items > 0 ? n_items : 1) * chains * n_z * n_theta;
  if ((double)o_part + part_bytes > (double)kNoAllocScratchBytes) return KMV_EINVAL;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return KMV_ECUDA;
  unsigned char* base = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!base) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return KMV_ECUDA;
    }
    base = static_cast<unsigned char*>(p);
    g_scratch_addr[dev].store(base, std::memory_order_release);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  if (cudaMemcpyAsync(base + o_off, pts->offsets, sizeof(int64_t) * (pts->n_inst + 1), cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return KMV_ECUDA;
  DevLayout L;
  L.offsets = reinterpret_cast<const int64_t*>(base + o_off);
  L.inst_item0 = reinterpret_cast<const int32_t*>(base + o_ii);
  L.item_inst = reinterpret_cast<const int32_t*>(base + o_inst);
  L.item_row0 = reinterpret_cast<const int64_t*>(base + o_row0);
  noalloc_items_kernel<<<1, 256, 0, st>>>(
      pts->n_inst, L.offsets, reinterpret_cast<int32_t*>(base + o_ii), reinterpret_cast<int32_t*>(base + o_inst),
      reinterpret_cast<int64_t*>(base + o_row0));

  KmvArgs a{};
  a.L = L;
  a.chains = chains;
  a.d = pts->d;
  a.ard = pts->ard;
  a.n_theta = n_theta;
  a.n_total = n_total;
  a.x = pts->x;
  a.theta = theta;
  a.V = V;
  a.G = G;
  a.m = m;
  a.Y = grad_V;
  a.n_z = n_z;
  a.grad_partial = reinterpret_cast<double*>(base + o_part);
  if (n_items > 0 && launch_backward_simt(a, (int)n_items, st) != cudaSuccess) return KMV_ECUDA;
  if (launch_grad_finalize(L, pts->n_inst, chains, n_theta, pts->ard, pts->d, n_z, theta, a.grad_partial,
                           grad_theta, st) != cudaSuccess)
    return KMV_ECUDA;
  return cudaGetLastError() == cudaSuccess ? KMV_OK : KMV_ECUDA;
}

// tcgen05.mma issue rate (M=128, K=16, kind::f16) from 1, 2 or 4 issuing warps into separate accumulators,
// with B from shared memory and A from shared memory ("ss") or from tensor memory ("ts").
// Build and run (from this folder): nvcc -std=c++17 -O3 -gencode arch=compute_103a,code=sm_103a -o mma_issue_rate mma_issue_rate.cu && ./mma_issue_rate
#include <cstdio>
#include <cuda_runtime.h>
#include <stdint.h>
#include "../csrc/tc_ptx.cuh"
using namespace kmv::ptx;

// Each issuing warp w owns TMEM columns [w * stride, (w + 1) * stride): the accumulator
// (N columns) and, for "ts", the A tile (8 columns of packed 16-bit values) after it.
template <int N, bool TS>
__global__ void __launch_bounds__(128, 1) probe(int nwarps, int stride, int reps, long long* out, int* err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* bar = (uint64_t*)(sm + 65536);
  uint32_t* slot = (uint32_t*)(bar + 4);
  volatile int* abort = (volatile int*)(slot + 1);
  for (int i = threadIdx.x; i < 65536 / 4; i += blockDim.x) ((uint32_t*)sm)[i] = 0;
  if (threadIdx.x == 0) { for (int i = 0; i < 4; ++i) mbar_init(&bar[i], 1); *abort = 0; fence_barrier_init(); }
  if (threadIdx.x < 32) { tmem_alloc(slot, 512); tmem_relinquish(); }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before(); __syncthreads(); tc_fence_after();
  uint32_t tb = *slot;
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0 && w < nwarps) {
    const uint64_t da = sdesc(smem_u32(sm), 128, 512);
    const uint64_t db = sdesc(smem_u32(sm + 32768), 128, 512);
    const uint32_t idb = idesc_f16(128, N, 1, 1);
    const uint32_t d = tb + stride * w;
    const uint32_t at = d + N;
    long long t0 = clock64();
    for (int r = 0; r < reps; r += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (TS)
          mma_ts(d, at, db, idb, 1);
        else
          mma_ss(d, da, db, idb, 1);
      }
    }
    long long t1 = clock64();
    tc_commit(&bar[w]);
    bool ok = mbar_wait(&bar[w], 0, abort, err, 1);
    long long t2 = clock64();
    if (blockIdx.x == 0 && w == 0) { out[0] = t1 - t0; out[1] = t2 - t0; out[2] = ok; }
  }
  tc_fence_before(); __syncthreads(); tc_fence_after();
  if (threadIdx.x < 32) tmem_dealloc(tb, 512);
}

template <int N, bool TS>
void run(long long* out, int* err, int reps) {
  cudaFuncSetAttribute(probe<N, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 140 * 1024);
  const int need = N + (TS ? 8 : 0);
  const int stride = need <= 128 ? 128 : 256;
  for (int nw : {1, 2, 4}) {
    if (nw * stride > 512) continue;
    long long h[3];
    probe<N, TS><<<152, 128, 140 * 1024>>>(nw, stride, reps, out, err);
    cudaMemcpy(h, out, sizeof(h), cudaMemcpyDeviceToHost);
    printf("%s N=%-3d warps=%d: issue %6.1f clk/instr/warp, complete %6.1f, aggregate %6.1f clk/instr (ok=%lld)\n",
           TS ? "ts" : "ss", N, nw, (double)h[0] / reps, (double)h[1] / reps, (double)h[1] / reps / nw, h[2]);
  }
}

int main() {
  long long* out; int* err; cudaMalloc(&out, 64); cudaMalloc(&err, 4); cudaMemset(err, 0, 4);
  const int reps = 512;
  run<16, false>(out, err, reps);
  run<32, false>(out, err, reps);
  run<64, false>(out, err, reps);
  run<128, false>(out, err, reps);
  run<256, false>(out, err, reps);
  run<16, true>(out, err, reps);
  run<64, true>(out, err, reps);
  run<112, true>(out, err, reps);
  int e; cudaMemcpy(&e, err, 4, cudaMemcpyDeviceToHost);
  cudaError_t ce = cudaDeviceSynchronize();
  printf("err=%d cuda=%s\n", e, cudaGetErrorString(ce));
  return ce == cudaSuccess ? 0 : 1;
}

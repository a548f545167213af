// tcgen05.ld round trip (load + wait::ld) and throughput from 4 or 8 warps (one or two
// warpgroups), for 16-, 32- and 128-column loads per wait.
// Build and run (from this folder): nvcc -std=c++17 -O3 -gencode arch=compute_103a,code=sm_103a -o tmem_ld_rate tmem_ld_rate.cu && ./tmem_ld_rate
#include <cstdio>
#include <cuda_runtime.h>
#include <stdint.h>
#include "../csrc/tc_ptx.cuh"
using namespace kmv::ptx;

// CHUNKS loads of 32 (or 16 when HALF) columns, then one wait, REPS times.
template <int CHUNKS, bool HALF>
__global__ void __launch_bounds__(256, 1) probe(int nwarps, int reps, long long* out, float* sink) {
  __shared__ uint32_t slot;
  const int warp = threadIdx.x >> 5;
  if (warp == 0) { tmem_alloc(&slot, 512); tmem_relinquish(); }
  tc_fence_before(); __syncthreads(); tc_fence_after();
  const uint32_t tb = slot;
  // warpgroup g reads columns [256 g, 256 g + 128) of its lane quarter
  const uint32_t tl = tb + 256 * (warp >> 2) + ((uint32_t)(32 * (warp & 3)) << 16);
  float acc = 0.f;
  long long t0 = clock64();
  if (warp < nwarps) {
    for (int r = 0; r < reps; ++r) {
      uint32_t v[CHUNKS][32];
#pragma unroll
      for (int c = 0; c < CHUNKS; ++c) {
        if (HALF) {
          uint32_t (&h)[16] = *reinterpret_cast<uint32_t (*)[16]>(&v[c][0]);
          tmem_ld16(tl + 16 * c, h);
        } else {
          tmem_ld32(tl + 32 * c, v[c]);
        }
      }
      tmem_ld_wait();
#pragma unroll
      for (int c = 0; c < CHUNKS; ++c) acc += __uint_as_float(v[c][0]) + __uint_as_float(v[c][HALF ? 15 : 31]);
    }
  }
  long long t1 = clock64();
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = t1 - t0;
  if (acc == 123.f) sink[threadIdx.x] = acc;
  tc_fence_before(); __syncthreads(); tc_fence_after();
  if (warp == 0) tmem_dealloc(tb, 512);
}

template <int CHUNKS, bool HALF>
void run(long long* out, float* sink) {
  const int reps = 1024;
  for (int nw : {4, 8}) {
    long long h = 0;
    probe<CHUNKS, HALF><<<152, 256>>>(nw, reps, out, sink);
    cudaMemcpy(&h, out, sizeof(h), cudaMemcpyDeviceToHost);
    const int cols = CHUNKS * (HALF ? 16 : 32);
    printf("%d x ld.x%d (%3d columns) per wait, %d warps: %7.1f clk per round, %6.1f B/clk/SM\n", CHUNKS,
           HALF ? 16 : 32, cols, nw, (double)h / reps, (double)cols * 128 * nw / ((double)h / reps));
  }
}

int main() {
  long long* out; float* sink;
  cudaMalloc(&out, 64); cudaMalloc(&sink, 256 * 4);
  run<1, true>(out, sink);
  run<1, false>(out, sink);
  run<2, false>(out, sink);
  run<4, false>(out, sink);
  cudaError_t ce = cudaDeviceSynchronize();
  printf("cuda=%s\n", cudaGetErrorString(ce));
  return ce == cudaSuccess ? 0 : 1;
}

// Which part of the exp step limits it: 8 warps per SM, each iteration one 64-column half per
// thread.  MODE 0: TMEM loads (2 x ld.x32 + waits) and a sum; 1: loads and ex2; 2: ex2 of values
// made from the loop counter and TMEM stores of the packed results; 3: ex2 of such values only;
// 4: loads, ex2 and stores (the full step, bf16 packing by byte permute).
// Build and run (from this folder): nvcc -std=c++17 -O3 -gencode arch=compute_103a,code=sm_103a -o exp_tmem_parts exp_tmem_parts.cu && ./exp_tmem_parts
#include <cstdio>
#include <cuda_runtime.h>
#include <stdint.h>
#include "../csrc/tc_ptx.cuh"
using namespace kmv::ptx;

template <int MODE>
__global__ void __launch_bounds__(256, 1) probe(int reps, long long* out, uint32_t* sink) {
  __shared__ uint32_t slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) { tmem_alloc(&slot, 512); tmem_relinquish(); }
  tc_fence_before(); __syncthreads(); tc_fence_after();
  const uint32_t tb = slot;
  const uint32_t tl = tb + ((uint32_t)(32 * (warp & 3)) << 16) + 128 * (warp >> 2);
  {
    uint32_t v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __float_as_uint(-0.01f * (i + lane));
    tmem_st32(tl, v);
    tmem_st32(tl + 32, v);
    tmem_st_wait();
  }
  uint32_t acc = 0;
  float facc = 0.f;
  __syncthreads();
  const long long t0 = clock64();
  for (int r = 0; r < reps; ++r) {
    uint32_t s0[32], s1[32], qq[16];
    if (MODE == 0 || MODE == 1 || MODE == 4) {
      tmem_ld32(tl, s0);
      tmem_ld_wait_regs(s0);
      tmem_ld32(tl + 32, s1);
      tmem_ld_wait_regs(s1);
    } else {
      const float base = -0.001f * (float)(r + lane);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        s0[i] = __float_as_uint(base - 0.01f * i);
        s1[i] = __float_as_uint(base - 0.02f * i);
      }
    }
    if (MODE == 0) {
#pragma unroll
      for (int i = 0; i < 32; ++i) acc += s0[i] ^ s1[i];
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q)
        qq[q] = __byte_perm(__float_as_uint(ex2(__uint_as_float(s0[2 * q]))),
                            __float_as_uint(ex2(__uint_as_float(s0[2 * q + 1]))), 0x7632);
      if (MODE == 2 || MODE == 4) tmem_st16(tl + 64, qq);
      else
#pragma unroll
        for (int q = 0; q < 16; ++q) acc += qq[q];
#pragma unroll
      for (int q = 0; q < 16; ++q)
        qq[q] = __byte_perm(__float_as_uint(ex2(__uint_as_float(s1[2 * q]))),
                            __float_as_uint(ex2(__uint_as_float(s1[2 * q + 1]))), 0x7632);
      if (MODE == 2 || MODE == 4) {
        tmem_st16(tl + 80, qq);
        tmem_st_wait();
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) acc += qq[q];
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  if (acc == 0x1234567u || facc == 1.f) sink[threadIdx.x] = acc;
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = t1 - t0;
  tc_fence_before(); __syncthreads(); tc_fence_after();
  if (warp == 0) tmem_dealloc(tb, 512);
}

template <int MODE>
void run(const char* name, long long* out, uint32_t* sink) {
  const int reps = 2048;
  long long h = 0;
  probe<MODE><<<152, 256>>>(reps, out, sink);
  cudaMemcpy(&h, out, sizeof(h), cudaMemcpyDeviceToHost);
  const double per = (double)h / reps;
  printf("%-16s: %7.1f clk per half per warp, %6.2f elements/clk/SM\n", name, per, 64.0 * 256 / per);
}

int main() {
  long long* out; uint32_t* sink;
  cudaMalloc(&out, 64); cudaMalloc(&sink, 256 * 4);
  run<0>("ld", out, sink);
  run<1>("ld + ex2", out, sink);
  run<2>("ex2 + st", out, sink);
  run<3>("ex2", out, sink);
  run<4>("ld + ex2 + st", out, sink);
  cudaError_t ce = cudaDeviceSynchronize();
  printf("cuda=%s\n", cudaGetErrorString(ce));
  return ce == cudaSuccess ? 0 : 1;
}

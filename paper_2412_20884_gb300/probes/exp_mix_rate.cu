// Throughput of the per-element instruction mixes of the exp warpgroups, 8 or 16 warps per SM:
//   ex2            : MUFU ex2 alone
//   ex2 mul f16    : ex2, multiply, pack pairs to f16x2 (the adjoint's Q = W 2^S)
//   ex2 f16        : ex2, pack pairs to f16x2 (the forward's P)
//   mul f16        : multiply, pack pairs to f16x2 (no exp)
//   ex2 mul bf16t  : ex2, multiply, pack pairs to bf16x2 by keeping the high halves (byte permute)
// Times are the block span (between two block barriers) in SM clocks.
// Build and run (from this folder): nvcc -std=c++17 -O3 -gencode arch=compute_103a,code=sm_103a -o exp_mix_rate exp_mix_rate.cu && ./exp_mix_rate
#include <cstdio>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

__device__ __forceinline__ float ex2f(float v) {
  float r;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ uint32_t pack_f16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ uint32_t pack_bf16_trunc(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

template <int MODE>
__global__ void __launch_bounds__(512, 1) probe(int reps, uint32_t* sink, long long* out) {
  float s[32], w[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    s[q] = -0.001f * (threadIdx.x + q);
    w[q] = 1.0f + 0.001f * q;
  }
  uint32_t acc = 0;
  __syncthreads();
  const long long t0 = clock64();
  for (int r = 0; r < reps; ++r) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float a = s[2 * q] + (float)r * 1e-9f, b = s[2 * q + 1] - (float)r * 1e-9f;
      uint32_t v;
      if (MODE == 0) {
        v = __float_as_uint(ex2f(a)) ^ __float_as_uint(ex2f(b));
      } else if (MODE == 1) {
        v = pack_f16(ex2f(a) * w[2 * q], ex2f(b) * w[2 * q + 1]);
      } else if (MODE == 2) {
        v = pack_f16(ex2f(a), ex2f(b));
      } else if (MODE == 3) {
        v = pack_f16(a * w[2 * q], b * w[2 * q + 1]);
      } else {
        v = pack_bf16_trunc(ex2f(a) * w[2 * q], ex2f(b) * w[2 * q + 1]);
      }
      acc += v;
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  if (acc == 0x12345678u) sink[threadIdx.x] = acc;
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = t1 - t0;
}

template <int MODE>
void run(const char* name, uint32_t* sink, long long* out) {
  const int reps = 4096;
  for (int threads : {256, 512}) {
    long long h = 0;
    probe<MODE><<<152, threads>>>(reps, sink, out);
    cudaMemcpy(&h, out, sizeof(h), cudaMemcpyDeviceToHost);
    const double elems = (double)reps * 32 * threads;   // elements per SM
    printf("%-14s %2d warps/SM: %6.2f elements/clk/SM\n", name, threads / 32, elems / (double)h);
  }
}

int main() {
  uint32_t* sink; long long* out;
  cudaMalloc(&sink, 512 * 4); cudaMalloc(&out, 64);
  run<0>("ex2", sink, out);
  run<1>("ex2 mul f16", sink, out);
  run<2>("ex2 f16", sink, out);
  run<3>("mul f16", sink, out);
  run<4>("ex2 mul bf16t", sink, out);
  cudaError_t ce = cudaDeviceSynchronize();
  printf("cuda=%s\n", cudaGetErrorString(ce));
  return ce == cudaSuccess ? 0 : 1;
}

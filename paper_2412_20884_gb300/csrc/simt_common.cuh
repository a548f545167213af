// Device helpers shared by the plain-FP32 (SIMT) kernels.
#pragma once

#include "kmv_internal.cuh"

namespace kmv {

// Rows of X / V / G staged in shared memory per step of the column loop.
constexpr int kJT = 64;

__device__ __forceinline__ float ex2_approx(float v) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

// sc[k] = sqrt(h) / l_k for the system's lengthscales (h = log2(e)/2), so that
// K0_ij = 2^(-sum_k (sc_k x_ik - sc_k x_jk)^2) = exp(-sum_k (x_ik - x_jk)^2 / (2 l_k^2)).
__device__ __forceinline__ void load_scale(const double* th, int d, int ard, float* sc) {
  for (int k = threadIdx.x; k < d; k += blockDim.x)
    sc[k] = (float)(sqrt(kHalfLog2e) * exp(-th[1 + (ard ? k : 0)]));
}

// Deterministic block sum of one double per thread; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

inline int pow2ceil(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

}  // namespace kmv

// The exp step in isolation, with 8 or 16 exp warps per SM (2 or 4 per scheduler).  Per
// 64-column half each thread loads its row's 64 S values (and, for the adjoint form, 64 W
// values) from TMEM, forms P = 2^S (forward) or Q = W 2^S (adjoint) packed to 16 bits, and
// stores the 32 packed words back to TMEM.  The loads go in two 32-column chunks, the second in
// flight while the first is used.  Packing: PK 0 = cvt.rn.f16x2.f32; PK 1 = f16 bits by integer
// arithmetic on the f32 bits of x 2^-112 (round half up; the 2^-112 is folded into the
// exponent or the W scale); PK 2 = as 1 with the non-flushing ex2; PK 3 = bf16 by keeping the
// high halves (byte permute, truncation).
// Build and run (from this folder): nvcc -std=c++17 -O3 -gencode arch=compute_103a,code=sm_103a -o exp_tmem_loop exp_tmem_loop.cu && ./exp_tmem_loop
#include <cstdio>
#include <cuda_runtime.h>
#include <stdint.h>
#include "../csrc/tc_ptx.cuh"
using namespace kmv::ptx;

// Warp w works on TMEM lanes 32 (w % 4) .. +31 and column block (w / 4): S at 128 cb, W at
// 128 cb + 64, and writes its packed result over its S columns.
__device__ __forceinline__ float ex2_noftz(float v) {
  float r;
  asm("ex2.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
// two non-negative floats already scaled by 2^-112 -> f16x2 (lo in the low half)
__device__ __forceinline__ uint32_t pack_int_f16x2(float lo, float hi) {
  const uint32_t a = (__float_as_uint(lo) + 0x1000u) >> 13;
  const uint32_t b = __float_as_uint(hi) * 8u + 0x8000u;
  return (b & 0xffff0000u) | a;
}
template <int PK>
__device__ __forceinline__ float e2(float v) {
  return PK == 2 ? ex2_noftz(v - 112.f) : PK == 1 ? ex2(v - 112.f) : ex2(v);
}
template <int PK>
__device__ __forceinline__ uint32_t pk2(float lo, float hi) {
  if (PK == 0) return pack_f16x2(lo, hi);
  if (PK == 3) return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
  return pack_int_f16x2(lo, hi);
}

template <bool ADJ, int NT, int PK>
__global__ void __launch_bounds__(NT, 1) probe(int reps, long long* out) {
  __shared__ uint32_t slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) { tmem_alloc(&slot, 512); tmem_relinquish(); }
  tc_fence_before(); __syncthreads(); tc_fence_after();
  const uint32_t tb = slot;
  const int cb = warp >> 2;
  const uint32_t tl = tb + ((uint32_t)(32 * (warp & 3)) << 16) + 128 * cb;
  {
    uint32_t v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __float_as_uint(-0.01f * (i + lane));
    tmem_st32(tl, v);
    tmem_st32(tl + 32, v);
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __float_as_uint(1.0f + 0.01f * i);
    tmem_st32(tl + 64, v);
    tmem_st32(tl + 96, v);
    tmem_st_wait();
  }
  __syncthreads();
  const long long t0 = clock64();
  for (int r = 0; r < reps; ++r) {
    uint32_t s0[32], w0[32], s1[32], w1[32], qq[16];
    tmem_ld32(tl, s0);
    if (ADJ) tmem_ld32(tl + 64, w0);
    if (ADJ) tmem_ld_wait_regs(s0, w0); else tmem_ld_wait_regs(s0);
    tmem_ld32(tl + 32, s1);
    if (ADJ) tmem_ld32(tl + 96, w1);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float p0 = e2<PK>(__uint_as_float(s0[2 * q])), p1 = e2<PK>(__uint_as_float(s0[2 * q + 1]));
      qq[q] = ADJ ? pk2<PK>(p0 * __uint_as_float(w0[2 * q]), p1 * __uint_as_float(w0[2 * q + 1])) : pk2<PK>(p0, p1);
    }
    if (ADJ) tmem_ld_wait_regs(s1, w1); else tmem_ld_wait_regs(s1);
    tmem_st16(tl, qq);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float p0 = e2<PK>(__uint_as_float(s1[2 * q])), p1 = e2<PK>(__uint_as_float(s1[2 * q + 1]));
      qq[q] = ADJ ? pk2<PK>(p0 * __uint_as_float(w1[2 * q]), p1 * __uint_as_float(w1[2 * q + 1])) : pk2<PK>(p0, p1);
    }
    tmem_st16(tl + 16, qq);
    tmem_st_wait();
  }
  __syncthreads();
  const long long t1 = clock64();
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = t1 - t0;
  tc_fence_before(); __syncthreads(); tc_fence_after();
  if (warp == 0) tmem_dealloc(tb, 512);
}

template <bool ADJ, int NT, int PK>
void run(long long* out) {
  const int reps = 2048;
  long long h = 0;
  probe<ADJ, NT, PK><<<152, NT>>>(reps, out);
  cudaMemcpy(&h, out, sizeof(h), cudaMemcpyDeviceToHost);
  const double per = (double)h / reps;
  const char* pk[4] = {"cvt f16x2", "int f16", "int f16 noftz", "bf16 trunc"};
  printf("%-8s %-14s %2d warps/SM: %7.1f clk per half per warp, %6.2f elements/clk/SM\n",
         ADJ ? "adjoint" : "forward", pk[PK], NT / 32, per, 64.0 * NT / per);
}

int main() {
  long long* out;
  cudaMalloc(&out, 64);
  run<false, 256, 0>(out);
  run<false, 256, 1>(out);
  run<false, 256, 2>(out);
  run<false, 256, 3>(out);
  run<false, 512, 1>(out);
  run<true, 256, 0>(out);
  run<true, 256, 1>(out);
  run<true, 256, 3>(out);
  run<true, 512, 1>(out);
  cudaError_t ce = cudaDeviceSynchronize();
  printf("cuda=%s\n", cudaGetErrorString(ce));
  return ce == cudaSuccess ? 0 : 1;
}

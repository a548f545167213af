// Issue-rate microbenchmark behind the roofline: MUFU ex2.approx.ftz.f32 vs FP32 FFMA per SM per clock.
// Build and run: nvcc -O3 -gencode arch=compute_103a,code=sm_103a -o ex2_ffma_rate ex2_ffma_rate.cu && ./ex2_ffma_rate
#include <cstdio>
#include <cuda_runtime.h>
__device__ __forceinline__ float ex2(float v){float r;asm volatile("ex2.approx.ftz.f32 %0, %1;":"=f"(r):"f"(v));return r;}
__global__ void k_ex2(float* out, int iters, float seed){
  float a[8];
  #pragma unroll
  for(int i=0;i<8;++i) a[i]=seed*(threadIdx.x+i)*1e-6f-1.0f;
  for(int it=0;it<iters;++it){
    #pragma unroll
    for(int i=0;i<8;++i) a[i]=ex2(a[i])-1.5f;   // ex2 + FADD per element
  }
  float s=0; for(int i=0;i<8;++i) s+=a[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
__global__ void k_ffma(float* out, int iters, float seed){
  float a[8];
  #pragma unroll
  for(int i=0;i<8;++i) a[i]=seed*(threadIdx.x+i);
  for(int it=0;it<iters;++it){
    #pragma unroll
    for(int i=0;i<8;++i) a[i]=fmaf(a[i],0.999f,0.001f);
  }
  float s=0; for(int i=0;i<8;++i) s+=a[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
int main(){
  int sms=0; cudaDeviceGetAttribute(&sms,cudaDevAttrMultiProcessorCount,0);
  int clk=0; cudaDeviceGetAttribute(&clk,cudaDevAttrClockRate,0);
  const int blocks=sms*8, threads=256, iters=4096;
  float* out; cudaMalloc(&out,sizeof(float)*blocks*threads);
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  for(int rep=0;rep<2;++rep){
    float ms_ex=0, ms_fm=0;
    k_ex2<<<blocks,threads>>>(out,iters,1.f); k_ffma<<<blocks,threads>>>(out,iters,1.f);
    cudaEventRecord(e0); k_ex2<<<blocks,threads>>>(out,iters,1.f); cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms_ex,e0,e1);
    cudaEventRecord(e0); k_ffma<<<blocks,threads>>>(out,iters,1.f); cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms_fm,e0,e1);
    double n=(double)blocks*threads*iters*8;
    printf("sms=%d attr_clock_khz=%d  ex2: %.3f ms %.3f Tex2/s   ffma: %.3f ms %.3f Tffma/s  => ex2/clk/SM = %.1f (if FFMA=128/clk/SM)\n",
      sms, clk, ms_ex, n/ms_ex/1e9, ms_fm, n/ms_fm/1e9, 128.0*(n/ms_ex)/(n/ms_fm));
  }
  cudaError_t e=cudaGetLastError(); printf("status %s\n", cudaGetErrorString(e));
  return e==cudaSuccess?0:1;
}

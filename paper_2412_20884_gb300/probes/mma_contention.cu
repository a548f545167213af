// Issue time of a chain of tcgen05.mma (M=128, N=64, K=16, A and B from shared memory or A from
// tensor memory) followed by tcgen05.commit, from one issuing warp, while 8 other warps are idle,
// stream tcgen05.ld from other TMEM columns, or run MUFU ex2.  The issue loop runs either in
// lane 0 alone or in the whole warp with one elected lane issuing (WIDE), with the chain length
// a run-time value (LEN = 0) or a compile-time one.
// Build and run (from this folder): nvcc -std=c++17 -O3 -gencode arch=compute_103a,code=sm_103a -o mma_contention mma_contention.cu && ./mma_contention
#include <cstdio>
#include <cuda_runtime.h>
#include <stdint.h>
#include "../csrc/tc_ptx.cuh"
using namespace kmv::ptx;

enum Load { kIdle = 0, kTmemLd = 1, kMufu = 2 };

// Warps 0-7 generate `load`, warp 8 issues `chains` chains of `len` MMAs, each followed by a
// commit and (when `wait_each`) a wait for that commit.
template <bool TS, bool WIDE, int LEN>
__global__ void __launch_bounds__(288, 1) probe(int load, int chains, int len_rt, int wait_each, long long* out,
                                                 float* sink, int* err) {
  const int len = LEN > 0 ? LEN : len_rt;
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* bar = (uint64_t*)(sm + 65536);
  uint32_t* slot = (uint32_t*)(bar + 2);
  volatile int* stop = (volatile int*)(slot + 1);
  volatile int* abort = (volatile int*)(slot + 2);
  for (int i = threadIdx.x; i < 65536 / 4; i += blockDim.x) ((uint32_t*)sm)[i] = 0;
  if (threadIdx.x == 0) { mbar_init(&bar[0], 1); mbar_init(&bar[1], 1); *stop = 0; *abort = 0; fence_barrier_init(); }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 8) { tmem_alloc(slot, 512); tmem_relinquish(); }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before(); __syncthreads(); tc_fence_after();
  const uint32_t tb = *slot;
  if (warp == 8) {
    const bool leader = WIDE ? elect_one() : lane == 0;
    if (WIDE || lane == 0) {
      const uint64_t da = sdesc(smem_u32(sm), 128, 512);
      const uint64_t db = sdesc(smem_u32(sm + 32768), 128, 512);
      const uint32_t id = idesc_f16(128, 64, 1, 1);
      uint32_t ph = 0;
      long long t0 = clock64();
      for (int c = 0; c < chains; ++c) {
#pragma unroll
        for (int k = 0; k < (LEN > 0 ? LEN : 8); ++k) {
          if (LEN == 0 && k >= len) break;
          if (leader) {
            if (TS)
              mma_ts(tb, tb + 64 + 8 * (k & 3), db + 16 * (k & 3), id, k > 0);
            else
              mma_ss(tb, da + 16 * (k & 3), db + 16 * (k & 3), id, k > 0);
          }
        }
        if (leader) tc_commit(&bar[0]);
        if (wait_each) {
          mbar_wait(&bar[0], ph, abort, err, 1);
          ph ^= 1;
          tc_fence_after();
        }
      }
      long long t1 = clock64();
      // drain: a commit on a second barrier completes after every MMA issued so far
      if (leader) tc_commit(&bar[1]);
      mbar_wait(&bar[1], 0, abort, err, 2);
      if (blockIdx.x == 0 && leader) out[0] = t1 - t0;
      if (leader) *stop = 1;
    }
    __syncwarp();
  } else {
    // load generators on TMEM columns [256, 512) of their lane quarter
    const uint32_t tl = tb + 256 + 64 * (warp >> 2) + ((uint32_t)(32 * (warp & 3)) << 16);
    float acc = 0.f, x = 0.001f * lane;
    if (load == kTmemLd) {
      while (!*stop) {
        uint32_t v[32];
        tmem_ld32(tl, v);
        tmem_ld_wait();
        acc += __uint_as_float(v[0]) + __uint_as_float(v[31]);
      }
    } else if (load == kMufu) {
      while (!*stop) {
#pragma unroll
        for (int i = 0; i < 64; ++i) x = ex2(x) * 0.5f;
        acc += x;
      }
    }
    if (acc == 123.f) sink[threadIdx.x] = acc;
  }
  tc_fence_before(); __syncthreads(); tc_fence_after();
  if (warp == 8) tmem_dealloc(tb, 512);
}

template <bool TS, bool WIDE, int LEN>
void run(long long* out, float* sink, int* err) {
  cudaFuncSetAttribute(probe<TS, WIDE, LEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 140 * 1024);
  const char* names[3] = {"idle", "tmem-ld", "mufu"};
  const int chains = 256, len = 5;
  for (int wait_each : {0, 1}) {
    for (int load = 0; load < 3; ++load) {
      long long h = 0;
      probe<TS, WIDE, LEN><<<152, 288, 140 * 1024>>>(load, chains, len, wait_each, out, sink, err);
      cudaMemcpy(&h, out, sizeof(h), cudaMemcpyDeviceToHost);
      printf("%s %s len %s %d%s, other warps %-8s: %7.1f clk per chain, %6.1f per MMA\n", TS ? "ts" : "ss",
             WIDE ? "warp  " : "lane 0", LEN ? "const" : "rt   ", len, wait_each ? " + wait" : "       ",
             names[load], (double)h / chains, (double)h / chains / len);
    }
  }
}

int main() {
  long long* out; float* sink; int* err;
  cudaMalloc(&out, 64); cudaMalloc(&sink, 288 * 4); cudaMalloc(&err, 4); cudaMemset(err, 0, 4);
  run<false, false, 5>(out, sink, err);
  run<false, true, 5>(out, sink, err);
  run<true, false, 5>(out, sink, err);
  run<true, true, 5>(out, sink, err);
  int e = 0; cudaMemcpy(&e, err, 4, cudaMemcpyDeviceToHost);
  cudaError_t ce = cudaDeviceSynchronize();
  printf("err=%d cuda=%s\n", e, cudaGetErrorString(ce));
  return ce == cudaSuccess ? 0 : 1;
}

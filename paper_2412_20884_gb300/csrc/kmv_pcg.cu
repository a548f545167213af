// Preconditioned CG (the textbook recurrences with z = P^{-1} r) for the
// batched single right-hand-side solves, with the randomized Nystrom
// preconditioner of kmv_nystrom.cu applied as
//   z = r + U (d o (U^T r)),   d_k = (lambda_r + mu) / (lambda_k + mu) - 1,
// mu = sigma_s^2 of the system's current theta (the Woodbury form for
// A = K + sigma^2 I; the factorisation may come from an earlier theta).
// Per iteration: q = A p (with p.q fused in the product), alpha, x and r,
// U^T r per tile, the per-system coefficients, z and r.z, beta, p.  FP64
// scalars from per-tile partials summed in a fixed order.
#include <algorithm>

#include "kmv_internal.cuh"
#include "simt_common.cuh"

namespace kmv {
namespace {

__device__ __forceinline__ double tile_sum(const DevLayout& L, int b, int c, int chains, const double* partial,
                                           int stride, int k) {
  double acc = 0.0;
  for (int it = L.inst_item0[b]; it < L.inst_item0[b + 1]; ++it) acc += partial[((int64_t)it * chains + c) * stride + k];
  return acc;
}

// r = rhs - q (warm) or rhs (cold, x = 0); partials of r.r and rhs.rhs
__global__ void pcg_init_kernel(DevLayout L, int chains, int64_t n_total, const float* rhs, int64_t rhs_stride,
                                const float* q, float* x, float* r, int warm, double* partial2) {
  __shared__ double red[kTile / 32];
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int64_t i = L.item_row0[item] + threadIdx.x;
  double rr = 0.0, bb = 0.0;
  if (i < L.offsets[b + 1]) {
    const int64_t v = (int64_t)c * n_total + i;
    const float bv = rhs[(int64_t)c * rhs_stride + i];
    float rv = bv;
    if (warm) rv = bv - q[v];
    else x[v] = 0.f;
    r[v] = rv;
    rr = (double)rv * rv;
    bb = (double)bv * bv;
  }
  const double t0 = block_sum(rr, red);
  const double t1 = block_sum(bb, red);
  if (threadIdx.x == 0) {
    partial2[((int64_t)item * chains + c) * 2] = t0;
    partial2[((int64_t)item * chains + c) * 2 + 1] = t1;
  }
}

// partial[tile, c, k] = sum over the tile's rows of U[c, k, i] r_i (warp per k)
__global__ void pcg_proj_kernel(DevLayout L, int chains, int64_t n_total, int rank, const float* U, const float* r,
                                const int32_t* active, double* partial) {
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  if (active && !active[b * chains + c]) return;
  const int64_t r0 = L.item_row0[item], r1 = L.offsets[b + 1];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  float rv[kTile / 32];
#pragma unroll
  for (int u = 0; u < kTile / 32; ++u) {
    const int64_t i = r0 + l + 32 * u;
    rv[u] = i < r1 ? r[(int64_t)c * n_total + i] : 0.f;
  }
  for (int k = w; k < rank; k += kTile / 32) {
    const float* Uk = U + ((int64_t)c * rank + k) * n_total;
    double acc = 0.0;
#pragma unroll
    for (int u = 0; u < kTile / 32; ++u) {
      const int64_t i = r0 + l + 32 * u;
      if (i < r1) acc += (double)Uk[i] * (double)rv[u];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (l == 0) partial[((int64_t)item * chains + c) * rank + k] = acc;
  }
}

// coef[s, k] = d_k * sum over the instance's tiles of partial[., k]
__global__ void pcg_coef_kernel(DevLayout L, int n_inst, int chains, int rank, int n_theta, const double* theta,
                                const double* lam, const double* partial, const int32_t* active, double* coef) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)n_inst * chains * rank) return;
  const int s = (int)(e / rank), k = (int)(e - (int64_t)s * rank);
  if (active && !active[s]) return;
  const int b = s / chains, c = s - b * chains;
  const double mu = exp(theta[(int64_t)s * n_theta + n_theta - 1]);
  const double lr = lam[(int64_t)s * rank + rank - 1];
  const double d = (lr + mu) / (lam[(int64_t)s * rank + k] + mu) - 1.0;
  coef[e] = d * tile_sum(L, b, c, chains, partial, rank, k);
}

// z = r + U coef; partials of r.z
__global__ void pcg_apply_kernel(DevLayout L, int chains, int64_t n_total, int rank, const float* U,
                                 const double* coef, const float* r, float* z, const int32_t* active,
                                 double* partial) {
  __shared__ double red[kTile / 32];
  __shared__ float cf[kMaxRank];
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int s = b * chains + c;
  if (active && !active[s]) return;
  for (int k = threadIdx.x; k < rank; k += blockDim.x) cf[k] = (float)coef[(int64_t)s * rank + k];
  __syncthreads();
  const int64_t i = L.item_row0[item] + threadIdx.x;
  double rz = 0.0;
  if (i < L.offsets[b + 1]) {
    const int64_t v = (int64_t)c * n_total + i;
    const float rv = r[v];
    float acc = 0.f;
    for (int k = 0; k < rank; ++k) acc = fmaf(U[((int64_t)c * rank + k) * n_total + i], cf[k], acc);
    const float zv = rv + acc;
    z[v] = zv;
    rz = (double)rv * zv;
  }
  const double t = block_sum(rz, red);
  if (threadIdx.x == 0) partial[(int64_t)item * chains + c] = t;
}

// rr, bb, rz of every system; active while rr > tol^2 bb; beta = 0 (p = z)
__global__ void pcg_setup_kernel(DevLayout L, int n_inst, int chains, const double* partial2, const double* prz,
                                 double tol, PcgSys* sys, int32_t* active, int32_t* n_active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_inst * chains) return;
  const int b = s / chains, c = s - b * chains;
  PcgSys& y = sys[s];
  y.rr = tile_sum(L, b, c, chains, partial2, 2, 0);
  y.bb = tile_sum(L, b, c, chains, partial2, 2, 1);
  y.rz = tile_sum(L, b, c, chains, prz, 1, 0);
  y.alpha = y.beta = 0.0;
  y.iters = 0;
  y.status = isfinite(y.rr) ? KMV_OK : KMV_ENONFINITE;
  const int act = (y.status == KMV_OK && y.bb > 0.0 && y.rr > tol * tol * y.bb) ? 1 : 0;
  active[s] = act;
  if (act) atomicAdd(n_active, 1);
}

__global__ void pcg_alpha_kernel(DevLayout L, int n_inst, int chains, const double* partial, PcgSys* sys,
                                 int32_t* active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_inst * chains || !active[s]) return;
  const int b = s / chains, c = s - b * chains;
  PcgSys& y = sys[s];
  const double pq = tile_sum(L, b, c, chains, partial, 1, 0);
  if (!(pq > 0.0) || !isfinite(pq) || !(y.rz > 0.0)) {
    y.status = isfinite(pq) && isfinite(y.rz) ? KMV_ENOTCONV : KMV_ENONFINITE;
    y.alpha = 0.0;
    active[s] = 0;
    return;
  }
  y.alpha = y.rz / pq;
}

// x += alpha p, r -= alpha q; partials of r.r
__global__ void pcg_update_xr_kernel(DevLayout L, int chains, int64_t n_total, const PcgSys* sys,
                                     const int32_t* active, float* x, float* r, const float* p, const float* q,
                                     double* partial) {
  __shared__ double red[kTile / 32];
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int s = b * chains + c;
  if (!active[s]) return;
  const float al = (float)sys[s].alpha;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  double rr = 0.0;
  if (i < L.offsets[b + 1]) {
    const int64_t v = (int64_t)c * n_total + i;
    x[v] = fmaf(al, p[v], x[v]);
    const float rv = fmaf(-al, q[v], r[v]);
    r[v] = rv;
    rr = (double)rv * rv;
  }
  const double t = block_sum(rr, red);
  if (threadIdx.x == 0) partial[(int64_t)item * chains + c] = t;
}

// stopping test on r.r; beta = r.z' / r.z
__global__ void pcg_beta_kernel(DevLayout L, int n_inst, int chains, const double* prr, const double* prz,
                                double tol, int maxiter, PcgSys* sys, int32_t* active, int32_t* n_active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_inst * chains || !active[s]) return;
  const int b = s / chains, c = s - b * chains;
  PcgSys& y = sys[s];
  const double rr = tile_sum(L, b, c, chains, prr, 1, 0);
  const double rz = tile_sum(L, b, c, chains, prz, 1, 0);
  y.iters += 1;
  y.beta = rz / y.rz;
  y.rr = rr;
  y.rz = rz;
  int act = 1;
  if (!isfinite(rr) || !isfinite(rz)) {
    y.status = KMV_ENONFINITE;
    act = 0;
  } else if (rr <= tol * tol * y.bb) {
    act = 0;
  } else if (y.iters >= maxiter) {
    y.status = KMV_ENOTCONV;
    act = 0;
  }
  active[s] = act;
  if (act) atomicAdd(n_active, 1);
}

// p = z + beta p
__global__ void pcg_update_p_kernel(DevLayout L, int chains, int64_t n_total, const PcgSys* sys,
                                    const int32_t* active, const float* z, float* p) {
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int s = b * chains + c;
  if (!active[s]) return;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  if (i >= L.offsets[b + 1]) return;
  const int64_t v = (int64_t)c * n_total + i;
  p[v] = fmaf((float)sys[s].beta, p[v], z[v]);
}

__global__ void pcg_finish_kernel(int n_sys, const PcgSys* sys, const int32_t* active, int32_t* status,
                                  int32_t* iters) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sys; s += gridDim.x * blockDim.x) {
    status[s] = sys[s].status != KMV_OK ? sys[s].status : (active[s] ? KMV_ENOTCONV : KMV_OK);
    if (iters) iters[s] = sys[s].iters;
  }
}

}  // namespace

cudaError_t launch_pcg_init(const DevLayout& L, int n_items, int chains, int64_t n_total, const float* rhs,
                            int64_t rhs_stride, const float* q, float* x, float* r, int warm, double* partial2,
                            cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  pcg_init_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, rhs, rhs_stride, q, x, r, warm,
                                                           partial2);
  return cudaGetLastError();
}

cudaError_t launch_pcg_precond(const DevLayout& L, int n_items, int n_inst, int chains, int64_t n_total,
                               const PcgPrecond& P, const double* theta, int n_theta, const float* r, float* z,
                               const int32_t* active, double* proj, double* coef, double* prz, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  pcg_proj_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, P.rank, P.U, r, active, proj);
  const int64_t n = (int64_t)n_inst * chains * P.rank;
  pcg_coef_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(L, n_inst, chains, P.rank, n_theta, theta, P.lam,
                                                               proj, active, coef);
  pcg_apply_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, P.rank, P.U, coef, r, z, active,
                                                            prz);
  return cudaGetLastError();
}

cudaError_t launch_pcg_setup(const DevLayout& L, int n_inst, int chains, const double* partial2, const double* prz,
                             double tol, PcgSys* sys, int32_t* active, int32_t* n_active, cudaStream_t st) {
  const int n = n_inst * chains;
  pcg_setup_kernel<<<(n + 127) / 128, 128, 0, st>>>(L, n_inst, chains, partial2, prz, tol, sys, active, n_active);
  return cudaGetLastError();
}

cudaError_t launch_pcg_alpha(const DevLayout& L, int n_inst, int chains, const double* partial, PcgSys* sys,
                             int32_t* active, cudaStream_t st) {
  const int n = n_inst * chains;
  pcg_alpha_kernel<<<(n + 127) / 128, 128, 0, st>>>(L, n_inst, chains, partial, sys, active);
  return cudaGetLastError();
}

cudaError_t launch_pcg_update_xr(const DevLayout& L, int n_items, int chains, int64_t n_total, const PcgSys* sys,
                                 const int32_t* active, float* x, float* r, const float* p, const float* q,
                                 double* partial, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  pcg_update_xr_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, sys, active, x, r, p, q,
                                                                partial);
  return cudaGetLastError();
}

cudaError_t launch_pcg_beta(const DevLayout& L, int n_inst, int chains, const double* prr, const double* prz,
                            double tol, int maxiter, PcgSys* sys, int32_t* active, int32_t* n_active,
                            cudaStream_t st) {
  const int n = n_inst * chains;
  pcg_beta_kernel<<<(n + 127) / 128, 128, 0, st>>>(L, n_inst, chains, prr, prz, tol, maxiter, sys, active,
                                                   n_active);
  return cudaGetLastError();
}

cudaError_t launch_pcg_update_p(const DevLayout& L, int n_items, int chains, int64_t n_total, const PcgSys* sys,
                                const int32_t* active, const float* z, float* p, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  pcg_update_p_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, sys, active, z, p);
  return cudaGetLastError();
}

cudaError_t launch_pcg_finish(int n_sys, const PcgSys* sys, const int32_t* active, int32_t* status, int32_t* iters,
                              cudaStream_t st) {
  if (n_sys == 0) return cudaSuccess;
  pcg_finish_kernel<<<(n_sys + 255) / 256, 256, 0, st>>>(n_sys, sys, active, status, iters);
  return cudaGetLastError();
}

}  // namespace kmv

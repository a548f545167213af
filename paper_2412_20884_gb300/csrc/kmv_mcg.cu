// Conjugate gradients on several shifted systems per (instance, chain) at once:
// (A_s + shift_{s,q} I) x_q = b_q for the m columns q of every system s, one
// m-column product per iteration (the shifted systems of the pole expansion of
// App. A, Sec. 3.1).  Each column runs its own CG (its own alpha, beta and
// stopping test); a system whose columns have all stopped drops out of the
// product.  FP64 scalars, per-(tile, chain, column) partial sums reduced in a
// fixed order, so the iterates are bitwise reproducible.
#include <algorithm>

#include "kmv_internal.cuh"
#include "simt_common.cuh"

namespace kmv {
namespace {

// Sums v over the block (kTile threads) for every column, writing one partial per column.
__device__ __forceinline__ void block_sum_cols(double v, double* red, double* out) {
  const double t = block_sum(v, red);
  if (threadIdx.x == 0) *out = t;
}

// x = 0 (cold) or kept (warm, with q = A x given); r = b - q; p = r; partials of r.r and b.b.
// b is (chains, N) shared by the m columns when b_cols == 0, else (chains, N, m).
__global__ void mcg_init_kernel(DevLayout L, int chains, int64_t n_total, int m, const float* b, int b_cols,
                                const float* q, int warm, float* x, float* r, float* p, double* partial2) {
  __shared__ double red[kTile / 32];
  const int item = blockIdx.x, c = blockIdx.y;
  const int bi = L.item_inst[item];
  const int64_t i = L.item_row0[item] + threadIdx.x;
  const bool valid = i < L.offsets[bi + 1];
  for (int col = 0; col < m; ++col) {
    double rr = 0.0, bb = 0.0;
    if (valid) {
      const int64_t v = ((int64_t)c * n_total + i) * m + col;
      const float bv = b_cols ? b[v] : b[(int64_t)c * n_total + i];
      float rv = bv;
      if (warm) rv = bv - q[v];
      else x[v] = 0.f;
      r[v] = rv;
      p[v] = rv;
      rr = (double)rv * rv;
      bb = (double)bv * bv;
    }
    const int64_t o = (((int64_t)item * chains + c) * m + col) * 2;
    block_sum_cols(rr, red, partial2 + o);
    block_sum_cols(bb, red, partial2 + o + 1);
  }
}

// Per system: sum the partials of its tiles in order; a column is active while
// r.r > tol^2 b.b.  sys_any[s] = some column of s active.
__global__ void mcg_reduce_init_kernel(DevLayout L, int n_inst, int chains, int m, const double* partial2,
                                       double tol, McgCol* st, int32_t* sys_any, int32_t* n_active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_inst * chains) return;
  const int bi = s / chains, c = s - bi * chains;
  int any = 0;
  for (int col = 0; col < m; ++col) {
    double rr = 0.0, bb = 0.0;
    for (int it = L.inst_item0[bi]; it < L.inst_item0[bi + 1]; ++it) {
      const int64_t o = (((int64_t)it * chains + c) * m + col) * 2;
      rr += partial2[o];
      bb += partial2[o + 1];
    }
    McgCol& k = st[(int64_t)s * m + col];
    k.rr = rr;
    k.bb = bb;
    k.alpha = k.beta = 0.0;
    k.iters = 0;
    k.status = KMV_OK;
    k.pad = 0;
    k.active = (bb > 0.0 && rr > tol * tol * bb) ? 1 : 0;
    if (!isfinite(rr)) {
      k.active = 0;
      k.status = KMV_ENONFINITE;
    }
    any |= k.active;
    if (k.active) atomicAdd(n_active, 1);
  }
  sys_any[s] = any;
}

// partials of p.q per column
__global__ void mcg_dot_kernel(DevLayout L, int chains, int64_t n_total, int m, const float* p, const float* q,
                               const int32_t* sys_any, double* partial) {
  __shared__ double red[kTile / 32];
  const int item = blockIdx.x, c = blockIdx.y;
  const int bi = L.item_inst[item];
  if (!sys_any[bi * chains + c]) return;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  const bool valid = i < L.offsets[bi + 1];
  for (int col = 0; col < m; ++col) {
    double v = 0.0;
    if (valid) {
      const int64_t o = ((int64_t)c * n_total + i) * m + col;
      v = (double)p[o] * q[o];
    }
    block_sum_cols(v, red, partial + ((int64_t)item * chains + c) * m + col);
  }
}

// alpha = r.r / p.q (r.z / p.q when preconditioned) for the active columns; a
// non-positive p.q is a breakdown.
__global__ void mcg_alpha_kernel(DevLayout L, int n_inst, int chains, int m, const double* partial, McgCol* st,
                                 const int32_t* sys_any, int pre) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_inst * chains || !sys_any[s]) return;
  const int bi = s / chains, c = s - bi * chains;
  for (int col = 0; col < m; ++col) {
    McgCol& k = st[(int64_t)s * m + col];
    if (!k.active) {
      k.alpha = 0.0;
      continue;
    }
    double pq = 0.0;
    for (int it = L.inst_item0[bi]; it < L.inst_item0[bi + 1]; ++it)
      pq += partial[((int64_t)it * chains + c) * m + col];
    const double num = pre ? k.rz : k.rr;
    if (!(pq > 0.0) || !isfinite(pq) || !(num > 0.0)) {
      k.alpha = 0.0;
      k.active = 0;
      k.status = (isfinite(pq) && isfinite(num)) ? KMV_ENOTCONV : KMV_ENONFINITE;
    } else {
      k.alpha = num / pq;
    }
  }
}

// x += alpha p, r -= alpha q on the active columns; partials of the new r.r
__global__ void mcg_update_xr_kernel(DevLayout L, int chains, int64_t n_total, int m, const McgCol* st,
                                     const int32_t* sys_any, float* x, float* r, const float* p, const float* q,
                                     double* partial) {
  __shared__ double red[kTile / 32];
  const int item = blockIdx.x, c = blockIdx.y;
  const int bi = L.item_inst[item];
  const int s = bi * chains + c;
  if (!sys_any[s]) return;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  const bool valid = i < L.offsets[bi + 1];
  for (int col = 0; col < m; ++col) {
    const McgCol& k = st[(int64_t)s * m + col];
    double rr = 0.0;
    if (valid) {
      const int64_t o = ((int64_t)c * n_total + i) * m + col;
      float rv = r[o];
      if (k.active) {
        const float al = (float)k.alpha;
        x[o] = fmaf(al, p[o], x[o]);
        rv = fmaf(-al, q[o], rv);
        r[o] = rv;
      }
      rr = (double)rv * rv;
    }
    block_sum_cols(rr, red, partial + ((int64_t)item * chains + c) * m + col);
  }
}

// beta = r.r_new / r.r (r.z_new / r.z when preconditioned, prz != NULL); stop
// converged columns (r.r <= tol^2 b.b) and those at maxiter
__global__ void mcg_beta_kernel(DevLayout L, int n_inst, int chains, int m, const double* partial,
                                const double* prz, double tol, int maxiter, McgCol* st, int32_t* sys_any,
                                int32_t* n_active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_inst * chains || !sys_any[s]) return;
  const int bi = s / chains, c = s - bi * chains;
  int any = 0;
  for (int col = 0; col < m; ++col) {
    McgCol& k = st[(int64_t)s * m + col];
    if (!k.active) continue;
    double rr = 0.0;
    for (int it = L.inst_item0[bi]; it < L.inst_item0[bi + 1]; ++it)
      rr += partial[((int64_t)it * chains + c) * m + col];
    if (prz) {
      double rz = 0.0;
      for (int it = L.inst_item0[bi]; it < L.inst_item0[bi + 1]; ++it)
        rz += prz[((int64_t)it * chains + c) * m + col];
      k.beta = rz / k.rz;
      k.rz = rz;
    } else {
      k.beta = rr / k.rr;
    }
    k.rr = rr;
    k.iters += 1;
    if (!isfinite(rr)) {
      k.active = 0;
      k.status = KMV_ENONFINITE;
    } else if (rr <= tol * tol * k.bb) {
      k.active = 0;
    } else if (k.iters >= maxiter) {
      k.active = 0;
      k.status = KMV_ENOTCONV;
    }
    any |= k.active;
    if (k.active) atomicAdd(n_active, 1);
  }
  sys_any[s] = any;
}

// p = r + beta p on the active columns (r is z when preconditioned)
__global__ void mcg_update_p_kernel(DevLayout L, int chains, int64_t n_total, int m, const McgCol* st,
                                    const int32_t* sys_any, const float* r, float* p) {
  const int item = blockIdx.x, c = blockIdx.y;
  const int bi = L.item_inst[item];
  const int s = bi * chains + c;
  if (!sys_any[s]) return;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  if (i >= L.offsets[bi + 1]) return;
  for (int col = 0; col < m; ++col) {
    const McgCol& k = st[(int64_t)s * m + col];
    if (!k.active) continue;
    const int64_t o = ((int64_t)c * n_total + i) * m + col;
    p[o] = fmaf((float)k.beta, p[o], r[o]);
  }
}

// Column results of a finished solve: col_status = the column's status
// (KMV_ENOTCONV if still active), col_iters = its iterations.  With accumulate
// (an inner solve of the refinement) the iterations add up and only a
// non-finite inner solve marks the column.
__global__ void mcg_finish_kernel(int64_t n_cols, const McgCol* cols, int accumulate, int32_t* col_status,
                                  int32_t* col_iters) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_cols; e += (int64_t)gridDim.x * blockDim.x) {
    const McgCol& k = cols[e];
    if (accumulate) {
      col_iters[e] += k.iters;
      if (k.status == KMV_ENONFINITE) col_status[e] = KMV_ENONFINITE;
    } else {
      col_status[e] = k.active ? KMV_ENOTCONV : k.status;
      col_iters[e] = k.iters;
    }
  }
}

// r[., ., q] = 0 for the columns the refinement no longer corrects.
__global__ void mcg_mask_kernel(DevLayout L, int chains, int64_t n_total, int m, const McgCol* cols, float* r) {
  const int item = blockIdx.x, c = blockIdx.y;
  const int bi = L.item_inst[item];
  const int s = bi * chains + c;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  if (i >= L.offsets[bi + 1]) return;
  for (int col = 0; col < m; ++col)
    if (!cols[(int64_t)s * m + col].active) r[((int64_t)c * n_total + i) * m + col] = 0.f;
}

// Refinement step bookkeeping per column, as for the single-column refinement:
// a column whose true residual fell by less than half since the last step has
// reached the floor of the FP32 operator and stops; one whose residual rose is
// marked (pad = 1) for the last correction to be taken back.  n_active =
// columns left, worst = the largest rr / bb among them.  One block.
__global__ void mcg_refine_kernel(int64_t n_cols, int outer, McgCol* cols, double* prev_rr, int32_t* n_active,
                                  double* worst) {
  __shared__ int cnt[8];
  __shared__ double wmax[8];
  int v = 0;
  double wr = 0.0;
  for (int64_t e = threadIdx.x; e < n_cols; e += blockDim.x) {
    McgCol& k = cols[e];
    if (k.active && outer > 0 && k.rr > 0.25 * prev_rr[e]) {
      k.active = 0;
      if (k.rr > prev_rr[e]) {
        k.pad = 1;
        k.rr = prev_rr[e];
      }
    }
    prev_rr[e] = k.rr;
    v += k.active;
    if (k.active && k.bb > 0.0) wr = fmax(wr, k.rr / k.bb);
  }
  for (int o = 16; o > 0; o >>= 1) {
    v += __shfl_down_sync(0xffffffffu, v, o);
    wr = fmax(wr, __shfl_down_sync(0xffffffffu, wr, o));
  }
  if ((threadIdx.x & 31) == 0) {
    cnt[threadIdx.x >> 5] = v;
    wmax[threadIdx.x >> 5] = wr;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    double mx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t += cnt[w];
      mx = fmax(mx, wmax[w]);
    }
    *n_active = t;
    *worst = mx;
  }
}

// x[., ., q] -= dx[., ., q] for the columns whose last correction raised the residual.
__global__ void mcg_undo_kernel(DevLayout L, int chains, int64_t n_total, int m, const McgCol* cols,
                                const float* dx, float* x) {
  const int item = blockIdx.x, c = blockIdx.y;
  const int bi = L.item_inst[item];
  const int s = bi * chains + c;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  if (i >= L.offsets[bi + 1]) return;
  for (int col = 0; col < m; ++col) {
    if (!cols[(int64_t)s * m + col].pad) continue;
    const int64_t o = ((int64_t)c * n_total + i) * m + col;
    x[o] -= dx[o];
  }
}

// Final refinement status: a column still active after the last step did not converge.
__global__ void mcg_refine_finish_kernel(int64_t n_cols, const McgCol* cols, int32_t* col_status) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_cols; e += (int64_t)gridDim.x * blockDim.x) {
    if (col_status[e] != KMV_OK) continue;
    if (cols[e].status != KMV_OK) col_status[e] = cols[e].status;
    else if (cols[e].active) col_status[e] = KMV_ENOTCONV;
  }
}

// Multi-column projection: partial[tile, c, q, k] = sum over the tile's rows of
// U[c, k, i] r[c, i, q]; the tile's r columns are staged in shared memory and
// each U row segment is read once for all columns.
__global__ void mcg_proj_kernel(DevLayout L, int chains, int64_t n_total, int m, int rank, const float* U,
                                const float* r, const int32_t* sys_any, double* partial) {
  __shared__ float rs[kMaxShifts][kTile];
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  if (sys_any && !sys_any[b * chains + c]) return;
  const int64_t r0 = L.item_row0[item], r1 = L.offsets[b + 1];
  for (int e = threadIdx.x; e < m * kTile; e += blockDim.x) {
    const int row = e / m, q = e - row * m;
    const int64_t i = r0 + row;
    rs[q][row] = i < r1 ? r[((int64_t)c * n_total + i) * m + q] : 0.f;
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int k = w; k < rank; k += kTile / 32) {
    const float* Uk = U + ((int64_t)c * rank + k) * n_total;
    float u[kTile / 32];
#pragma unroll
    for (int t = 0; t < kTile / 32; ++t) {
      const int64_t i = r0 + l + 32 * t;
      u[t] = i < r1 ? Uk[i] : 0.f;
    }
    for (int q = 0; q < m; ++q) {
      double acc = 0.0;
#pragma unroll
      for (int t = 0; t < kTile / 32; ++t) acc += (double)u[t] * (double)rs[q][l + 32 * t];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (l == 0) partial[(((int64_t)item * chains + c) * m + q) * rank + k] = acc;
    }
  }
}

// coef[s, q, k] = d_{q,k} sum over the instance's tiles of partial[., q, k],
// d = (lambda_r + mu_q) / (lambda_k + mu_q) - 1, mu_q = sigma_s^2 + shift[s, q]
__global__ void mcg_coef_kernel(DevLayout L, int n_inst, int chains, int m, int rank, int n_theta,
                                const double* theta, const float* shifts, const double* lam, const double* partial,
                                const int32_t* sys_any, double* coef) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)n_inst * chains * m * rank) return;
  const int k = (int)(e % rank);
  const int64_t sq = e / rank;
  const int q = (int)(sq % m), s = (int)(sq / m);
  if (sys_any && !sys_any[s]) return;
  const int b = s / chains, c = s - b * chains;
  const double mu = exp(theta[(int64_t)s * n_theta + n_theta - 1]) + (double)shifts[(int64_t)s * m + q];
  const double lr = lam[(int64_t)s * rank + rank - 1];
  const double d = (lr + mu) / (lam[(int64_t)s * rank + k] + mu) - 1.0;
  double acc = 0.0;
  for (int it = L.inst_item0[b]; it < L.inst_item0[b + 1]; ++it)
    acc += partial[(((int64_t)it * chains + c) * m + q) * rank + k];
  coef[e] = d * acc;
}

// z[c, i, q] = r[c, i, q] + sum_k U[c, k, i] coef[s, q, k]; partials of r.z per column
__global__ void mcg_apply_kernel(DevLayout L, int chains, int64_t n_total, int m, int rank, const float* U,
                                 const double* coef, const float* r, float* z, const int32_t* sys_any,
                                 double* prz) {
  extern __shared__ float cf[];   // m x rank
  __shared__ double red[kTile / 32][kMaxShifts];
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int s = b * chains + c;
  if (sys_any && !sys_any[s]) return;
  for (int e = threadIdx.x; e < m * rank; e += blockDim.x) cf[e] = (float)coef[(int64_t)s * m * rank + e];
  __syncthreads();
  const int64_t i = L.item_row0[item] + threadIdx.x;
  const bool valid = i < L.offsets[b + 1];
  float acc[kMaxShifts];
#pragma unroll
  for (int q = 0; q < kMaxShifts; ++q) acc[q] = 0.f;
  if (valid) {
    for (int k = 0; k < rank; ++k) {
      const float u = U[((int64_t)c * rank + k) * n_total + i];
#pragma unroll
      for (int q = 0; q < kMaxShifts; ++q)
        if (q < m) acc[q] = fmaf(u, cf[q * rank + k], acc[q]);
    }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < kMaxShifts; ++q) {
    if (q >= m) break;
    double v = 0.0;
    if (valid) {
      const int64_t o = ((int64_t)c * n_total + i) * m + q;
      const float rv = r[o];
      const float zv = rv + acc[q];
      z[o] = zv;
      v = (double)rv * zv;
    }
    for (int o2 = 16; o2 > 0; o2 >>= 1) v += __shfl_down_sync(0xffffffffu, v, o2);
    if (l == 0) red[w][q] = v;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    double t = 0.0;
    for (int u = 0; u < kTile / 32; ++u) t += red[u][q];
    prz[((int64_t)item * chains + c) * m + q] = t;
  }
}

// rz of every column from the per-tile partials (after the first preconditioning)
__global__ void mcg_set_rz_kernel(DevLayout L, int n_inst, int chains, int m, const double* prz, McgCol* cols) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_inst * chains) return;
  const int b = s / chains, c = s - b * chains;
  for (int q = 0; q < m; ++q) {
    double rz = 0.0;
    for (int it = L.inst_item0[b]; it < L.inst_item0[b + 1]; ++it) rz += prz[((int64_t)it * chains + c) * m + q];
    cols[(int64_t)s * m + q].rz = rz;
  }
}

}  // namespace

cudaError_t launch_mcg_precond(const DevLayout& L, int n_items, int n_inst, int chains, int64_t n_total, int m,
                               const PcgPrecond& P, const double* theta, int n_theta, const float* shifts,
                               const float* r, float* z, const int32_t* sys_any, double* proj, double* coef,
                               double* prz, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  mcg_proj_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, m, P.rank, P.U, r, sys_any, proj);
  const int64_t n = (int64_t)n_inst * chains * m * P.rank;
  mcg_coef_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(L, n_inst, chains, m, P.rank, n_theta, theta, shifts,
                                                               P.lam, proj, sys_any, coef);
  mcg_apply_kernel<<<dim3(n_items, chains), kTile, sizeof(float) * m * P.rank, st>>>(L, chains, n_total, m, P.rank,
                                                                                     P.U, coef, r, z, sys_any, prz);
  return cudaGetLastError();
}

cudaError_t launch_mcg_set_rz(const DevLayout& L, int n_inst, int chains, int m, const double* prz, McgCol* cols,
                              cudaStream_t st) {
  const int n = n_inst * chains;
  mcg_set_rz_kernel<<<(n + 127) / 128, 128, 0, st>>>(L, n_inst, chains, m, prz, cols);
  return cudaGetLastError();
}

cudaError_t launch_mcg_finish(int64_t n_cols, const McgCol* cols, int accumulate, int32_t* col_status,
                              int32_t* col_iters, cudaStream_t st) {
  if (n_cols == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n_cols + 255) / 256, 1024);
  mcg_finish_kernel<<<blocks, 256, 0, st>>>(n_cols, cols, accumulate, col_status, col_iters);
  return cudaGetLastError();
}

cudaError_t launch_mcg_mask(const DevLayout& L, int n_items, int chains, int64_t n_total, int m, const McgCol* cols,
                            float* r, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  mcg_mask_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, m, cols, r);
  return cudaGetLastError();
}

cudaError_t launch_mcg_refine(int64_t n_cols, int outer, McgCol* cols, double* prev_rr, int32_t* n_active,
                              double* worst, cudaStream_t st) {
  mcg_refine_kernel<<<1, 256, 0, st>>>(n_cols, outer, cols, prev_rr, n_active, worst);
  return cudaGetLastError();
}

cudaError_t launch_mcg_undo(const DevLayout& L, int n_items, int chains, int64_t n_total, int m, const McgCol* cols,
                            const float* dx, float* x, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  mcg_undo_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, m, cols, dx, x);
  return cudaGetLastError();
}

cudaError_t launch_mcg_refine_finish(int64_t n_cols, const McgCol* cols, int32_t* col_status, cudaStream_t st) {
  if (n_cols == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n_cols + 255) / 256, 1024);
  mcg_refine_finish_kernel<<<blocks, 256, 0, st>>>(n_cols, cols, col_status);
  return cudaGetLastError();
}

cudaError_t launch_mcg_init(const DevLayout& L, int n_items, int chains, int64_t n_total, int m, const float* b,
                            int b_cols, const float* q, int warm, float* x, float* r, float* p, double* partial2,
                            cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  mcg_init_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, m, b, b_cols, q, warm, x, r, p,
                                                           partial2);
  return cudaGetLastError();
}

cudaError_t launch_mcg_reduce_init(const DevLayout& L, int n_inst, int chains, int m, const double* partial2,
                                   double tol, McgCol* st, int32_t* sys_any, int32_t* n_active, cudaStream_t s) {
  const int n = n_inst * chains;
  mcg_reduce_init_kernel<<<(n + 127) / 128, 128, 0, s>>>(L, n_inst, chains, m, partial2, tol, st, sys_any,
                                                         n_active);
  return cudaGetLastError();
}

cudaError_t launch_mcg_dot(const DevLayout& L, int n_items, int chains, int64_t n_total, int m, const float* p,
                           const float* q, const int32_t* sys_any, double* partial, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  mcg_dot_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, m, p, q, sys_any, partial);
  return cudaGetLastError();
}

cudaError_t launch_mcg_alpha(const DevLayout& L, int n_inst, int chains, int m, const double* partial, McgCol* st,
                             const int32_t* sys_any, int pre, cudaStream_t s) {
  const int n = n_inst * chains;
  mcg_alpha_kernel<<<(n + 127) / 128, 128, 0, s>>>(L, n_inst, chains, m, partial, st, sys_any, pre);
  return cudaGetLastError();
}

cudaError_t launch_mcg_update_xr(const DevLayout& L, int n_items, int chains, int64_t n_total, int m,
                                 const McgCol* stt, const int32_t* sys_any, float* x, float* r, const float* p,
                                 const float* q, double* partial, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  mcg_update_xr_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, m, stt, sys_any, x, r, p, q,
                                                                partial);
  return cudaGetLastError();
}

cudaError_t launch_mcg_beta(const DevLayout& L, int n_inst, int chains, int m, const double* partial,
                            const double* prz, double tol, int maxiter, McgCol* st, int32_t* sys_any,
                            int32_t* n_active, cudaStream_t s) {
  const int n = n_inst * chains;
  mcg_beta_kernel<<<(n + 127) / 128, 128, 0, s>>>(L, n_inst, chains, m, partial, prz, tol, maxiter, st, sys_any,
                                                  n_active);
  return cudaGetLastError();
}

cudaError_t launch_mcg_update_p(const DevLayout& L, int n_items, int chains, int64_t n_total, int m,
                                const McgCol* stt, const int32_t* sys_any, const float* r, float* p,
                                cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  mcg_update_p_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, m, stt, sys_any, r, p);
  return cudaGetLastError();
}

}  // namespace kmv

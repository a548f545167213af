// Batched conjugate gradients, the leapfrog map and the FP64 energy.
//
// All systems s = (instance b, chain c) advance in lockstep; a system that has
// converged (or failed) is masked by its entry in the active[] array, and its
// CTAs return at once.
// Dot products are FP64 per-CTA partials over kTile rows, reduced per system
// in a fixed order (bitwise reproducible).
#include "cg_common.cuh"
#include "simt_common.cuh"

namespace kmv {

// --- CG vectors ------------------------------------------------------------

// r = rhs - q (warm) or rhs (cold), p = r, x = 0 (cold); partials of r.r and rhs.rhs.
__global__ void cg_init_kernel(DevLayout L, int chains, int64_t n_total, const float* rhs,
                               int64_t rhs_stride, const float* q, float* x, float* r, float* p,
                               int warm, double* partial2) {
  __shared__ double red[kTile / 32];
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int64_t i = L.item_row0[item] + threadIdx.x;
  const bool valid = i < L.offsets[b + 1];
  double rr = 0.0, bb = 0.0;
  if (valid) {
    const int64_t v = (int64_t)c * n_total + i;
    const float bi = rhs[(int64_t)c * rhs_stride + i];
    float ri = bi;
    if (warm) ri = bi - q[v];
    else x[v] = 0.f;
    r[v] = ri;
    p[v] = ri;
    rr = (double)ri * ri;
    bb = (double)bi * bi;
  }
  const double t0 = block_sum(rr, red);
  const double t1 = block_sum(bb, red);
  if (threadIdx.x == 0) {
    partial2[((int64_t)item * chains + c) * 2 + 0] = t0;
    partial2[((int64_t)item * chains + c) * 2 + 1] = t1;
  }
}

cudaError_t launch_cg_init(const DevLayout& L, int n_items, int chains, int64_t n_total,
                           const float* rhs, int64_t rhs_stride, const float* q, float* x,
                           float* r, float* p, int warm, double* partial2, cudaStream_t st) {
  cg_init_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, rhs, rhs_stride, q, x,
                                                          r, p, warm, partial2);
  return cudaGetLastError();
}

// Sum of per-item partials of system s (stride entries apart, component k).
// Number of active systems, counted by one CTA (deterministic).
__device__ __forceinline__ void count_active(int n_sys, const int32_t* active, int32_t* n_active) {
  __shared__ int cnt[8];
  int v = 0;
  for (int s = threadIdx.x; s < n_sys; s += blockDim.x) v += active[s];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) cnt[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += cnt[w];
    *n_active = t;
  }
}

__global__ void cg_reduce_init_kernel(DevLayout L, int n_inst, int chains, const double* partial2,
                                      double tol, CgSys* sys, int32_t* active, int32_t* n_active) {
  const int n_sys = n_inst * chains;
  for (int s = threadIdx.x; s < n_sys; s += blockDim.x) {
    const int b = s / chains, c = s - b * chains;
    const double rr = sys_sum(L, b, c, chains, partial2, 2, 0);
    const double bb = sys_sum(L, b, c, chains, partial2, 2, 1);
    CgSys& S = sys[s];
    S.rr = rr;
    S.bb = bb;
    S.pq = 0.0;
    S.alpha = 0.0;
    S.beta = 0.0;
    S.iters = 0;
    S.status = (isfinite(rr) && isfinite(bb)) ? KMV_OK : KMV_ENONFINITE;
    active[s] = (S.status == KMV_OK && rr > tol * tol * bb) ? 1 : 0;
  }
  __syncthreads();
  count_active(n_sys, active, n_active);
}

__global__ void loop_cond_kernel(cudaGraphConditionalHandle cond, const int32_t* n_active) {
  cudaGraphSetConditional(cond, *n_active > 0 ? 1u : 0u);
}

cudaError_t launch_loop_cond(cudaGraphConditionalHandle cond, const int32_t* n_active, cudaStream_t st) {
  loop_cond_kernel<<<1, 1, 0, st>>>(cond, n_active);
  return cudaGetLastError();
}

cudaError_t launch_cg_reduce_init(const DevLayout& L, int n_inst, int chains, const double* partial2,
                                  double tol, CgSys* sys, int32_t* active, int32_t* n_active,
                                  cudaStream_t st) {
  cg_reduce_init_kernel<<<1, 256, 0, st>>>(L, n_inst, chains, partial2, tol, sys, active, n_active);
  return cudaGetLastError();
}

__global__ void cg_reduce_pq_kernel(DevLayout L, int n_inst, int chains, const double* partial,
                                    CgSys* sys, int32_t* active) {
  const int n_sys = n_inst * chains;
  for (int s = threadIdx.x; s < n_sys; s += blockDim.x) {
    if (!active[s]) continue;
    const int b = s / chains, c = s - b * chains;
    if (!cg_pq_step(sys[s], sys_sum(L, b, c, chains, partial, 1, 0))) active[s] = 0;
  }
}

cudaError_t launch_cg_reduce_pq(const DevLayout& L, int n_inst, int chains, const double* partial,
                                CgSys* sys, int32_t* active, cudaStream_t st) {
  cg_reduce_pq_kernel<<<1, 256, 0, st>>>(L, n_inst, chains, partial, sys, active);
  return cudaGetLastError();
}

__global__ void cg_update_xr_kernel(DevLayout L, int chains, int64_t n_total, const CgSys* sys,
                                    const int32_t* active, float* x, float* r, const float* p,
                                    const float* q, double* partial) {
  __shared__ double red[kTile / 32];
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const CgSys& S = sys[b * chains + c];
  if (!active[b * chains + c]) return;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  double rr = 0.0;
  if (i < L.offsets[b + 1]) {
    const int64_t v = (int64_t)c * n_total + i;
    const float al = (float)S.alpha;
    x[v] = fmaf(al, p[v], x[v]);
    const float ri = fmaf(-al, q[v], r[v]);
    r[v] = ri;
    rr = (double)ri * ri;
  }
  const double t = block_sum(rr, red);
  if (threadIdx.x == 0) partial[(int64_t)item * chains + c] = t;
}

cudaError_t launch_cg_update_xr(const DevLayout& L, int n_items, int chains, int64_t n_total,
                                const CgSys* sys, const int32_t* active, float* x, float* r,
                                const float* p, const float* q, double* partial, cudaStream_t st) {
  cg_update_xr_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, sys, active, x, r,
                                                               p, q, partial);
  return cudaGetLastError();
}

// x += alpha p, r -= alpha q and the r.r partials, as cg_update_xr_kernel;
// the CTA of each system that finishes last then takes the system's r.r step
// (as cg_reduce_rr_kernel) and keeps n_active up to date by decrements, so an
// iteration needs no separate reduction launch.
__global__ void cg_update_xr_rr_kernel(DevLayout L, int chains, int64_t n_total, CgSys* sys, int32_t* active,
                                       float* x, float* r, const float* p, const float* q, double* partial,
                                       uint32_t* count, double tol, int maxiter, int32_t* n_active) {
  __shared__ double red[kTile / 32];
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int s = b * chains + c;
  if (!active[s]) return;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  double rr = 0.0;
  if (i < L.offsets[b + 1]) {
    const int64_t v = (int64_t)c * n_total + i;
    const float al = (float)sys[s].alpha;
    x[v] = fmaf(al, p[v], x[v]);
    const float ri = fmaf(-al, q[v], r[v]);
    r[v] = ri;
    rr = (double)ri * ri;
  }
  const double t = block_sum(rr, red);
  if (threadIdx.x == 0) {
    partial[(int64_t)item * chains + c] = t;
    const bool last = last_block_of_system(count, s, (uint32_t)(L.inst_item0[b + 1] - L.inst_item0[b]));
    if (last && !cg_rr_step(sys[s], sys_sum(L, b, c, chains, partial, 1, 0), tol, maxiter)) {
      active[s] = 0;
      atomicSub(n_active, 1);
    }
  }
}

cudaError_t launch_cg_update_xr_rr(const DevLayout& L, int n_items, int chains, int64_t n_total, CgSys* sys,
                                   int32_t* active, float* x, float* r, const float* p, const float* q,
                                   double* partial, uint32_t* count, double tol, int maxiter, int32_t* n_active,
                                   cudaStream_t st) {
  cg_update_xr_rr_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, sys, active, x, r, p, q,
                                                                  partial, count, tol, maxiter, n_active);
  return cudaGetLastError();
}

__global__ void cg_reduce_rr_kernel(DevLayout L, int n_inst, int chains, const double* partial,
                                    double tol, int maxiter, CgSys* sys, int32_t* active,
                                    int32_t* n_active) {
  const int n_sys = n_inst * chains;
  for (int s = threadIdx.x; s < n_sys; s += blockDim.x) {
    if (!active[s]) continue;
    const int b = s / chains, c = s - b * chains;
    if (!cg_rr_step(sys[s], sys_sum(L, b, c, chains, partial, 1, 0), tol, maxiter)) active[s] = 0;
  }
  __syncthreads();
  count_active(n_sys, active, n_active);
}

cudaError_t launch_cg_reduce_rr(const DevLayout& L, int n_inst, int chains, const double* partial,
                                double tol, int maxiter, CgSys* sys, int32_t* active,
                                int32_t* n_active, cudaStream_t st) {
  cg_reduce_rr_kernel<<<1, 256, 0, st>>>(L, n_inst, chains, partial, tol, maxiter, sys, active,
                                         n_active);
  return cudaGetLastError();
}

__global__ void cg_update_p_kernel(DevLayout L, int chains, int64_t n_total, const CgSys* sys,
                                   const int32_t* active, const float* r, float* p) {
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const CgSys& S = sys[b * chains + c];
  if (!active[b * chains + c]) return;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  if (i < L.offsets[b + 1]) {
    const int64_t v = (int64_t)c * n_total + i;
    p[v] = fmaf((float)S.beta, p[v], r[v]);
  }
}

cudaError_t launch_cg_update_p(const DevLayout& L, int n_items, int chains, int64_t n_total,
                               const CgSys* sys, const int32_t* active, const float* r, float* p,
                               cudaStream_t st) {
  cg_update_p_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, sys, active, r, p);
  return cudaGetLastError();
}

__global__ void cg_finish_kernel(int n_sys, const CgSys* sys, int32_t* status, int32_t* iters) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sys; s += gridDim.x * blockDim.x) {
    status[s] = sys[s].status;
    if (iters) iters[s] = sys[s].iters;
  }
}

cudaError_t launch_cg_finish(int n_sys, const CgSys* sys, int32_t* status, int32_t* iters,
                             cudaStream_t st) {
  cg_finish_kernel<<<(n_sys + 255) / 256, 256, 0, st>>>(n_sys, sys, status, iters);
  return cudaGetLastError();
}

// --- mixed-precision refinement helpers -------------------------------------------

// r[c, rows of b] = 0 for systems that are not active (their correction is 0).
__global__ void mask_rows_kernel(DevLayout L, int chains, int64_t n_total, const int32_t* active, float* r) {
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  if (active[b * chains + c]) return;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  if (i < L.offsets[b + 1]) r[(int64_t)c * n_total + i] = 0.f;
}

cudaError_t launch_mask_rows(const DevLayout& L, int n_items, int chains, int64_t n_total, const int32_t* active,
                             float* r, cudaStream_t st) {
  mask_rows_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, active, r);
  return cudaGetLastError();
}

__global__ void axpy_kernel(int64_t n, const float* dx, float* x) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    x[e] += dx[e];
}

cudaError_t launch_axpy(int64_t n, const float* dx, float* x, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 32);
  axpy_kernel<<<blocks, 256, 0, st>>>(n, dx, x);
  return cudaGetLastError();
}

// Folds an inner solve's per-system results into the outer ones: iterations
// add up; a failed inner solve marks the system.
__global__ void refine_merge_kernel(int n_sys, const int32_t* in_status, const int32_t* in_iters,
                                    int32_t* status, int32_t* iters) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sys; s += gridDim.x * blockDim.x) {
    if (iters) iters[s] += in_iters[s];
    // a correction solve that failed (non-finite, or cg_maxiter / breakdown) is
    // remembered; refine_finish clears the latter if the final residual meets tol
    if (in_status[s] == KMV_ENONFINITE) status[s] = KMV_ENONFINITE;
    else if (in_status[s] == KMV_ENOTCONV && status[s] == KMV_OK) status[s] = KMV_ENOTCONV;
  }
}

cudaError_t launch_refine_merge(int n_sys, const int32_t* in_status, const int32_t* in_iters, int32_t* status,
                                int32_t* iters, cudaStream_t st) {
  refine_merge_kernel<<<(n_sys + 255) / 256, 256, 0, st>>>(n_sys, in_status, in_iters, status, iters);
  return cudaGetLastError();
}

// Stops refinement of systems whose true residual no longer falls by at least
// half per outer step: the residual has reached the floor set by the FP32
// operator it is measured with, which is as far as the solve can go (the FP32
// CG stops on its recurrence residual, which passes below that floor).
// Also reports, in worst[0], the largest rr / bb over the systems still active.
__global__ void refine_stagnation_kernel(int n_sys, int outer, const CgSys* sys, double* prev_rr, int32_t* active,
                                         int32_t* n_active, double* worst) {
  __shared__ int cnt[8];
  __shared__ double wmax[8];
  int v = 0;
  double wr = 0.0;
  for (int s = threadIdx.x; s < n_sys; s += blockDim.x) {
    const double rr = sys[s].rr;
    if (active[s] && outer > 0 && rr > 0.25 * prev_rr[s]) active[s] = 0;
    prev_rr[s] = rr;
    v += active[s];
    if (active[s] && sys[s].bb > 0.0) wr = fmax(wr, rr / sys[s].bb);
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
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t += cnt[w];
      m = fmax(m, wmax[w]);
    }
    *n_active = t;
    *worst = m;
  }
}

cudaError_t launch_refine_stagnation(int n_sys, int outer, const CgSys* sys, double* prev_rr, int32_t* active,
                                     int32_t* n_active, double* worst, cudaStream_t st) {
  refine_stagnation_kernel<<<1, 256, 0, st>>>(n_sys, outer, sys, prev_rr, active, n_active, worst);
  return cudaGetLastError();
}

// Final outer status from the last true residual rr (sys[s].rr): converged if
// rr <= tol^2 bb; otherwise converged only when the residual stopped falling
// with every correction solve converged (the floor of the FP32 operator),
// and not converged when a correction solve failed or the system is still active.
__global__ void refine_finish_kernel(int n_sys, const int32_t* active, const CgSys* sys, double tol,
                                     int32_t* status) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sys; s += gridDim.x * blockDim.x) {
    if (status[s] == KMV_ENONFINITE) continue;
    if (sys[s].status != KMV_OK) {
      status[s] = sys[s].status;
    } else if (sys[s].rr <= tol * tol * sys[s].bb) {
      status[s] = KMV_OK;
    } else if (active[s]) {
      status[s] = KMV_ENOTCONV;
    }
  }
}

cudaError_t launch_refine_finish(int n_sys, const int32_t* active, const CgSys* sys, double tol, int32_t* status,
                                 cudaStream_t st) {
  refine_finish_kernel<<<(n_sys + 255) / 256, 256, 0, st>>>(n_sys, active, sys, tol, status);
  return cudaGetLastError();
}

// --- leapfrog (Sec. 3.2.2) ----------------------------------------------------

__global__ void lf_drift_kernel(int n, int n_theta, const double* theta, const double* pi,
                                const uint8_t* mask, double half_dt, double* theta_h) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int p = e % n_theta;
    const double f = (mask == nullptr || mask[p]) ? 1.0 : 0.0;
    theta_h[e] = theta[e] + half_dt * pi[e] * f;
  }
}

cudaError_t launch_lf_drift(int n_sys, int n_theta, const double* theta, const double* pi,
                            const uint8_t* mask, double half_dt, double* theta_h, cudaStream_t st) {
  const int n = n_sys * n_theta;
  lf_drift_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, n_theta, theta, pi, mask, half_dt, theta_h);
  return cudaGetLastError();
}

// V = [x, phi], G = [-x/2, phi/2] per row: L = -x^T A x / 2 + phi^T A phi / 2 (Eq. u).
__global__ void pack_force_kernel(int64_t n, const float* xs, const float* phi, float* Vf, float* Gf) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float xv = xs[e], pv = phi[e];
    Vf[2 * e] = xv;
    Vf[2 * e + 1] = pv;
    Gf[2 * e] = -0.5f * xv;
    Gf[2 * e + 1] = 0.5f * pv;
  }
}

cudaError_t launch_pack_force(int chains, int64_t n_total, const float* xsol, const float* phi,
                              float* Vf, float* Gf, cudaStream_t st) {
  const int64_t n = (int64_t)chains * n_total;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 32);
  if (n == 0) return cudaSuccess;
  pack_force_kernel<<<blocks, 256, 0, st>>>(n, xsol, phi, Vf, Gf);
  return cudaGetLastError();
}

__global__ void lf_kick_drift_kernel(int n, int n_theta, const double* theta_h, const double* grad,
                                     const double* mu, const double* prec, const uint8_t* mask,
                                     const int32_t* status, double dt, double* theta, double* pi) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int s = e / n_theta, p = e - s * n_theta;
    const double f = (mask == nullptr || mask[p]) ? 1.0 : 0.0;
    const double th = theta_h[e];
    if (status[s] != KMV_OK) {
      theta[e] = th;   // the caller rejects this trajectory
      continue;
    }
    double F = grad[e];
    if (prec) F += prec[p] * (th - mu[p]);
    const double pn = pi[e] - dt * F * f;
    pi[e] = pn;
    theta[e] = th + 0.5 * dt * pn * f;
  }
}

cudaError_t launch_lf_kick_drift(int n_sys, int n_theta, const double* theta_h, const double* grad,
                                 const double* mu, const double* prec, const uint8_t* mask,
                                 const int32_t* status, double dt, double* theta, double* pi,
                                 cudaStream_t st) {
  const int n = n_sys * n_theta;
  lf_kick_drift_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, n_theta, theta_h, grad, mu, prec, mask,
                                                        status, dt, theta, pi);
  return cudaGetLastError();
}

// --- energy (Eq. U) ---------------------------------------------------------------

// partial[item, c] = sum_i a[c*a_stride + i] * b[c*N + i] (b FP32 or FP64)
__global__ void dot_partial_kernel(DevLayout L, int chains, int64_t n_total, const float* a,
                                   int64_t a_stride, const float* b32, const double* b64,
                                   double* partial) {
  __shared__ double red[kTile / 32];
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int64_t i = L.item_row0[item] + threadIdx.x;
  double v = 0.0;
  if (i < L.offsets[b + 1]) {
    const int64_t bi = (int64_t)c * n_total + i;
    const double bv = b64 ? b64[bi] : (double)b32[bi];
    v = (double)a[(int64_t)c * a_stride + i] * bv;
  }
  const double t = block_sum(v, red);
  if (threadIdx.x == 0) partial[(int64_t)item * chains + c] = t;
}

cudaError_t launch_dot_partial(const DevLayout& L, int n_items, int chains, int64_t n_total,
                               const float* a, int64_t a_stride, const float* b32, const double* b64,
                               double* partial, cudaStream_t st) {
  dot_partial_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, a, a_stride, b32,
                                                              b64, partial);
  return cudaGetLastError();
}

__global__ void energy_finalize_kernel(DevLayout L, int n_inst, int chains, int n_theta,
                                       const double* theta, const double* pi, const double* mu,
                                       const double* prec, const double* partial_yx,
                                       const double* partial_pap, int32_t* status, double* H,
                                       double* terms) {
  const int n_sys = n_inst * chains;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sys; s += gridDim.x * blockDim.x) {
    const int b = s / chains, c = s - b * chains;
    const double yx = sys_sum(L, b, c, chains, partial_yx, 1, 0);
    const double pap = sys_sum(L, b, c, chains, partial_pap, 1, 0);
    double S = 0.0, kin = 0.0;
    for (int p = 0; p < n_theta; ++p) {
      const double th = theta[(int64_t)s * n_theta + p];
      if (prec) S += 0.5 * prec[p] * (th - mu[p]) * (th - mu[p]);
      if (pi) {
        const double v = pi[(int64_t)s * n_theta + p];
        kin += 0.5 * v * v;
      }
    }
    const double U = S + 0.5 * yx + 0.5 * pap;
    const double h = U + kin;
    H[s] = h;
    if (terms) {
      terms[3 * s + 0] = S;
      terms[3 * s + 1] = 0.5 * yx;
      terms[3 * s + 2] = 0.5 * pap;
    }
    if (!isfinite(h) && status[s] == KMV_OK) status[s] = KMV_ENONFINITE;
  }
}

cudaError_t launch_energy_finalize(const DevLayout& L, int n_inst, int chains, int n_theta,
                                   const double* theta, const double* pi, const double* mu,
                                   const double* prec, const double* partial_yx,
                                   const double* partial_pap, int32_t* status, double* H,
                                   double* terms, cudaStream_t st) {
  const int n_sys = n_inst * chains;
  energy_finalize_kernel<<<(n_sys + 127) / 128, 128, 0, st>>>(L, n_inst, chains, n_theta, theta, pi,
                                                              mu, prec, partial_yx, partial_pap,
                                                              status, H, terms);
  return cudaGetLastError();
}

// --- Metropolis test (Algorithm 1) ----------------------------------------------

// fail[s] = the first non-OK status seen (keeps an earlier failure)
__global__ void status_merge_kernel(int n, const int32_t* src, int32_t* dst) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
    if (dst[s] == KMV_OK && src[s] != KMV_OK) dst[s] = src[s];
}

cudaError_t launch_status_merge(int n, const int32_t* src, int32_t* dst, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  status_merge_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, src, dst);
  return cudaGetLastError();
}

// accept iff the trajectory's status is OK and log u <= H_old - H_new (the event
// u <= min(1, exp(H_old - H_new)) for u in (0, 1]); a rejected system gets theta_old
__global__ void accept_kernel(int n_sys, int n_theta, const double* H_old, const double* H_new, const double* u,
                              const int32_t* status, const double* theta_old, double* theta, int32_t* accepted) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sys; s += gridDim.x * blockDim.x) {
    const bool ok = (status == nullptr || status[s] == KMV_OK) && isfinite(H_new[s]) && isfinite(H_old[s]);
    const bool acc = ok && log(u[s]) <= H_old[s] - H_new[s];
    accepted[s] = acc ? 1 : 0;
    if (!acc)
      for (int p = 0; p < n_theta; ++p) theta[(int64_t)s * n_theta + p] = theta_old[(int64_t)s * n_theta + p];
  }
}

cudaError_t launch_accept(int n_sys, int n_theta, const double* H_old, const double* H_new, const double* u,
                          const int32_t* status, const double* theta_old, double* theta, int32_t* accepted,
                          cudaStream_t st) {
  if (n_sys == 0) return cudaSuccess;
  accept_kernel<<<(n_sys + 127) / 128, 128, 0, st>>>(n_sys, n_theta, H_old, H_new, u, status, theta_old, theta,
                                                     accepted);
  return cudaGetLastError();
}

}  // namespace kmv

// Multi-shift conjugate gradients: (A_s + lambda_{s,j} I) x_j = b for the m
// shifts j of every system s from ONE Krylov sequence per system.
//
// The shifted systems of the pole expansion (App. A, Sec. 3.1) share the
// right-hand side, and a Krylov space does not change when a multiple of I is
// added to the operator, so CG on the base system B = A + lambda_min I carries
// every shifted solve: the shifted residuals stay parallel to the base one,
// r_j = zeta_j r, and the shifted iterates follow from the base CG scalars by
// scalar recurrences in zeta (the multi-shift CG of Jegerlehner, and of
// Frommer, "BiCGStab(l) for families of shifted linear systems", 2003, in
// its CG form).  With sigma_j = lambda_j - lambda_min >= 0, per iteration k:
//   alpha = r.r / p.Bp,
//   zeta_j' = zeta_j zeta_j^- alpha^- / (alpha beta^- (zeta_j^- - zeta_j)
//                                         + zeta_j^- alpha^- (1 + sigma_j alpha)),
//   alpha_j = alpha zeta_j' / zeta_j,   x_j += alpha_j p_j,
//   r -= alpha Bp,   beta = r'.r' / r.r,   beta_j = beta (zeta_j' / zeta_j)^2,
//   p = r' + beta p,   p_j = zeta_j' r' + beta_j p_j,
// with zeta = zeta^- = 1, alpha^- = 1, beta^- = 0 at the start (the ^-
// quantities are those of the previous iteration).  One m = 1 product per
// iteration serves all m shifts.  A shift stops once its residual
// |zeta_j| |r| <= tol |b| (before zeta_j can underflow); a system stops when
// all its shifts have.  FP64 scalars, per-tile partial sums reduced in a fixed
// order.
#include <algorithm>

#include "cg_common.cuh"
#include "kmv_internal.cuh"
#include "simt_common.cuh"

namespace kmv {
namespace {

__device__ __forceinline__ double tile_sum(const DevLayout& L, int bi, int c, int chains, const double* partial) {
  double acc = 0.0;
  for (int it = L.inst_item0[bi]; it < L.inst_item0[bi + 1]; ++it) acc += partial[(int64_t)it * chains + c];
  return acc;
}

// r = p = b, x_j = 0, p_j = b; partials of b.b
__global__ void mscg_init_kernel(DevLayout L, int chains, int64_t n_total, int m, const float* b, float* r, float* p,
                                 float* xs, float* ps, double* partial) {
  __shared__ double red[kTile / 32];
  const int item = blockIdx.x, c = blockIdx.y;
  const int bi = L.item_inst[item];
  const int64_t i = L.item_row0[item] + threadIdx.x;
  double bb = 0.0;
  if (i < L.offsets[bi + 1]) {
    const int64_t v = (int64_t)c * n_total + i;
    const float bv = b[v];
    r[v] = bv;
    p[v] = bv;
    for (int j = 0; j < m; ++j) {
      xs[v * m + j] = 0.f;
      ps[v * m + j] = bv;
    }
    bb = (double)bv * bv;
  }
  const double t = block_sum(bb, red);
  if (threadIdx.x == 0) partial[(int64_t)item * chains + c] = t;
}

// Per system: |b|^2, the base shift (the smallest) and the shift offsets sigma_j.
__global__ void mscg_setup_kernel(DevLayout L, int n_inst, int chains, int m, const double* partial,
                                  const float* shifts, double tol, MscgSys* sys, MscgShift* sh, float* base_shift,
                                  int32_t* sys_active, int32_t* n_active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_inst * chains) return;
  const int bi = s / chains, c = s - bi * chains;
  const double bb = tile_sum(L, bi, c, chains, partial);
  float base = shifts[(int64_t)s * m];
  for (int j = 1; j < m; ++j) base = fminf(base, shifts[(int64_t)s * m + j]);
  base_shift[s] = base;
  const bool finite = isfinite(bb);
  const int act = (finite && bb > 0.0 && tol < 1.0) ? 1 : 0;
  MscgSys& y = sys[s];
  y.rr = bb;
  y.bb = bb;
  y.alpha = 0.0;
  y.beta = 0.0;
  y.alpha_prev = 1.0;
  y.beta_prev = 0.0;
  y.iters = 0;
  for (int j = 0; j < m; ++j) {
    MscgShift& k = sh[(int64_t)s * m + j];
    k.sigma = (double)shifts[(int64_t)s * m + j] - (double)base;
    k.zeta = k.zeta_prev = k.zeta_next = 1.0;
    k.alpha_s = k.beta_s = 0.0;
    k.iters = 0;
    k.status = finite ? KMV_OK : KMV_ENONFINITE;
    k.active = act;
  }
  sys_active[s] = act;
  if (act) atomicAdd(n_active, 1);
}

// alpha of the base CG and, per active shift, zeta_j' and alpha_j.
__global__ void mscg_alpha_kernel(DevLayout L, int n_inst, int chains, int m, const double* partial, MscgSys* sys,
                                  MscgShift* sh, int32_t* sys_active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_inst * chains || !sys_active[s]) return;
  const int bi = s / chains, c = s - bi * chains;
  if (!mscg_alpha_step(sys[s], sh + (int64_t)s * m, m, tile_sum(L, bi, c, chains, partial))) sys_active[s] = 0;
}

// x_j += alpha_j p_j (active shifts), r -= alpha Bp; partials of the new r.r
__global__ void mscg_update_xr_kernel(DevLayout L, int chains, int64_t n_total, int m, const MscgSys* sys,
                                      const MscgShift* sh, const int32_t* sys_active, float* r, const float* q,
                                      float* xs, const float* ps, double* partial) {
  __shared__ double red[kTile / 32];
  __shared__ float as[kMaxShifts];
  __shared__ int on[kMaxShifts];
  const int item = blockIdx.x, c = blockIdx.y;
  const int bi = L.item_inst[item];
  const int s = bi * chains + c;
  if (!sys_active[s]) return;
  if (threadIdx.x < m) {
    const MscgShift& k = sh[(int64_t)s * m + threadIdx.x];
    as[threadIdx.x] = (float)k.alpha_s;
    on[threadIdx.x] = k.active;
  }
  __syncthreads();
  const int64_t i = L.item_row0[item] + threadIdx.x;
  double rr = 0.0;
  if (i < L.offsets[bi + 1]) {
    const int64_t v = (int64_t)c * n_total + i;
    for (int j = 0; j < m; ++j)
      if (on[j]) xs[v * m + j] = fmaf(as[j], ps[v * m + j], xs[v * m + j]);
    const float rv = fmaf(-(float)sys[s].alpha, q[v], r[v]);
    r[v] = rv;
    rr = (double)rv * rv;
  }
  const double t = block_sum(rr, red);
  if (threadIdx.x == 0) partial[(int64_t)item * chains + c] = t;
}

// beta of the base CG; per active shift the stopping test and beta_j, then
// zeta advances; a system with no shift left stops.
__global__ void mscg_beta_kernel(DevLayout L, int n_inst, int chains, int m, const double* partial, double tol,
                                 int maxiter, MscgSys* sys, MscgShift* sh, int32_t* sys_active,
                                 int32_t* n_active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_inst * chains || !sys_active[s]) return;
  const int bi = s / chains, c = s - bi * chains;
  const bool any = mscg_beta_step(sys[s], sh + (int64_t)s * m, m, tile_sum(L, bi, c, chains, partial), tol, maxiter);
  sys_active[s] = any;
  if (any) atomicAdd(n_active, 1);
}

// mscg_update_xr, then, in the CTA that finishes each system last, the
// system's beta step (as mscg_beta_kernel); n_active is kept by decrements,
// so the iteration needs no separate beta launch or counter reset.
__global__ void mscg_update_xr_beta_kernel(DevLayout L, int chains, int64_t n_total, int m, MscgSys* sys,
                                           MscgShift* sh, int32_t* sys_active, float* r, const float* q, float* xs,
                                           const float* ps, double* partial, uint32_t* count, double tol,
                                           int maxiter, int32_t* n_active) {
  __shared__ double red[kTile / 32];
  __shared__ float as[kMaxShifts];
  __shared__ int on[kMaxShifts];
  const int item = blockIdx.x, c = blockIdx.y;
  const int bi = L.item_inst[item];
  const int s = bi * chains + c;
  if (!sys_active[s]) return;
  if (threadIdx.x < m) {
    const MscgShift& k = sh[(int64_t)s * m + threadIdx.x];
    as[threadIdx.x] = (float)k.alpha_s;
    on[threadIdx.x] = k.active;
  }
  __syncthreads();
  const int64_t i = L.item_row0[item] + threadIdx.x;
  double rr = 0.0;
  if (i < L.offsets[bi + 1]) {
    const int64_t v = (int64_t)c * n_total + i;
    for (int j = 0; j < m; ++j)
      if (on[j]) xs[v * m + j] = fmaf(as[j], ps[v * m + j], xs[v * m + j]);
    const float rv = fmaf(-(float)sys[s].alpha, q[v], r[v]);
    r[v] = rv;
    rr = (double)rv * rv;
  }
  const double t = block_sum(rr, red);
  if (threadIdx.x == 0) {
    partial[(int64_t)item * chains + c] = t;
    if (last_block_of_system(count, s, (uint32_t)(L.inst_item0[bi + 1] - L.inst_item0[bi])) &&
        !mscg_beta_step(sys[s], sh + (int64_t)s * m, m, tile_sum(L, bi, c, chains, partial), tol, maxiter)) {
      sys_active[s] = 0;
      atomicSub(n_active, 1);
    }
  }
}

// p = r + beta p; p_j = zeta_j r + beta_j p_j (active shifts)
__global__ void mscg_update_p_kernel(DevLayout L, int chains, int64_t n_total, int m, const MscgSys* sys,
                                     const MscgShift* sh, const int32_t* sys_active, const float* r, float* p,
                                     float* ps) {
  __shared__ float zs[kMaxShifts], bs[kMaxShifts];
  __shared__ int on[kMaxShifts];
  const int item = blockIdx.x, c = blockIdx.y;
  const int bi = L.item_inst[item];
  const int s = bi * chains + c;
  if (!sys_active[s]) return;
  if (threadIdx.x < m) {
    const MscgShift& k = sh[(int64_t)s * m + threadIdx.x];
    zs[threadIdx.x] = (float)k.zeta;
    bs[threadIdx.x] = (float)k.beta_s;
    on[threadIdx.x] = k.active;
  }
  __syncthreads();
  const int64_t i = L.item_row0[item] + threadIdx.x;
  if (i >= L.offsets[bi + 1]) return;
  const int64_t v = (int64_t)c * n_total + i;
  const float rv = r[v];
  p[v] = fmaf((float)sys[s].beta, p[v], rv);
  for (int j = 0; j < m; ++j)
    if (on[j]) ps[v * m + j] = fmaf(bs[j], ps[v * m + j], zs[j] * rv);
}

// Column results: status (KMV_ENOTCONV if still active) and iterations of every shift.
__global__ void mscg_finish_kernel(int64_t n_cols, const MscgShift* sh, int32_t* col_status, int32_t* col_iters) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_cols; e += (int64_t)gridDim.x * blockDim.x) {
    col_status[e] = sh[e].active ? KMV_ENOTCONV : sh[e].status;
    col_iters[e] = sh[e].iters;
  }
}

}  // namespace

cudaError_t launch_mscg_init(const DevLayout& L, int n_items, int chains, int64_t n_total, int m, const float* b,
                             float* r, float* p, float* xs, float* ps, double* partial, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  mscg_init_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, m, b, r, p, xs, ps, partial);
  return cudaGetLastError();
}

cudaError_t launch_mscg_setup(const DevLayout& L, int n_inst, int chains, int m, const double* partial,
                              const float* shifts, double tol, MscgSys* sys, MscgShift* sh, float* base_shift,
                              int32_t* sys_active, int32_t* n_active, cudaStream_t st) {
  const int n = n_inst * chains;
  mscg_setup_kernel<<<(n + 127) / 128, 128, 0, st>>>(L, n_inst, chains, m, partial, shifts, tol, sys, sh,
                                                     base_shift, sys_active, n_active);
  return cudaGetLastError();
}

cudaError_t launch_mscg_alpha(const DevLayout& L, int n_inst, int chains, int m, const double* partial, MscgSys* sys,
                              MscgShift* sh, int32_t* sys_active, cudaStream_t st) {
  const int n = n_inst * chains;
  mscg_alpha_kernel<<<(n + 127) / 128, 128, 0, st>>>(L, n_inst, chains, m, partial, sys, sh, sys_active);
  return cudaGetLastError();
}

cudaError_t launch_mscg_update_xr(const DevLayout& L, int n_items, int chains, int64_t n_total, int m,
                                  const MscgSys* sys, const MscgShift* sh, const int32_t* sys_active, float* r,
                                  const float* q, float* xs, const float* ps, double* partial, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  mscg_update_xr_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, m, sys, sh, sys_active, r, q,
                                                                 xs, ps, partial);
  return cudaGetLastError();
}

cudaError_t launch_mscg_beta(const DevLayout& L, int n_inst, int chains, int m, const double* partial, double tol,
                             int maxiter, MscgSys* sys, MscgShift* sh, int32_t* sys_active, int32_t* n_active,
                             cudaStream_t st) {
  const int n = n_inst * chains;
  mscg_beta_kernel<<<(n + 127) / 128, 128, 0, st>>>(L, n_inst, chains, m, partial, tol, maxiter, sys, sh,
                                                    sys_active, n_active);
  return cudaGetLastError();
}

cudaError_t launch_mscg_update_xr_beta(const DevLayout& L, int n_items, int chains, int64_t n_total, int m,
                                       MscgSys* sys, MscgShift* sh, int32_t* sys_active, float* r, const float* q,
                                       float* xs, const float* ps, double* partial, uint32_t* count, double tol,
                                       int maxiter, int32_t* n_active, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  mscg_update_xr_beta_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, m, sys, sh, sys_active, r,
                                                                      q, xs, ps, partial, count, tol, maxiter,
                                                                      n_active);
  return cudaGetLastError();
}

cudaError_t launch_mscg_update_p(const DevLayout& L, int n_items, int chains, int64_t n_total, int m,
                                 const MscgSys* sys, const MscgShift* sh, const int32_t* sys_active, const float* r,
                                 float* p, float* ps, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  mscg_update_p_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, m, sys, sh, sys_active, r, p,
                                                                ps);
  return cudaGetLastError();
}

cudaError_t launch_mscg_finish(int64_t n_cols, const MscgShift* sh, int32_t* col_status, int32_t* col_iters,
                               cudaStream_t st) {
  if (n_cols == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n_cols + 255) / 256, 1024);
  mscg_finish_kernel<<<blocks, 256, 0, st>>>(n_cols, sh, col_status, col_iters);
  return cudaGetLastError();
}

}  // namespace kmv

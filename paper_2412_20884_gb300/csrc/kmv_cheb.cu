// The non-stationary kernel family of Sec. 4:
//   K(x, x') = exp(C(x)) exp(C(x')) exp(-|x - x'|^2 / (2 l^2)),
//   C(x) = sum_t Theta_t T_t(x),  T_t(x) = T_{t_1}(x^1) ... T_{t_d}(x^d),
// with T_n the Chebyshev polynomials of the first kind and t running over
// [0, N_cheb)^d (row-major, t_1 slowest).  Every product kernel evaluates it as
// the stationary kernel (alpha = 1) between per-point amplitudes amp = exp(C):
// K = D K0 D, D = diag(amp), so the tiles stay those of the SE kernel.
//
// Gradient in Theta: dK_ij/dTheta_t = (T_t(x_i) + T_t(x_j)) K_ij, so for
// L = sum G o (A V)
//   dL/dTheta_t = sum_i T_t(x_i) h_i,   h_i = G_i . (K V)_i + V_i . (K G)_i,
// one reduction over the points given the two products K V and K G.
#include <algorithm>

#include "kmv_internal.cuh"
#include "simt_common.cuh"

namespace kmv {
namespace {

// T_0..T_{n-1} at x by the three-term recurrence.
__device__ __forceinline__ void cheb_values(double x, int n, double* t) {
  t[0] = 1.0;
  if (n > 1) t[1] = x;
  for (int k = 2; k < n; ++k) t[k] = 2.0 * x * t[k - 1] - t[k - 2];
}

// Basis value T_t(x_i) of flat multi-index t (row-major over d digits base n).
__device__ __forceinline__ double basis_at(const double* tv, int d, int n, int t) {
  double v = 1.0;
  for (int k = d - 1; k >= 0; --k) {
    const int dig = t % n;
    t /= n;
    v *= tv[k * kMaxChebOrder + dig];
  }
  return v;
}

// amp[c, i] = exp(C_{theta_s}(x_i)) for the rows of system s = (b, c)
__global__ void cheb_amp_kernel(DevLayout L, int chains, int64_t n_total, int d, int n_cheb, int n_coef,
                                int n_theta, const float* x, const double* theta, float* amp) {
  extern __shared__ double sm[];   // Theta of this system (n_coef) then per-thread T values
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int s = b * chains + c;
  const double* th = theta + (int64_t)s * n_theta;
  for (int t = threadIdx.x; t < n_coef; t += blockDim.x) sm[t] = th[t];
  __syncthreads();
  const int64_t i = L.item_row0[item] + threadIdx.x;
  if (i >= L.offsets[b + 1]) return;
  double acc = sm[0];   // N_cheb = 1: the constant term alone
  if (n_cheb > 1) {
    double tv[kMaxChebDims * kMaxChebOrder];
    for (int k = 0; k < d; ++k) cheb_values((double)x[i * d + k], n_cheb, tv + k * kMaxChebOrder);
    acc = 0.0;
    for (int t = 0; t < n_coef; ++t) acc += sm[t] * basis_at(tv, d, n_cheb, t);
  }
  amp[(int64_t)c * n_total + i] = (float)exp(acc);
}

// Internal stationary parameters [log alpha = 0, log l.., log sigma^2] per system.
__global__ void cheb_theta_kernel(int n_sys, int n_coef, int n_theta, int n_theta_int, const double* theta,
                                  double* theta_int) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_sys) return;
  const double* th = theta + (int64_t)s * n_theta;
  double* ti = theta_int + (int64_t)s * n_theta_int;
  ti[0] = 0.0;
  for (int k = 1; k < n_theta_int; ++k) ti[k] = th[n_coef + k - 1];
}

// Per (tile, chain): partial[t] = sum_i T_t(x_i) h_i over the tile's rows.
__global__ void cheb_grad_kernel(DevLayout L, int chains, int64_t n_total, int d, int n_cheb, int n_coef, int m,
                                 const float* x, const float* V, const float* G, const float* KV, const float* KG,
                                 const int32_t* sys_active, double* partial) {
  extern __shared__ double red[];   // [kTile / 32][n_coef]
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int s = b * chains + c;
  if (sys_active && !sys_active[s]) return;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  const bool valid = i < L.offsets[b + 1];
  double h = 0.0;
  double tv[kMaxChebDims * kMaxChebOrder];
  if (valid) {
    for (int q = 0; q < m; ++q) {
      const int64_t idx = ((int64_t)c * n_total + i) * m + q;
      h += (double)G[idx] * (double)KV[idx] + (double)V[idx] * (double)KG[idx];
    }
    if (n_cheb > 1)
      for (int k = 0; k < d; ++k) cheb_values((double)x[i * d + k], n_cheb, tv + k * kMaxChebOrder);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int t = 0; t < n_coef; ++t) {
    double v = valid ? (n_cheb > 1 ? h * basis_at(tv, d, n_cheb, t) : h) : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (l == 0) red[w * n_coef + t] = v;
  }
  __syncthreads();
  double* out = partial + ((int64_t)item * chains + c) * n_coef;
  for (int t = threadIdx.x; t < n_coef; t += blockDim.x) {
    double acc = 0.0;
    for (int u = 0; u < kTile / 32; ++u) acc += red[u * n_coef + t];
    out[t] = acc;
  }
}

// grad[s] = [sum over the instance's tiles of the Theta partials, the internal
// lengthscale and noise gradients]; tiles summed in a fixed order.
__global__ void cheb_grad_finalize_kernel(DevLayout L, int n_inst, int chains, int n_coef, int n_theta,
                                          int n_theta_int, const double* partial, const double* grad_int,
                                          const int32_t* sys_active, double* grad) {
  const int s = blockIdx.x;
  if (s >= n_inst * chains) return;
  if (sys_active && !sys_active[s]) return;
  const int b = s / chains, c = s - b * chains;
  double* g = grad + (int64_t)s * n_theta;
  for (int t = threadIdx.x; t < n_coef; t += blockDim.x) {
    double acc = 0.0;
    for (int it = L.inst_item0[b]; it < L.inst_item0[b + 1]; ++it)
      acc += partial[((int64_t)it * chains + c) * n_coef + t];
    g[t] = acc;
  }
  for (int k = 1 + threadIdx.x; k < n_theta_int; k += blockDim.x)
    g[n_coef + k - 1] = grad_int[(int64_t)s * n_theta_int + k];
}

}  // namespace

int cheb_n_coef(int n_cheb, int d) {
  int64_t v = 1;
  for (int k = 0; k < d; ++k) {
    v *= n_cheb;
    if (v > kMaxChebCoef) return -1;
  }
  return (int)v;
}

cudaError_t launch_cheb_prepare(const DevLayout& L, int n_items, int n_sys, int chains, int64_t n_total, int d,
                                int n_cheb, int n_coef, int n_theta, int n_theta_int, const float* x,
                                const double* theta, double* theta_int, float* amp, cudaStream_t st) {
  if (n_sys > 0)
    cheb_theta_kernel<<<(n_sys + 127) / 128, 128, 0, st>>>(n_sys, n_coef, n_theta, n_theta_int, theta, theta_int);
  if (n_items > 0)
    cheb_amp_kernel<<<dim3(n_items, chains), kTile, sizeof(double) * n_coef, st>>>(
        L, chains, n_total, d, n_cheb, n_coef, n_theta, x, theta, amp);
  return cudaGetLastError();
}

cudaError_t launch_cheb_grad(const DevLayout& L, int n_items, int n_inst, int chains, int64_t n_total, int d,
                             int n_cheb, int n_coef, int n_theta, int n_theta_int, int m, const float* x,
                             const float* V, const float* G, const float* KV, const float* KG,
                             const int32_t* sys_active, double* partial, const double* grad_int, double* grad,
                             cudaStream_t st) {
  if (n_items > 0) {
    const size_t smem = sizeof(double) * (kTile / 32) * n_coef;
    cheb_grad_kernel<<<dim3(n_items, chains), kTile, smem, st>>>(L, chains, n_total, d, n_cheb, n_coef, m, x, V, G,
                                                                 KV, KG, sys_active, partial);
  }
  const int n_sys = n_inst * chains;
  if (n_sys > 0)
    cheb_grad_finalize_kernel<<<n_sys, 128, 0, st>>>(L, n_inst, chains, n_coef, n_theta, n_theta_int, partial,
                                                     grad_int, sys_active, grad);
  return cudaGetLastError();
}

}  // namespace kmv

// The Gibbs draw of the auxiliary variable, phi = A^{-1/2} xi (Sec. 3.1), by
// the pole expansion of App. A: A^{-1/2} xi ~ sum_p w_p (A + lambda_p I)^{-1} xi.
// Device kernels of kmv_phi_refresh (kmv_api.cu): the spectral interval, the
// weights and shifts, and the weighted sum of the shifted solutions.
#include <algorithm>
#include <cmath>

#include "kmv_internal.cuh"
#include "simt_common.cuh"

namespace kmv {
namespace {

constexpr int kAgmMax = 24;

// Complete elliptic integral of the first kind, K(m) for parameter m in [0, 1),
// by the arithmetic-geometric mean: K(m) = pi / (2 AGM(1, sqrt(1 - m))).
__device__ double ellip_k(double m) {
  double a = 1.0, b = sqrt(1.0 - m);
  for (int n = 0; n < kAgmMax && fabs(a - b) > 1e-16 * a; ++n) {
    const double an = 0.5 * (a + b);
    b = sqrt(a * b);
    a = an;
  }
  return M_PI / (a + b);
}

// Jacobi elliptic functions sn, cn, dn of (u | m), m in [0, 1), by the
// descending AGM (Landen) scheme (Abramowitz & Stegun 16.4): with a_0 = 1,
// b_0 = sqrt(1 - m), c_0 = sqrt(m) and a_n = (a + b)/2, b_n = sqrt(a b),
// c_n = (a - b)/2 until c_N vanishes, phi_N = 2^N a_N u and
// phi_{n-1} = (phi_n + asin(c_n sin(phi_n) / a_n)) / 2; then sn = sin phi_0,
// cn = cos phi_0, dn = cos phi_0 / cos(phi_1 - phi_0).
__device__ void ellip_j(double u, double m, double& sn, double& cn, double& dn) {
  double a[kAgmMax + 1], c[kAgmMax + 1];
  a[0] = 1.0;
  c[0] = sqrt(m);
  double b = sqrt(1.0 - m);
  int n = 0;
  while (n < kAgmMax && fabs(c[n]) > 1e-17) {
    a[n + 1] = 0.5 * (a[n] + b);
    c[n + 1] = 0.5 * (a[n] - b);
    b = sqrt(a[n] * b);
    ++n;
  }
  double phi = ldexp(a[n] * u, n);
  double phi1 = phi;
  for (int k = n; k >= 1; --k) {
    phi1 = phi;
    phi = 0.5 * (phi + asin(c[k] * sin(phi) / a[k]));
  }
  sn = sin(phi);
  cn = cos(phi);
  dn = n == 0 ? 1.0 : cn / cos(phi1 - phi);
}

// bounds[s] = max over the rows of system s of (A 1)_i: the largest row sum,
// an upper bound on lambda_max(A) because K0 >= 0 entrywise.  One block per
// system; `slack` > 1 covers the rounding of the product.
__global__ void phi_bounds_kernel(DevLayout L, int chains, int64_t n_total, const float* Y, double slack,
                                  double* bounds) {
  __shared__ double red[32];
  const int s = blockIdx.x;
  const int b = s / chains, c = s - b * chains;
  double mx = 0.0;
  for (int64_t i = L.offsets[b] + threadIdx.x; i < L.offsets[b + 1]; i += blockDim.x)
    mx = fmax(mx, (double)Y[(int64_t)c * n_total + i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    bounds[s] = mx * slack;
  }
}

// Weights and shifts of App. A on [m, M] = [sigma_s^2, bounds[s]] (k^2 = m / M,
// K' = K(1 - k^2), u_p = (p + 1/2) K' / N_p, (sn, cn, dn) at (u_p | 1 - k^2)):
//   lambda_p = m (sn / cn)^2,  w_p = 2 K' sqrt(m) / (pi N_p) dn / cn^2.
// The shifts go to the column-shift table of the m = N_p product.  One thread per system.
__global__ void phi_poles_kernel(int n_sys, int n_theta, int n_poles, const double* theta, const double* bounds,
                                 float* shifts, double* weights, double* poles_out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_sys) return;
  const double* th = theta + (int64_t)s * n_theta;
  const double m_lo = exp(th[n_theta - 1]);
  const double M_hi = fmax(bounds[s], m_lo);
  const double mp = 1.0 - m_lo / M_hi;   // the complementary parameter 1 - k^2
  const double Kp = ellip_k(mp);
  const double scale = 2.0 * Kp * sqrt(m_lo) / (M_PI * n_poles);
  if (poles_out) {
    poles_out[(int64_t)s * (2 + 2 * n_poles) + 0] = m_lo;
    poles_out[(int64_t)s * (2 + 2 * n_poles) + 1] = M_hi;
  }
  for (int p = 0; p < n_poles; ++p) {
    double sn, cn, dn;
    ellip_j((p + 0.5) * Kp / n_poles, mp, sn, cn, dn);
    const double lam = m_lo * (sn / cn) * (sn / cn);
    const double wgt = scale * dn / (cn * cn);
    const int64_t sp = (int64_t)s * n_poles + p;
    shifts[sp] = (float)lam;
    weights[sp] = wgt;
    if (poles_out) {
      poles_out[(int64_t)s * (2 + 2 * n_poles) + 2 + p] = wgt;
      poles_out[(int64_t)s * (2 + 2 * n_poles) + 2 + n_poles + p] = lam;
    }
  }
}

__global__ void phi_fill_kernel(float* v, int64_t n, float val) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = val;
}

// phi[c, i] = sum_p w_{s p} x[c, i, p], summed in FP64 in the order p = 0, 1, ...
__global__ void phi_combine_kernel(DevLayout L, int chains, int n_poles, int64_t n_total, const double* weights,
                                   const float* x_p, float* phi) {
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int64_t i = L.item_row0[item] + threadIdx.x;
  if (i >= L.offsets[b + 1]) return;
  const int64_t s = (int64_t)b * chains + c;
  double acc = 0.0;
  for (int p = 0; p < n_poles; ++p)
    acc += weights[s * n_poles + p] * (double)x_p[((int64_t)c * n_total + i) * n_poles + p];
  phi[(int64_t)c * n_total + i] = (float)acc;
}

// A system's draw is KMV_OK only if all its shifted solves converged; its
// iteration count is the largest among them.
__global__ void phi_status_kernel(int n_sys, int n_poles, const int32_t* col_status, const int32_t* col_iters,
                                  int32_t* status, int32_t* iters) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_sys) return;
  int32_t st = KMV_OK, it = 0;
  for (int p = 0; p < n_poles; ++p) {
    const int32_t v = col_status[(int64_t)s * n_poles + p];
    if (v != KMV_OK && st == KMV_OK) st = v;
    it = max(it, col_iters[(int64_t)s * n_poles + p]);
  }
  status[s] = st;
  if (iters) iters[s] = it;
}

}  // namespace

cudaError_t launch_phi_fill(float* v, int64_t n, float val, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>(4096, (n + 255) / 256);
  phi_fill_kernel<<<blocks, 256, 0, st>>>(v, n, val);
  return cudaGetLastError();
}

cudaError_t launch_phi_bounds(DevLayout L, int n_sys, int chains, int64_t n_total, const float* Y, double slack,
                              double* bounds, cudaStream_t st) {
  phi_bounds_kernel<<<n_sys, 256, 0, st>>>(L, chains, n_total, Y, slack, bounds);
  return cudaGetLastError();
}

cudaError_t launch_phi_poles(int n_sys, int n_theta, int n_poles, const double* theta, const double* bounds,
                             float* shifts, double* weights, double* poles_out, cudaStream_t st) {
  phi_poles_kernel<<<(n_sys + 63) / 64, 64, 0, st>>>(n_sys, n_theta, n_poles, theta, bounds, shifts, weights,
                                                     poles_out);
  return cudaGetLastError();
}

cudaError_t launch_phi_combine(DevLayout L, int n_items, int chains, int n_poles, int64_t n_total,
                               const double* weights, const float* x_p, float* phi, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  phi_combine_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_poles, n_total, weights, x_p, phi);
  return cudaGetLastError();
}

cudaError_t launch_phi_status(int n_sys, int n_poles, const int32_t* col_status, const int32_t* col_iters,
                              int32_t* status, int32_t* iters, cudaStream_t st) {
  phi_status_kernel<<<(n_sys + 127) / 128, 128, 0, st>>>(n_sys, n_poles, col_status, col_iters, status, iters);
  return cudaGetLastError();
}

}  // namespace kmv

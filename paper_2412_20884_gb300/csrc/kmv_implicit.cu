// The implicit midpoint step of Sec. 3.2.3 (Eq. implicitsystem), solved by
// Anderson acceleration (App. B) of the fixed-point map of Eq. Phi on the
// stacked vector z = (theta, pi, x) of every system:
//   Phi(z) = (theta_0 + dt (pi_0 + pi)/2,
//             pi_0 - dt f_phi((theta_0 + theta)/2, x),
//             x + R (y - A((theta_0 + theta)/2) x)),
// with f_phi the frozen-x force of Sec. 3.2.1 (plus the prior's gradient) and
// R = (Nystrom P^{-1} or I) / c, c ~ rho(that A(theta_0)) from a power iteration.
// Anderson: the last k pairs (g_i = Phi(z_i), f_i = z_i - g_i) kept in a ring;
// alpha minimises |sum alpha_i f_i| subject to sum alpha_i = 1 (from the k x k
// Gram matrix of the f_i, FP64, updated by one row per iteration), and the next
// iterate is sum alpha_i g_i.  theta, pi (FP64) and x (FP32) form one vector;
// inner products are FP64, per-tile partials summed in a fixed order.
#include <algorithm>

#include "kmv_internal.cuh"
#include "simt_common.cuh"

namespace kmv {
namespace {

__device__ __forceinline__ double tsum(const DevLayout& L, int b, int c, int chains, const double* partial, int stride,
                                       int k) {
  double acc = 0.0;
  for (int it = L.inst_item0[b]; it < L.inst_item0[b + 1]; ++it) acc += partial[((int64_t)it * chains + c) * stride + k];
  return acc;
}

// theta_bar = (theta_0 + theta) / 2
__global__ void imp_mid_kernel(int n, const double* th0, const double* th, double* tb) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    tb[e] = 0.5 * (th0[e] + th[e]);
}

// r = y - q; partials of r.r and y.y
__global__ void imp_resid_kernel(DevLayout L, int chains, int64_t n_total, const float* y, const float* q,
                                 const int32_t* active, float* r, double* partial2) {
  __shared__ double red[kTile / 32];
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  if (!active[b * chains + c]) return;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  double rr = 0.0, yy = 0.0;
  if (i < L.offsets[b + 1]) {
    const int64_t v = (int64_t)c * n_total + i;
    const float rv = y[i] - q[v];
    r[v] = rv;
    rr = (double)rv * rv;
    yy = (double)y[i] * y[i];
  }
  const double t0 = block_sum(rr, red);
  const double t1 = block_sum(yy, red);
  if (threadIdx.x == 0) {
    partial2[((int64_t)item * chains + c) * 2] = t0;
    partial2[((int64_t)item * chains + c) * 2 + 1] = t1;
  }
}

// x part of Phi: g_x = x + z / c, f_x = x - g_x into ring slot `slot`; partials of
// <f_x, F_x[i]> for the stored slots i < cnt
__global__ void imp_x_kernel(DevLayout L, int chains, int64_t n_total, int k, int slot, int cnt, const float* x,
                             const float* z, const double* cscale, const int32_t* active, float* Gx, float* Fx,
                             double* partial) {
  __shared__ double red[kTile / 32];
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int s = b * chains + c;
  if (!active[s]) return;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  const bool valid = i < L.offsets[b + 1];
  const int64_t vec = (int64_t)chains * n_total;
  float f = 0.f;
  if (valid) {
    const int64_t v = (int64_t)c * n_total + i;
    const float step = (float)(1.0 / cscale[s]) * z[v];
    Gx[(int64_t)slot * vec + v] = x[v] + step;
    f = -step;
    Fx[(int64_t)slot * vec + v] = f;
  }
  for (int j = 0; j < cnt; ++j) {
    double t = 0.0;
    if (valid) t = (double)f * (double)Fx[(int64_t)j * vec + (int64_t)c * n_total + i];
    t = block_sum(t, red);
    if (threadIdx.x == 0) partial[((int64_t)item * chains + c) * k + j] = t;
  }
}

// theta, pi part of Phi, the new Gram row, the stopping test and the Anderson
// coefficients (one thread per system).  State per system: H (k x k Gram),
// alpha (k); ring slots of G_tp, F_tp (k x 2n).
__global__ void imp_aa_kernel(DevLayout L, int n_inst, int chains, int n, int k, int slot, int cnt,
                              const double* th0, const double* pi0, const double* th, const double* pi,
                              const double* grad, const double* mu, const double* prec, const uint8_t* mask, double dt,
                              const double* xpart, const double* rpart, double tol, int iter, int maxiter,
                              double* Gtp, double* Ftp, double* H, double* alpha, int32_t* active, int32_t* done_now,
                              int32_t* status, int32_t* iters, int32_t* n_active, double* best_rr,
                              int32_t* best_it) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_inst * chains) return;
  done_now[s] = 0;
  if (!active[s]) return;
  const int b = s / chains, c = s - b * chains;
  const int nn = 2 * n;
  double* g = Gtp + ((int64_t)slot * n_inst * chains + s) * nn;
  double* f = Ftp + ((int64_t)slot * n_inst * chains + s) * nn;
  double fm = 0.0, gm = 0.0;
  for (int p = 0; p < n; ++p) {
    const int64_t e = (int64_t)s * n + p;
    const double free = (mask == nullptr || mask[p]) ? 1.0 : 0.0;
    const double tb = 0.5 * (th0[e] + th[e]);
    double F = grad[e];
    if (prec) F += prec[p] * (tb - mu[p]);
    const double gt = th0[e] + dt * 0.5 * (pi0[e] + pi[e]) * free;
    const double gp = pi0[e] - dt * F * free;
    g[p] = gt;
    g[n + p] = gp;
    f[p] = th[e] - gt;
    f[n + p] = pi[e] - gp;
    fm = fmax(fm, fmax(fabs(f[p]), fabs(f[n + p])));
    gm = fmax(gm, fmax(fabs(gt), fabs(gp)));
  }
  // new Gram row: the theta-pi part plus the x part's tile partials
  double* Hs = H + (int64_t)s * k * k;
  for (int j = 0; j < cnt; ++j) {
    const double* fj = Ftp + ((int64_t)j * n_inst * chains + s) * nn;
    double v = tsum(L, b, c, chains, xpart, k, j);
    for (int p = 0; p < nn; ++p) v += f[p] * fj[p];
    Hs[slot * k + j] = v;
    Hs[j * k + slot] = v;
  }
  const double rr = tsum(L, b, c, chains, rpart, 2, 0), yy = tsum(L, b, c, chains, rpart, 2, 1);
  iters[s] = iter + 1;
  // the linear residual stops falling at the floor of the FP32 product (about
  // 2^-24 |A| |x|): below 1e-3 |y|, no halving for 8k iterations counts as
  // having reached it
  if (iter == 0 || rr < 0.25 * best_rr[s]) {
    best_rr[s] = rr;
    best_it[s] = iter;
  }
  const bool at_floor = iter - best_it[s] >= 8 * k && rr <= 1e-6 * yy;
  const bool finite = isfinite(rr) && isfinite(fm) && isfinite(Hs[slot * k + slot]);
  const bool conv = (rr <= tol * tol * yy || at_floor) && fm <= tol * (1.0 + gm);
  if (!finite || conv || iter + 1 >= maxiter) {
    status[s] = !finite ? KMV_ENONFINITE : (conv ? KMV_OK : KMV_ENOTCONV);
    active[s] = 0;
    done_now[s] = 1;   // the result is this iteration's Phi(z)
    return;
  }
  // alpha = H^{-1} 1 / (1^T H^{-1} 1), by Cholesky of H + ridge (newest slot alone on failure)
  double Hc[kMaxAA * kMaxAA], a[kMaxAA];
  double dmax = 0.0;
  for (int i = 0; i < cnt; ++i) dmax = fmax(dmax, Hs[i * k + i]);
  bool ok = dmax > 0.0;
  for (int i = 0; i < cnt && ok; ++i)
    for (int j = 0; j <= i; ++j) {
      double v = Hs[i * k + j] + (i == j ? 1e-13 * dmax : 0.0);
      for (int p = 0; p < j; ++p) v -= Hc[i * kMaxAA + p] * Hc[j * kMaxAA + p];
      if (i == j) {
        if (!(v > 0.0)) {
          ok = false;
          break;
        }
        Hc[i * kMaxAA + i] = sqrt(v);
      } else {
        Hc[i * kMaxAA + j] = v / Hc[j * kMaxAA + j];
      }
    }
  double* al = alpha + (int64_t)s * k;
  if (ok) {
    for (int i = 0; i < cnt; ++i) {   // forward: Hc u = 1
      double v = 1.0;
      for (int p = 0; p < i; ++p) v -= Hc[i * kMaxAA + p] * a[p];
      a[i] = v / Hc[i * kMaxAA + i];
    }
    for (int i = cnt - 1; i >= 0; --i) {   // back: Hc^T a = u
      double v = a[i];
      for (int p = i + 1; p < cnt; ++p) v -= Hc[p * kMaxAA + i] * a[p];
      a[i] = v / Hc[i * kMaxAA + i];
    }
    double sa = 0.0;
    for (int i = 0; i < cnt; ++i) sa += a[i];
    ok = sa != 0.0 && isfinite(sa);
    for (int i = 0; i < cnt && ok; ++i) al[i] = a[i] / sa;
  }
  if (!ok)
    for (int i = 0; i < cnt; ++i) al[i] = i == slot ? 1.0 : 0.0;
  atomicAdd(n_active, 1);
}

// theta, pi = sum_i alpha_i G_tp[i] (continuing systems) or the newest Phi (finished this iteration)
__global__ void imp_tp_mix_kernel(int n_sys, int n, int k, int slot, int cnt, const double* Gtp, const double* alpha,
                                  const int32_t* active, const int32_t* done_now, double* th, double* pi) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)n_sys * 2 * n) return;
  const int s = (int)(e / (2 * n)), p = (int)(e - (int64_t)s * 2 * n);
  if (!active[s] && !done_now[s]) return;
  double v;
  if (done_now[s]) {
    v = Gtp[((int64_t)slot * n_sys + s) * 2 * n + p];
  } else {
    v = 0.0;
    for (int i = 0; i < cnt; ++i) v += alpha[(int64_t)s * k + i] * Gtp[((int64_t)i * n_sys + s) * 2 * n + p];
  }
  if (p < n) th[(int64_t)s * n + p] = v;
  else pi[(int64_t)s * n + p - n] = v;
}

// x = sum_i alpha_i G_x[i] (continuing) or the newest Phi's x (finished this iteration)
__global__ void imp_x_mix_kernel(DevLayout L, int chains, int64_t n_total, int k, int slot, int cnt,
                                 const float* Gx, const double* alpha, const int32_t* active,
                                 const int32_t* done_now, float* x) {
  __shared__ double al[kMaxAA];
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int s = b * chains + c;
  if (!active[s] && !done_now[s]) return;
  if (threadIdx.x < cnt) al[threadIdx.x] = alpha[(int64_t)s * k + threadIdx.x];
  __syncthreads();
  const int64_t i = L.item_row0[item] + threadIdx.x;
  if (i >= L.offsets[b + 1]) return;
  const int64_t vec = (int64_t)chains * n_total, v = (int64_t)c * n_total + i;
  if (done_now[s]) {
    x[v] = Gx[(int64_t)slot * vec + v];
    return;
  }
  double acc = 0.0;
  for (int j = 0; j < cnt; ++j) acc += al[j] * (double)Gx[(int64_t)j * vec + v];
  x[v] = (float)acc;
}

// --- power iteration for c ~ rho(R~ A(theta_0)), R~ = P^{-1} or I -----------------------

// v = w / |w| per system (partial of w.w given), and the running estimate c = |w| / |v_prev| (|v_prev| = 1)
__global__ void imp_norm_kernel(DevLayout L, int n_inst, int chains, const double* partial, double* cscale) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_inst * chains) return;
  const int b = s / chains, c = s - b * chains;
  cscale[s] = sqrt(tsum(L, b, c, chains, partial, 1, 0));
}

__global__ void imp_scale_kernel(DevLayout L, int chains, int64_t n_total, const double* norm, const float* w,
                                 float* v, double* partial) {
  __shared__ double red[kTile / 32];
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int s = b * chains + c;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  double t = 0.0;
  if (i < L.offsets[b + 1]) {
    const int64_t e = (int64_t)c * n_total + i;
    const double nv = norm ? norm[s] : 0.0;
    const float val = norm ? (nv > 0.0 ? (float)(w[e] / nv) : 0.f) : w[e];
    v[e] = val;
    t = (double)val * val;
  }
  t = block_sum(t, red);
  if (threadIdx.x == 0) partial[(int64_t)item * chains + c] = t;
}

__global__ void imp_cfinal_kernel(int n_sys, double safety, double* cscale) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_sys) return;
  const double v = cscale[s] * safety;
  cscale[s] = (v > 0.0 && isfinite(v)) ? v : 1.0;
}

__global__ void fill_i32_kernel(int32_t* v, int n, int32_t val) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) v[e] = val;
}

}  // namespace

cudaError_t launch_fill_i32(int32_t* v, int n, int32_t val, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  fill_i32_kernel<<<(n + 255) / 256, 256, 0, st>>>(v, n, val);
  return cudaGetLastError();
}

cudaError_t launch_imp_mid(int n, const double* th0, const double* th, double* tb, cudaStream_t st) {
  imp_mid_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, th0, th, tb);
  return cudaGetLastError();
}

cudaError_t launch_imp_resid(const DevLayout& L, int n_items, int chains, int64_t n_total, const float* y,
                             const float* q, const int32_t* active, float* r, double* partial2, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  imp_resid_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, y, q, active, r, partial2);
  return cudaGetLastError();
}

cudaError_t launch_imp_x(const DevLayout& L, int n_items, int chains, int64_t n_total, int k, int slot, int cnt,
                         const float* x, const float* z, const double* cscale, const int32_t* active, float* Gx,
                         float* Fx, double* partial, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  imp_x_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, k, slot, cnt, x, z, cscale, active, Gx,
                                                        Fx, partial);
  return cudaGetLastError();
}

cudaError_t launch_imp_aa(const DevLayout& L, int n_inst, int chains, int n, int k, int slot, int cnt,
                          const double* th0, const double* pi0, const double* th, const double* pi,
                          const double* grad, const double* mu, const double* prec, const uint8_t* mask, double dt,
                          const double* xpart, const double* rpart, double tol, int iter, int maxiter, double* Gtp,
                          double* Ftp, double* H, double* alpha, int32_t* active, int32_t* done_now, int32_t* status,
                          int32_t* iters, int32_t* n_active, double* best_rr, int32_t* best_it, cudaStream_t st) {
  const int n_sys = n_inst * chains;
  imp_aa_kernel<<<(n_sys + 63) / 64, 64, 0, st>>>(L, n_inst, chains, n, k, slot, cnt, th0, pi0, th, pi, grad, mu,
                                                  prec, mask, dt, xpart, rpart, tol, iter, maxiter, Gtp, Ftp, H, alpha,
                                                  active, done_now, status, iters, n_active, best_rr, best_it);
  return cudaGetLastError();
}

cudaError_t launch_imp_mix(const DevLayout& L, int n_items, int n_inst, int chains, int64_t n_total, int n, int k,
                           int slot, int cnt, const double* Gtp, const float* Gx, const double* alpha,
                           const int32_t* active, const int32_t* done_now, double* th, double* pi, float* x,
                           cudaStream_t st) {
  const int n_sys = n_inst * chains;
  const int64_t e = (int64_t)n_sys * 2 * n;
  imp_tp_mix_kernel<<<(unsigned)((e + 255) / 256), 256, 0, st>>>(n_sys, n, k, slot, cnt, Gtp, alpha, active,
                                                                  done_now, th, pi);
  if (n_items > 0)
    imp_x_mix_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, k, slot, cnt, Gx, alpha, active,
                                                              done_now, x);
  return cudaGetLastError();
}

cudaError_t launch_imp_scale(const DevLayout& L, int n_items, int chains, int64_t n_total, const double* norm,
                             const float* w, float* v, double* partial, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  imp_scale_kernel<<<dim3(n_items, chains), kTile, 0, st>>>(L, chains, n_total, norm, w, v, partial);
  return cudaGetLastError();
}

cudaError_t launch_imp_norm(const DevLayout& L, int n_inst, int chains, const double* partial, double* cscale,
                            cudaStream_t st) {
  const int n = n_inst * chains;
  imp_norm_kernel<<<(n + 127) / 128, 128, 0, st>>>(L, n_inst, chains, partial, cscale);
  return cudaGetLastError();
}

cudaError_t launch_imp_cfinal(int n_sys, double safety, double* cscale, cudaStream_t st) {
  imp_cfinal_kernel<<<(n_sys + 127) / 128, 128, 0, st>>>(n_sys, safety, cscale);
  return cudaGetLastError();
}

}  // namespace kmv

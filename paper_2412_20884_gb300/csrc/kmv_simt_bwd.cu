// Plain FP32 adjoint of L = sum G o (A V) on the FMA/MUFU pipes.
//
// Same tiling as the forward kernel: a CTA owns kTile rows i of one system
// and one chunk of at most MP columns.  Per pair it recomputes K0_ij from
// direct differences and forms
//   W_ij = G_i . V_j             (this column chunk's share of (G V^T)_ij)
//   Q_ij = W_ij K0_ij
// and accumulates per row
//   sum_j Q_ij                                   -> d/dlog alpha
//   sum_j Q_ij (xh_ik - xh_jk)^2 (per k, or r^2) -> d/dlog l_k
//   sum_j K0_ij G_j                              -> dL/dV = A G
// With per-point amplitudes (Sec. 4) G and V enter as amp o G, amp o V.
// Because every dA/dtheta_p is symmetric, summing W_ij over all ordered
// pairs (i, j) gives the gradient without symmetrising W.  Per-CTA FP64
// partials go to a buffer that launch_grad_finalize reduces in a fixed order.
#include "simt_common.cuh"

namespace kmv {

template <int D, int MP, bool ARD>
__global__ void __launch_bounds__(kTile) bwd_simt_kernel(KmvArgs a) {
  constexpr int DA = D ? D : kMaxD;
  constexpr int DP = DA + 1;
  constexpr int DG = ARD ? DA : 1;
  const int dd = D ? D : a.d;
  const int item = blockIdx.x, c = blockIdx.y, z = blockIdx.z;
  const int b = a.L.item_inst[item];
  const int s = b * a.chains + c;
  if (a.sys_active && !a.sys_active[s]) return;

  __shared__ float sc[DA];
  __shared__ float sx[kJT * DP];
  __shared__ float sv[kJT * MP];
  __shared__ float sg[kJT * MP];
  __shared__ double red[kTile / 32];

  const int64_t j0 = a.L.offsets[b], j1 = a.L.offsets[b + 1];
  const int64_t r0 = a.L.item_row0[item];
  const int64_t i = r0 + threadIdx.x;
  const bool valid = i < j1;
  const double* th = a.theta + (int64_t)s * a.n_theta;
  load_scale(th, dd, a.ard, sc);
  const int c0 = z * MP;
  const int mc = min(MP, a.m - c0);
  const int64_t vbase = (int64_t)c * a.n_total;
  const bool want_gv = a.Y != nullptr;
  __syncthreads();

  float xi[DA];
  float gi[MP];
#pragma unroll
  for (int k = 0; k < DA; ++k) xi[k] = 0.f;
#pragma unroll
  for (int q = 0; q < MP; ++q) gi[q] = 0.f;
  const float amp_i = (a.amp && valid) ? a.amp[vbase + i] : 1.f;
  if (valid) {
    for (int k = 0; k < dd; ++k) xi[k] = a.x[i * dd + k] * sc[k];
#pragma unroll
    for (int q = 0; q < MP; ++q)
      if (q < mc) gi[q] = a.G[(vbase + i) * a.m + c0 + q] * amp_i;
  }

  float accq = 0.f, accg[DG], accv[MP];
  double accq64 = 0.0, accg64[DG], accv64[MP];
#pragma unroll
  for (int k = 0; k < DG; ++k) { accg[k] = 0.f; accg64[k] = 0.0; }
#pragma unroll
  for (int q = 0; q < MP; ++q) { accv[q] = 0.f; accv64[q] = 0.0; }

  int step = 0;
  for (int64_t jt = j0; jt < j1; jt += kJT, ++step) {
    const int nj = (int)min((int64_t)kJT, j1 - jt);
    for (int e = threadIdx.x; e < kJT * dd; e += kTile) {
      const int r = e / dd, k = e - r * dd;
      sx[r * DP + k] = r < nj ? a.x[(jt + r) * dd + k] * sc[k] : 0.f;
    }
    for (int e = threadIdx.x; e < kJT * MP; e += kTile) {
      const int r = e / MP, q = e - r * MP;
      const bool in = r < nj && q < mc;
      const int64_t idx = (vbase + jt + r) * a.m + c0 + q;
      const float am = (in && a.amp) ? a.amp[vbase + jt + r] : 1.f;
      sv[e] = in ? a.V[idx] * am : 0.f;
      sg[e] = (in && want_gv) ? a.G[idx] * am : 0.f;
    }
    __syncthreads();
#pragma unroll 2
    for (int jj = 0; jj < kJT; ++jj) {
      float r2 = 0.f;
      float df2[DG];
      if (D) {
#pragma unroll
        for (int k = 0; k < DA; ++k) {
          const float df = xi[k] - sx[jj * DP + k];
          const float t = df * df;
          if (ARD) df2[k] = t;
          r2 += t;
        }
      } else {
        for (int k = 0; k < dd; ++k) {
          const float df = xi[k] - sx[jj * DP + k];
          const float t = df * df;
          if (ARD) df2[k] = t;
          r2 += t;
        }
      }
      const float p = ex2_approx(-r2);
      float w = 0.f;
#pragma unroll
      for (int q = 0; q < MP; ++q) w = fmaf(gi[q], sv[jj * MP + q], w);
      const float Q = w * p;
      accq += Q;
      if (ARD) {
        if (D) {
#pragma unroll
          for (int k = 0; k < DG; ++k) accg[k] = fmaf(Q, df2[k], accg[k]);
        } else {
          for (int k = 0; k < dd; ++k) accg[k] = fmaf(Q, df2[k], accg[k]);
        }
      } else {
        accg[0] = fmaf(Q, r2, accg[0]);
      }
      if (want_gv) {
#pragma unroll
        for (int q = 0; q < MP; ++q) accv[q] = fmaf(p, sg[jj * MP + q], accv[q]);
      }
    }
    __syncthreads();
    if ((step + 1) % (kFoldTiles * kTile / kJT) == 0) {
      accq64 += (double)accq;
      accq = 0.f;
#pragma unroll
      for (int k = 0; k < DG; ++k) { accg64[k] += (double)accg[k]; accg[k] = 0.f; }
#pragma unroll
      for (int q = 0; q < MP; ++q) { accv64[q] += (double)accv[q]; accv[q] = 0.f; }
    }
  }
  accq64 += (double)accq;
#pragma unroll
  for (int k = 0; k < DG; ++k) accg64[k] += (double)accg[k];
#pragma unroll
  for (int q = 0; q < MP; ++q) accv64[q] += (double)accv[q];

  double noise = 0.0;
  if (valid) {
    const double alpha = exp(th[0]);
    const double s2 = exp(th[a.n_theta - 1]);
#pragma unroll
    for (int q = 0; q < MP; ++q) {
      if (q < mc) {
        const int64_t idx = (vbase + i) * a.m + c0 + q;
        const double g = (double)a.G[idx];
        noise += g * (double)a.V[idx];
        if (want_gv) a.Y[idx] = (float)(alpha * (double)amp_i * accv64[q] + s2 * g);
      }
    }
  }
  // Per-CTA partials: [sum Q, sum Q d2 (k entries or 1), sum G.V]
  double* out = a.grad_partial + (((int64_t)item * a.chains + c) * a.n_z + z) * a.n_theta;
  double t = block_sum(accq64, red);
  if (threadIdx.x == 0) out[0] = t;
  const int kk = a.n_theta - 2;
  for (int k = 0; k < kk; ++k) {
    double v = 0.0;
    if (ARD) {
      if (D) {
#pragma unroll
        for (int u = 0; u < DG; ++u) v = (u == k) ? accg64[u] : v;
      } else {
        v = accg64[k];
      }
    } else {
      v = accg64[0];
    }
    t = block_sum(v, red);
    if (threadIdx.x == 0) out[1 + k] = t;
  }
  t = block_sum(noise, red);
  if (threadIdx.x == 0) out[a.n_theta - 1] = t;
}

int backward_mp(int m) { return m >= kMaxMPBwd ? kMaxMPBwd : pow2ceil(m); }

template <int MP, bool ARD>
static cudaError_t bwd_by_d(const KmvArgs& a, dim3 grid, cudaStream_t st) {
  switch (a.d) {
    case 1: bwd_simt_kernel<1, MP, ARD><<<grid, kTile, 0, st>>>(a); break;
    case 2: bwd_simt_kernel<2, MP, ARD><<<grid, kTile, 0, st>>>(a); break;
    case 3: bwd_simt_kernel<3, MP, ARD><<<grid, kTile, 0, st>>>(a); break;
    case 4: bwd_simt_kernel<4, MP, ARD><<<grid, kTile, 0, st>>>(a); break;
    case 8: bwd_simt_kernel<8, MP, ARD><<<grid, kTile, 0, st>>>(a); break;
    case 16: bwd_simt_kernel<16, MP, ARD><<<grid, kTile, 0, st>>>(a); break;
    case 32: bwd_simt_kernel<32, MP, ARD><<<grid, kTile, 0, st>>>(a); break;
    default: bwd_simt_kernel<0, MP, ARD><<<grid, kTile, 0, st>>>(a); break;
  }
  return cudaGetLastError();
}

template <bool ARD>
static cudaError_t bwd_by_mp(const KmvArgs& a, dim3 grid, int mp, cudaStream_t st) {
  switch (mp) {
    case 1: return bwd_by_d<1, ARD>(a, grid, st);
    case 2: return bwd_by_d<2, ARD>(a, grid, st);
    case 4: return bwd_by_d<4, ARD>(a, grid, st);
    case 8: return bwd_by_d<8, ARD>(a, grid, st);
    case 16: return bwd_by_d<16, ARD>(a, grid, st);
    default: return bwd_by_d<32, ARD>(a, grid, st);
  }
}

cudaError_t launch_backward_simt(const KmvArgs& a, int n_items, cudaStream_t st) {
  const int mp = backward_mp(a.m);
  dim3 grid(n_items, a.chains, a.n_z);
  return a.ard ? bwd_by_mp<true>(a, grid, mp, st) : bwd_by_mp<false>(a, grid, mp, st);
}

// grad[s, p] = scale_p * sum over the instance's items and column chunks of partial[..., p]
__global__ void grad_finalize_kernel(DevLayout L, int n_inst, int chains, int n_theta, int n_z,
                                     const double* theta, const double* partial, double* grad) {
  const int s = blockIdx.x;
  const int b = s / chains, c = s - b * chains;
  const double* th = theta + (int64_t)s * n_theta;
  for (int p = threadIdx.x; p < n_theta; p += blockDim.x) {
    double acc = 0.0;
    for (int it = L.inst_item0[b]; it < L.inst_item0[b + 1]; ++it)
      for (int z = 0; z < n_z; ++z)
        acc += partial[(((int64_t)it * chains + c) * n_z + z) * n_theta + p];
    double scale;
    if (p == 0) scale = exp(th[0]);
    else if (p == n_theta - 1) scale = exp(th[n_theta - 1]);
    else scale = exp(th[0]) / kHalfLog2e;
    grad[(int64_t)s * n_theta + p] = scale * acc;
  }
}

cudaError_t launch_grad_finalize(const DevLayout& L, int n_inst, int chains, int n_theta, int ard,
                                 int d, int n_z, const double* theta, const double* partial,
                                 double* grad, cudaStream_t st) {
  (void)ard;
  (void)d;
  grad_finalize_kernel<<<n_inst * chains, 64, 0, st>>>(L, n_inst, chains, n_theta, n_z, theta,
                                                       partial, grad);
  return cudaGetLastError();
}

}  // namespace kmv

// Randomized Nystrom preconditioner (Frangella, Tropp and Udell), which the
// paper uses for its solves (Sec. 3.1, end; Sec. 3.2.3; Sec. 4), one per
// system s = (instance, chain):
//   Y = K Omega (one r-column product, no noise term), nu a small shift (below),
//   Y_nu = Y + nu Omega,  Omega^T Y_nu = L L^T,  B = Y_nu L^{-T} = U S W^T,
//   Lambda = max(S^2 - nu, 0),  K ~ U Lambda U^T,
// and for A = K + mu I the Woodbury form
//   P^{-1} = (lambda_r + mu) U (Lambda + mu)^{-1} U^T + (I - U U^T).
// B's SVD is taken through r x r matrices: with the three Gram matrices
// O^T Y, O^T O and Y^T Y (one pass over the rows), B^T B = L^{-1} Y_nu^T Y_nu
// L^{-T} = M, M = W S^2 W^T by cyclic Jacobi (FP64), and U = Y_nu T with
// T = L^{-T} W S^{-1}.  U is stored column by column, (chains, r, N_total),
// so that U^T r and U w read it with coalesced rows in the CG.
#include <algorithm>
#include <cmath>

#include "kmv_internal.cuh"
#include "simt_common.cuh"

namespace kmv {
namespace {

constexpr int kGB = 32;   // Gram / U block edge

// grams[s] = [O^T Y, O^T O, Y^T Y] (r x r each, FP64 products and sums), one
// 32 x 32 block per CTA, rows staged 32 at a time.  FP64 throughout: the columns
// of U = Y_nu T come out orthonormal only as far as these sums are exact, and
// the preconditioner stays positive definite only while that error is below
// (lambda_r + mu) / (lambda_1 + mu).
__global__ void __launch_bounds__(256) ny_gram_kernel(DevLayout L, int chains, int64_t n_total, int r, int nb,
                                                      const float* Om, const float* Y, double* grams) {
  __shared__ float ok[kGB][kGB + 1], ol[kGB][kGB + 1], yk[kGB][kGB + 1], yl[kGB][kGB + 1];
  const int s = blockIdx.x;
  const int b = s / chains, c = s - b * chains;
  const int kb = blockIdx.y / nb, lb = blockIdx.y - (blockIdx.y / nb) * nb;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  const int64_t j0 = L.offsets[b], j1 = L.offsets[b + 1];
  double a64[3][4] = {};
  for (int64_t i0 = j0; i0 < j1; i0 += kGB) {
    for (int e = threadIdx.x; e < kGB * kGB; e += 256) {
      const int rr = e / kGB, cc = e - rr * kGB;
      const int64_t i = i0 + rr;
      const bool in = i < j1;
      const int k = kb * kGB + cc, l = lb * kGB + cc;
      const int64_t base = ((int64_t)c * n_total + i) * r;
      ok[rr][cc] = (in && k < r) ? Om[base + k] : 0.f;
      yk[rr][cc] = (in && k < r) ? Y[base + k] : 0.f;
      ol[rr][cc] = (in && l < r) ? Om[base + l] : 0.f;
      yl[rr][cc] = (in && l < r) ? Y[base + l] : 0.f;
    }
    __syncthreads();
    for (int rr = 0; rr < kGB; ++rr) {
      const double oL = ol[rr][tx], yL = yl[rr][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int kk = ty + 8 * q;
        const double oK = ok[rr][kk], yK = yk[rr][kk];
        a64[0][q] = fma(oK, yL, a64[0][q]);
        a64[1][q] = fma(oK, oL, a64[1][q]);
        a64[2][q] = fma(yK, yL, a64[2][q]);
      }
    }
    __syncthreads();
  }
  const int l = lb * kGB + tx;
  for (int q = 0; q < 4; ++q) {
    const int k = kb * kGB + ty + 8 * q;
    if (k < r && l < r)
      for (int g = 0; g < 3; ++g) grams[(((int64_t)s * 3 + g) * r + k) * r + l] = a64[g][q];
  }
}

// W = sym(O^T Y) + nu O^T O (block-wide).
__device__ void fill_w(const double* OY, const double* OO, double nu, int r, double* W) {
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int k = e / r, l = e - k * r;
    W[e] = 0.5 * (OY[e] + OY[l * r + k]) + nu * OO[e];
  }
  __syncthreads();
}

// In-place Cholesky W = L L^T (lower triangle) by the whole block, right-looking;
// false (for every thread) at a pivot that is not positive and finite.
__device__ bool block_cholesky(double* W, int r, int* fail) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) *fail = 0;
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (tid == 0) {
      const double piv = W[j * r + j];
      if (!(piv > 0.0) || !isfinite(piv)) *fail = 1;
      else W[j * r + j] = sqrt(piv);
    }
    __syncthreads();
    if (*fail) break;
    const double djj = W[j * r + j];
    for (int i = j + 1 + tid; i < r; i += nt) W[i * r + j] /= djj;
    __syncthreads();
    const int m = r - j - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int i = j + 1 + e / m, k = j + 1 + e % m;
      if (k <= i) W[i * r + k] -= W[i * r + j] * W[k * r + j];
    }
    __syncthreads();
  }
  const bool ok = *fail == 0;
  __syncthreads();
  return ok;
}

// The r x r part per system (one CTA, FP64, matrices in the system's scratch):
// nu, W = sym(O^T Y) + nu O^T O = L L^T, M = L^{-1} G_nu L^{-T}, Jacobi M = V S2 V^T,
// sorted descending; lam = max(S2 - nu, 0); T = L^{-T} V S2^{-1/2} (FP32 out).
// A system whose Cholesky fails at every shift (or with fewer rows than r) gets
// lam = 0 and T = 0: its preconditioner is the identity.
__global__ void __launch_bounds__(256) ny_small_kernel(DevLayout L, int chains, int r, const double* grams,
                                                       double* scratch, double* T, double* lam, double* nu_out,
                                                       int32_t* status) {
  __shared__ double red[8];
  __shared__ double cs[kMaxRank / 2 + 1][2];
  __shared__ int pq[kMaxRank / 2 + 1][2];
  __shared__ int perm[kMaxRank];
  __shared__ int fail;
  const int s = blockIdx.x;
  const int b = s / chains;
  const int64_t nb_rows = L.offsets[b + 1] - L.offsets[b];
  const double* OY = grams + (int64_t)s * 3 * r * r;
  const double* OO = OY + r * r;
  const double* YY = OO + r * r;
  double* W = scratch + (int64_t)s * 4 * r * r;   // W, then L in its lower triangle
  double* G = W + r * r;                          // G_nu, then X = L^{-1} G_nu
  double* M = G + r * r;
  double* V = M + r * r;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int rr = r * r;

  // nu: Frangella et al.'s shift sqrt(N) eps |Y| for an orthonormal test matrix,
  // with eps the FP64 unit roundoff and |Y| / |Omega| (Frobenius) for the
  // Gaussian one; Y carries the FP32 product's rounding, so nu is raised by
  // decades until the Cholesky of W succeeds, then by one decade more.
  double ty = 0.0, to = 0.0;
  for (int k = tid; k < r; k += nt) {
    ty += YY[k * r + k];
    to += OO[k * r + k];
  }
  for (int o = 16; o > 0; o >>= 1) {
    ty += __shfl_down_sync(0xffffffffu, ty, o);
    to += __shfl_down_sync(0xffffffffu, to, o);
  }
  if ((tid & 31) == 0) {
    red[tid >> 5] = ty;
    cs[tid >> 5][0] = to;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < nt / 32; ++w) {
      a += red[w];
      c += cs[w][0];
    }
    red[0] = sqrt((double)nb_rows) * 0x1p-52 * sqrt(fmax(a, 0.0) / fmax(c, 1e-300));
    fail = (nb_rows < r || !(a > 0.0)) ? 1 : 0;
  }
  __syncthreads();
  double nu = red[0];
  bool ok = fail == 0;
  __syncthreads();
  if (ok) {
    ok = false;
    for (int attempt = 0; attempt < 18 && !ok; ++attempt) {
      if (attempt > 0) nu *= 10.0;
      fill_w(OY, OO, nu, r, W);
      ok = block_cholesky(W, r, &fail);
    }
    if (ok) {
      nu *= 10.0;
      fill_w(OY, OO, nu, r, W);
      ok = block_cholesky(W, r, &fail);
    }
  }
  if (!ok) {
    for (int e = tid; e < rr; e += nt) T[(int64_t)s * rr + e] = 0.0;
    for (int k = tid; k < r; k += nt) lam[(int64_t)s * r + k] = 0.0;
    if (tid == 0) {
      nu_out[s] = 0.0;
      status[s] = KMV_ENOTCONV;
    }
    return;
  }
  for (int e = tid; e < rr; e += nt) {
    const int k = e / r, l = e - k * r;
    const double oy = 0.5 * (OY[e] + OY[l * r + k]);
    G[e] = YY[e] + 2.0 * nu * oy + nu * nu * OO[e];
  }
  __syncthreads();
  // X = L^{-1} G_nu, column by column (one thread per column)
  for (int c = tid; c < r; c += nt)
    for (int i = 0; i < r; ++i) {
      double v = G[i * r + c];
      for (int p = 0; p < i; ++p) v -= W[i * r + p] * G[p * r + c];
      G[i * r + c] = v / W[i * r + i];
    }
  __syncthreads();
  // M = L^{-1} X^T: column c of M solves L m = (row c of X)
  for (int c = tid; c < r; c += nt)
    for (int i = 0; i < r; ++i) {
      double v = G[c * r + i];
      for (int p = 0; p < i; ++p) v -= W[i * r + p] * M[p * r + c];
      M[i * r + c] = v / W[i * r + i];
    }
  __syncthreads();
  for (int e = tid; e < rr; e += nt) {
    const int k = e / r, l = e - k * r;
    V[e] = k == l ? 1.0 : 0.0;
    if (k < l) {
      const double v = 0.5 * (M[e] + M[l * r + k]);
      M[e] = v;
      M[l * r + k] = v;
    }
  }
  __syncthreads();
  // cyclic Jacobi, round-robin pairs (r rounded up to even; index r is a bye)
  const int n2 = r + (r & 1), np = n2 / 2;
  for (int sweep = 0; sweep < 20; ++sweep) {
    for (int t = 0; t < n2 - 1; ++t) {
      for (int k = tid; k < np; k += nt) {
        int p, q;
        if (k == 0) {
          p = t;
          q = n2 - 1;
        } else {
          p = (t + k) % (n2 - 1);
          q = (t - k + n2 - 1) % (n2 - 1);
        }
        if (p > q) {
          const int u = p;
          p = q;
          q = u;
        }
        double c = 1.0, sn = 0.0;
        if (q < r) {
          const double apq = M[p * r + q];
          if (apq != 0.0) {
            const double th = (M[q * r + q] - M[p * r + p]) / (2.0 * apq);
            const double tt = copysign(1.0, th) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(tt * tt + 1.0);
            sn = tt * c;
          }
        }
        pq[k][0] = p;
        pq[k][1] = q;
        cs[k][0] = c;
        cs[k][1] = sn;
      }
      __syncthreads();
      for (int e = tid; e < np * r; e += nt) {   // rows p, q of J^T M
        const int k = e / r, col = e - k * r;
        const int p = pq[k][0], q = pq[k][1];
        if (q >= r) continue;
        const double c = cs[k][0], sn = cs[k][1];
        const double mp = M[p * r + col], mq = M[q * r + col];
        M[p * r + col] = c * mp - sn * mq;
        M[q * r + col] = sn * mp + c * mq;
      }
      __syncthreads();
      for (int e = tid; e < np * r; e += nt) {   // columns p, q of (J^T M) J and of V J
        const int k = e / r, row = e - k * r;
        const int p = pq[k][0], q = pq[k][1];
        if (q >= r) continue;
        const double c = cs[k][0], sn = cs[k][1];
        const double mp = M[row * r + p], mq = M[row * r + q];
        M[row * r + p] = c * mp - sn * mq;
        M[row * r + q] = sn * mp + c * mq;
        const double vp = V[row * r + p], vq = V[row * r + q];
        V[row * r + p] = c * vp - sn * vq;
        V[row * r + q] = sn * vp + c * vq;
      }
      __syncthreads();
    }
    // stop when the off-diagonal part is at rounding level
    double off = 0.0, all = 0.0;
    for (int e = tid; e < rr; e += nt) {
      const double v = M[e] * M[e];
      all += v;
      if (e / r != e % r) off += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      all += __shfl_down_sync(0xffffffffu, all, o);
    }
    __syncthreads();
    if ((tid & 31) == 0) {
      red[tid >> 5] = off;
    }
    __syncthreads();
    double off_t = 0.0;
    for (int w = 0; w < nt / 32; ++w) off_t += red[w];
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = all;
    __syncthreads();
    double all_t = 0.0;
    for (int w = 0; w < nt / 32; ++w) all_t += red[w];
    __syncthreads();
    if (off_t <= 1e-30 * all_t) break;
  }
  // eigenvalues in descending order
  if (tid == 0) {
    for (int k = 0; k < r; ++k) perm[k] = k;
    for (int a = 0; a < r; ++a) {
      int best = a;
      for (int k = a + 1; k < r; ++k)
        if (M[perm[k] * r + perm[k]] > M[perm[best] * r + perm[best]]) best = k;
      const int u = perm[a];
      perm[a] = perm[best];
      perm[best] = u;
    }
  }
  __syncthreads();
  // T[:, j] = L^{-T} V[:, perm_j] / sqrt(s2_j) (back substitution per column)
  for (int j = tid; j < r; j += nt) {
    const int pj = perm[j];
    const double s2 = M[pj * r + pj];
    lam[(int64_t)s * r + j] = fmax(s2 - nu, 0.0);
    double* t = G + j;   // column j of G as scratch (X is no longer needed), stride r
    for (int i = r - 1; i >= 0; --i) {
      double v = V[i * r + pj];
      for (int p = i + 1; p < r; ++p) v -= W[p * r + i] * t[p * r];
      t[i * r] = v / W[i * r + i];
    }
    const double inv = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
    for (int i = 0; i < r; ++i) T[(int64_t)s * rr + i * r + j] = t[i * r] * inv;
  }
  if (tid == 0) {
    nu_out[s] = nu;
    status[s] = KMV_OK;
  }
}

// U[c, j, i] = sum_l (Y[i, l] + nu_s Omega[i, l]) T_s[l, j] in FP64 (T's columns
// are scaled by 1/S, so the sum cancels), 16 columns j per CTA.
constexpr int kUB = 16;
__global__ void __launch_bounds__(kTile) ny_u_kernel(DevLayout L, int chains, int64_t n_total, int r,
                                                     const float* Om, const float* Y, const double* T,
                                                     const double* nu, float* U) {
  extern __shared__ double tcol[];   // r x 16 block of T
  const int item = blockIdx.x, c = blockIdx.y, jb = blockIdx.z;
  const int b = L.item_inst[item];
  const int s = b * chains + c;
  const double* Ts = T + (int64_t)s * r * r;
  for (int e = threadIdx.x; e < r * kUB; e += blockDim.x) {
    const int l = e / kUB, j = jb * kUB + e % kUB;
    tcol[e] = j < r ? Ts[l * r + j] : 0.0;
  }
  __syncthreads();
  const int64_t i = L.item_row0[item] + threadIdx.x;
  if (i >= L.offsets[b + 1]) return;
  const double nus = nu[s];
  const int64_t base = ((int64_t)c * n_total + i) * r;
  double acc[kUB];
#pragma unroll
  for (int j = 0; j < kUB; ++j) acc[j] = 0.0;
  for (int l = 0; l < r; ++l) {
    const double y = fma(nus, (double)Om[base + l], (double)Y[base + l]);
#pragma unroll
    for (int j = 0; j < kUB; ++j) acc[j] = fma(y, tcol[l * kUB + j], acc[j]);
  }
  for (int j = 0; j < kUB; ++j) {
    const int jj = jb * kUB + j;
    if (jj < r) U[((int64_t)c * r + jj) * n_total + i] = (float)acc[j];
  }
}

}  // namespace

cudaError_t launch_nystrom_finish(const DevLayout& L, int n_items, int n_inst, int chains, int64_t n_total, int r,
                                  const float* Om, const float* Y, double* grams, double* scratch, double* T,
                                  double* nu, float* U, double* lam, int32_t* status, cudaStream_t st) {
  const int n_sys = n_inst * chains;
  if (n_sys == 0) return cudaSuccess;
  const int nb = (r + kGB - 1) / kGB, nu_b = (r + kUB - 1) / kUB;
  ny_gram_kernel<<<dim3(n_sys, nb * nb), 256, 0, st>>>(L, chains, n_total, r, nb, Om, Y, grams);
  ny_small_kernel<<<n_sys, 256, 0, st>>>(L, chains, r, grams, scratch, T, lam, nu, status);
  if (n_items > 0)
    ny_u_kernel<<<dim3(n_items, chains, nu_b), kTile, sizeof(double) * r * kUB, st>>>(L, chains, n_total, r, Om, Y,
                                                                                      T, nu, U);
  return cudaGetLastError();
}

}  // namespace kmv

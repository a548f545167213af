// Plain FP32 forward product Y = A(theta) V on the FMA/MUFU pipes.
//
// One CTA of kTile threads owns kTile rows i of one (instance, chain) system
// and one chunk of at most MP columns of V.  It streams the instance's rows j
// through shared memory kJT at a time and, per pair, evaluates
//   K0_ij = 2^(-sum_k (xh_ik - xh_jk)^2),  xh = x sqrt(log2(e)/2) / l,
// from direct differences (no |x|^2 expansion, so no cancellation), then
// accumulates K0_ij V_j in FP32, folded into FP64 every 512 columns.
// Epilogue (Eq. kerdef): Y_i = alpha * acc_i + (sigma^2 + shift) V_i.  With
// per-point amplitudes (the kernel family of Sec. 4) V_j enters as amp_j V_j
// and acc_i is scaled by amp_i.
// When that grid would leave most SMs idle (small N), the J range is split
// into jsplit chunks of whole J tiles: each CTA writes its FP64 row sums, and
// a combine kernel adds the chunks in chunk order before the same epilogue.
#include <algorithm>

#include "cg_common.cuh"
#include "simt_common.cuh"

namespace kmv {

// Y, the optional FP64 rows and the per-item dot partial of rows i of one
// CTA from their FP64 sums acc64 (columns c0 .. c0 + mc - 1).
template <int MP>
__device__ __forceinline__ void fwd_simt_epilogue(const KmvArgs& a, int s, int item, int c, int c0, int mc,
                                                  int64_t i, bool valid, const double (&acc64)[MP], double* red) {
  const double* th = a.theta + (int64_t)s * a.n_theta;
  const int64_t vbase = (int64_t)c * a.n_total;
  const double alpha = exp(th[0]);
  const double s2 = exp(th[a.n_theta - 1]);
  double dot = 0.0;
  if (valid) {
    const double ai = a.amp ? alpha * (double)a.amp[vbase + i] : alpha;
#pragma unroll
    for (int q = 0; q < MP; ++q) {
      if (q < mc) {
        const int64_t idx = (vbase + i) * a.m + c0 + q;
        const double shift =
            a.col_shift ? (double)a.col_shift[(int64_t)s * a.col_shift_stride + c0 + q] : 0.0;
        const double vi = (double)a.V[idx];
        const double y = ai * acc64[q] + (a.no_diag ? 0.0 : (s2 + shift) * vi);
        a.Y[idx] = (float)y;
        if (a.Y64) a.Y64[idx] = y;
        dot += vi * y;
      }
    }
  }
  if (a.dot_partial) {
    const double t = block_sum(dot, red);
    if (threadIdx.x == 0) {
      a.dot_partial[(int64_t)item * a.chains + c] = t;
      // inside a (multi-shift) CG iteration (one column): the system's last
      // CTA takes its p.q (alpha) step
      const int b = a.L.item_inst[item];
      if ((a.cg_sys || a.ms_sys) &&
          last_block_of_system(a.cg_count, s, (uint32_t)(a.L.inst_item0[b + 1] - a.L.inst_item0[b]))) {
        const double pq = sys_sum(a.L, b, c, a.chains, a.dot_partial, 1, 0);
        const bool go = a.cg_sys ? cg_pq_step(a.cg_sys[s], pq)
                                 : mscg_alpha_step(a.ms_sys[s], a.ms_sh + (int64_t)s * a.ms_m, a.ms_m, pq);
        if (!go) {
          a.cg_active[s] = 0;
          atomicSub(a.cg_n_active, 1);
        }
      }
    }
  }
}

template <int D, int MP>
__global__ void __launch_bounds__(kTile) fwd_simt_kernel(KmvArgs a, int jsplit, double* jpart) {
  constexpr int DA = D ? D : kMaxD;
  constexpr int DP = DA + 1;  // padded row stride of the staged X tile
  const int dd = D ? D : a.d;
  const int item = blockIdx.x, c = blockIdx.y, z = blockIdx.z / jsplit, jc = blockIdx.z % jsplit;
  const int b = a.L.item_inst[item];
  const int s = b * a.chains + c;
  if (a.sys_active && !a.sys_active[s]) return;

  __shared__ float sc[DA];
  __shared__ float sx[kJT * DP];
  __shared__ float sv[kJT * MP];
  __shared__ double red[kTile / 32];

  const int64_t j0 = a.L.offsets[b], j1 = a.L.offsets[b + 1];
  const int64_t r0 = a.L.item_row0[item];
  const int64_t i = r0 + threadIdx.x;
  const bool valid = i < j1;
  const double* th = a.theta + (int64_t)s * a.n_theta;
  load_scale(th, dd, a.ard, sc);
  const int c0 = z * MP;
  const int mc = min(MP, a.m - c0);
  const int64_t vbase = (int64_t)c * a.n_total;  // row offset of chain c
  __syncthreads();

  float xi[DA];
#pragma unroll
  for (int k = 0; k < DA; ++k) xi[k] = 0.f;
  if (valid) {
    for (int k = 0; k < dd; ++k) xi[k] = a.x[i * dd + k] * sc[k];
  }
  float acc[MP];
  double acc64[MP];
#pragma unroll
  for (int q = 0; q < MP; ++q) { acc[q] = 0.f; acc64[q] = 0.0; }

  // this CTA's J tiles: chunk jc of jsplit (all of them when jsplit == 1)
  const int64_t n_jt = (j1 - j0 + kJT - 1) / kJT, per = (n_jt + jsplit - 1) / jsplit;
  const int64_t jb = j0 + jc * per * kJT, je = min(j1, jb + per * kJT);
  int step = 0;
  for (int64_t jt = jb; jt < je; jt += kJT, ++step) {
    const int nj = (int)min((int64_t)kJT, je - jt);
    for (int e = threadIdx.x; e < kJT * dd; e += kTile) {
      const int r = e / dd, k = e - r * dd;
      sx[r * DP + k] = r < nj ? a.x[(jt + r) * dd + k] * sc[k] : 0.f;
    }
    for (int e = threadIdx.x; e < kJT * MP; e += kTile) {
      const int r = e / MP, q = e - r * MP;
      sv[e] = (r < nj && q < mc) ? a.V[(vbase + jt + r) * a.m + c0 + q] * (a.amp ? a.amp[vbase + jt + r] : 1.f)
                                 : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < kJT; ++jj) {
      float r2 = 0.f;
      if (D) {
#pragma unroll
        for (int k = 0; k < DA; ++k) {
          const float df = xi[k] - sx[jj * DP + k];
          r2 = fmaf(df, df, r2);
        }
      } else {
        for (int k = 0; k < dd; ++k) {
          const float df = xi[k] - sx[jj * DP + k];
          r2 = fmaf(df, df, r2);
        }
      }
      const float p = ex2_approx(-r2);
#pragma unroll
      for (int q = 0; q < MP; ++q) acc[q] = fmaf(p, sv[jj * MP + q], acc[q]);
    }
    __syncthreads();
    if ((step + 1) % (kFoldTiles * kTile / kJT) == 0) {
#pragma unroll
      for (int q = 0; q < MP; ++q) { acc64[q] += (double)acc[q]; acc[q] = 0.f; }
    }
  }
#pragma unroll
  for (int q = 0; q < MP; ++q) acc64[q] += (double)acc[q];

  if (jsplit > 1) {
    // the chunk's row sums, (jsplit, chains, N_total, m); the combine kernel
    // adds the chunks in order and writes Y
    if (valid) {
#pragma unroll
      for (int q = 0; q < MP; ++q)
        if (q < mc) jpart[(((int64_t)jc * a.chains + c) * a.n_total + i) * a.m + c0 + q] = acc64[q];
    }
    return;
  }
  fwd_simt_epilogue<MP>(a, s, item, c, c0, mc, i, valid, acc64, red);
}

template <int MP>
__global__ void __launch_bounds__(kTile) fwd_simt_combine_kernel(KmvArgs a, int jsplit, const double* jpart) {
  __shared__ double red[kTile / 32];
  const int item = blockIdx.x, c = blockIdx.y, z = blockIdx.z;
  const int b = a.L.item_inst[item];
  const int s = b * a.chains + c;
  if (a.sys_active && !a.sys_active[s]) return;
  const int64_t i = a.L.item_row0[item] + threadIdx.x;
  const bool valid = i < a.L.offsets[b + 1];
  const int c0 = z * MP;
  const int mc = min(MP, a.m - c0);
  double acc64[MP];
#pragma unroll
  for (int q = 0; q < MP; ++q) {
    acc64[q] = 0.0;
    if (valid && q < mc)
      for (int jc = 0; jc < jsplit; ++jc) acc64[q] += jpart[(((int64_t)jc * a.chains + c) * a.n_total + i) * a.m + c0 + q];
  }
  fwd_simt_epilogue<MP>(a, s, item, c, c0, mc, i, valid, acc64, red);
}

int forward_mp(int m) { return m >= kMaxMPFwd ? kMaxMPFwd : pow2ceil(m); }

template <int MP>
static cudaError_t fwd_by_d(const KmvArgs& a, dim3 grid, int jsplit, double* jpart, cudaStream_t st) {
  switch (a.d) {
    case 1: fwd_simt_kernel<1, MP><<<grid, kTile, 0, st>>>(a, jsplit, jpart); break;
    case 2: fwd_simt_kernel<2, MP><<<grid, kTile, 0, st>>>(a, jsplit, jpart); break;
    case 3: fwd_simt_kernel<3, MP><<<grid, kTile, 0, st>>>(a, jsplit, jpart); break;
    case 4: fwd_simt_kernel<4, MP><<<grid, kTile, 0, st>>>(a, jsplit, jpart); break;
    case 8: fwd_simt_kernel<8, MP><<<grid, kTile, 0, st>>>(a, jsplit, jpart); break;
    case 16: fwd_simt_kernel<16, MP><<<grid, kTile, 0, st>>>(a, jsplit, jpart); break;
    case 32: fwd_simt_kernel<32, MP><<<grid, kTile, 0, st>>>(a, jsplit, jpart); break;
    default: fwd_simt_kernel<0, MP><<<grid, kTile, 0, st>>>(a, jsplit, jpart); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || jsplit == 1) return e;
  fwd_simt_combine_kernel<MP><<<dim3(grid.x, grid.y, grid.z / jsplit), kTile, 0, st>>>(a, jsplit, jpart);
  return cudaGetLastError();
}

int forward_jsplit(int n_items, int chains, int m, int64_t max_rows, int num_sms) {
  const int mp = forward_mp(m);
  const int64_t ctas = (int64_t)n_items * chains * ((m + mp - 1) / mp);
  if (ctas <= 0 || ctas >= 2 * (int64_t)num_sms) return 1;
  // about two CTAs per SM, and at least two J tiles per chunk
  int64_t js = std::min<int64_t>(kMaxJSplit, (2 * (int64_t)num_sms) / ctas);
  js = std::min<int64_t>(js, ((max_rows + kJT - 1) / kJT) / 2);
  return (int)std::max<int64_t>(1, js);
}

cudaError_t launch_forward_simt(const KmvArgs& a, int n_items, int jsplit, double* jpart, cudaStream_t st) {
  const int mp = forward_mp(a.m);
  const int nz = (a.m + mp - 1) / mp;
  if (jsplit < 1 || (jsplit > 1 && !jpart)) return cudaErrorInvalidValue;
  dim3 grid(n_items, a.chains, nz * jsplit);
  switch (mp) {
    case 1: return fwd_by_d<1>(a, grid, jsplit, jpart, st);
    case 2: return fwd_by_d<2>(a, grid, jsplit, jpart, st);
    case 4: return fwd_by_d<4>(a, grid, jsplit, jpart, st);
    case 8: return fwd_by_d<8>(a, grid, jsplit, jpart, st);
    case 16: return fwd_by_d<16>(a, grid, jsplit, jpart, st);
    case 32: return fwd_by_d<32>(a, grid, jsplit, jpart, st);
    default: return fwd_by_d<64>(a, grid, jsplit, jpart, st);
  }
}

}  // namespace kmv

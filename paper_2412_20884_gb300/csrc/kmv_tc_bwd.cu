// Tensor-core (tcgen05) adjoint of L = sum G o (A V), KMV_BF16_HILO.
//
// For every pair the gradient needs W_ij = G_i . V_j, K0_ij and, per input
// dimension, (xt_ik - xt_jk)^2.  Per 64-column half tile and I tile g an MMA
// issuer writes into TMEM
//   S_g = XA_g XB^T           the base-2 exponent (BF16 hi/lo, as in the forward)
//   W_g = GI_g VJ^T           GI rows [gh, gh, gl], VJ rows [vh, vl, vh] (BF16 hi/lo)
// the exp warpgroup forms Q = W 2^S and writes it to its own TMEM columns as
// F16, and the issuer then accumulates, per row i,
//   ACC_g += Q BG             BG columns for dimension k: 4k..4k+3 = [xh, xl, sh, sl]
//                             (F16 hi/lo of xt_jk and of xt_jk^2), column 60 = 1;
//                             giving R_ik = sum_j Q_ij xt_jk, T_ik = sum_j Q_ij xt_jk^2
//                             and q_i = sum_j Q_ij
// dL/dV = A G is the forward product with G in place of V (kmv_tc.cu).
// Every kFoldH half tiles the warpgroup folds, per row,
//   sum_j Q_ij (xt_ik - xt_jk)^2 = xt_ik^2 q_i - 2 xt_ik R_ik + T_ik
// into FP64 accumulators.  Because q, R and T are formed from the same rounded
// Q, the rounding of Q cancels in this combination exactly as in the exact
// sum; the hi/lo splits keep xt and xt^2 to ~22 bits.  G is scaled by a power
// of two so that |W| <= 2^14 (F16 range); the scale is removed at the end.
// Per-warp FP64 partials are reduced per system in a fixed order.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "kmv_tc.cuh"
#include "simt_common.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace kmv {
namespace {

constexpr int kFoldH = 64;   // half tiles (64 columns) per FP32 accumulation (4096 columns)
constexpr int kMaxDB = 15;   // 4 d gradient features + the ones column fit a 64-column accumulator
constexpr int kNB = 64;      // accumulator columns; the ones column is kQCol
constexpr int kQCol = 60;
constexpr int kGW = 16;      // doubles per (item, warp) gradient partial: [q, contrib_0..d-1]

struct TcBwdArgs {
  const int4* items;
  int n_items;
  int chains;
  int T_total;
  int KX, KG, NB, S, NA;
  int d, n_theta, ard;
  DevLayout L;
  TcTables T;
  const float* x;
  const double* theta;
  const uint8_t* XA;
  const uint8_t* XB;
  const uint8_t* GI;
  const uint8_t* VJ;
  const uint8_t* BG;
  double* gpart;   // (n_items, 8 warps, kGW)
  int m;
  const int32_t* sys_active;
  int* err;
};

// Power-of-two factor putting max_i |G_i| max_j |V_j| (a bound on |W|) just below 2^14.
__device__ __forceinline__ double w_scale(uint32_t gbits, uint32_t vbits) {
  const double p = (double)__uint_as_float(gbits) * (double)__uint_as_float(vbits);
  if (!(p > 0.0) || !isfinite(p)) return 1.0;
  int e;
  frexp(p, &e);
  return ldexp(1.0, 14 - e);
}

__device__ __forceinline__ float xt_of(float xv, float sc) {
  const float xh = xv * sc;
  const __half hi = __float2half_rn(xh);
  const __half lo = __float2half_rn(xh - __half2float(hi));
  return __half2float(hi) + __half2float(lo);
}

__device__ __forceinline__ void issue_ss(uint32_t d_tmem, uint64_t da, uint64_t db, int nk, uint32_t idesc) {
  for (int k = 0; k < nk; ++k) ptx::mma_ss(d_tmem, da + 16 * k, db + 16 * k, idesc, k > 0);
}
// K = 64 from TMEM (four K = 16 steps of 8 columns each).
__device__ __forceinline__ void issue_ts4(uint32_t d_tmem, uint32_t a_tmem, uint64_t db, uint32_t idesc,
                                          uint32_t acc) {
#pragma unroll
  for (int k = 0; k < 4; ++k) ptx::mma_ts(d_tmem, a_tmem + 8 * k, db + 16 * k, idesc, (k > 0) || acc);
}

// Warp roles: warps 0-7 two exp warpgroups (one per I tile), warp 8 MMA
// issuer of I tile 0 (and TMEM owner), warp 9 producer, warp 10 MMA issuer of
// I tile 1.  TMEM per I tile g (256 columns from 256 g): S [0,64), W [64,128),
// Q [128,160), ACC [192,256).  A half tile's S and W are released as soon as
// the warpgroup has loaded them, so the next half's S, W MMAs run during this
// half's exps; Q has its own columns, so the feature-sum MMAs of this half run
// during the next half's exps.
constexpr int kBwdThreads = 352;
constexpr int kBwdIssue1Warp = 10;

__global__ void __launch_bounds__(kBwdThreads, 1) tc_bwd_kernel(TcBwdArgs a) {
  using namespace ptx;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  const uint32_t XT = a.KX * 256u, GT = a.KG * 256u, BT = a.NB * 256u;
  const uint32_t ABUF = 2 * XT + 2 * GT;   // one A buffer: XA g0, XA g1, GI g0, GI g1
  const uint32_t STG = XT + GT + BT;       // one stage: XB, VJ, BG
  const int S = a.S, NA = a.NA;
  uint8_t* sA = smem;
  uint8_t* sS = sA + NA * ABUF;
  uint64_t* full = reinterpret_cast<uint64_t*>(sS + S * STG);
  uint64_t* empty = full + S;
  uint64_t* a_full = empty + S;
  uint64_t* a_empty = a_full + 2;
  uint64_t* s_full = a_empty + 2;    // [g] S, W of a half tile written
  uint64_t* s_free = s_full + 2;     // [g] S, W loaded into registers
  uint64_t* q_ready = s_free + 2;    // [g] Q written
  uint64_t* q_free = q_ready + 2;    // [g] Q consumed by the feature-sum MMAs
  uint64_t* o_ready = q_free + 2;
  uint64_t* o_free = o_ready + 2;
  uint64_t* done = o_free + 2;       // [g]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 2);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 2);
    }
    for (int g = 0; g < 2; ++g) {
      mbar_init(&a_full[g], 1);
      mbar_init(&a_empty[g], 2);
      mbar_init(&s_full[g], 1);
      mbar_init(&s_free[g], 128);
      mbar_init(&q_ready[g], 128);
      mbar_init(&q_free[g], 1);
      mbar_init(&o_ready[g], 1);
      mbar_init(&o_free[g], 128);
      mbar_init(&done[g], 1);
    }
    *abort = 0;
    fence_barrier_init();
  }
  if (warp == kMmaWarp) {
    tmem_alloc(tslot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;

  if (warp == kLoadWarp) {
    if (lane == 0) {
      // ------------------------------------------------------------ producer
      int it = 0, n_issued = 0, n_a_issued = 0;
      uint32_t stage = 0, sph = 0;
      bool aborted = false;
      for (int t = blockIdx.x; t < a.n_items && !aborted; t += gridDim.x) {
        const int4 item = a.items[t];
        if (a.sys_active && !a.sys_active[item.x]) continue;
        const int c = item.x % a.chains;
        const int ab = it % NA;
        if (!mbar_wait(&a_empty[ab], ((it / NA) & 1) ^ 1, abort, a.err, 21)) { aborted = true; break; }
        mbar_arrive_expect_tx(&a_full[ab], ABUF);
        const size_t ti = (size_t)c * a.T_total + item.y;
        uint8_t* ad = sA + ab * ABUF;
        bulk_g2s(ad, a.XA + ti * XT, 2 * XT, &a_full[ab]);
        bulk_g2s(ad + 2 * XT, a.GI + ti * GT, 2 * GT, &a_full[ab]);
        ++n_a_issued;
        for (int j = 0; j < item.w; ++j) {
          if (!mbar_wait(&empty[stage], sph ^ 1, abort, a.err, 22)) { aborted = true; break; }
          mbar_arrive_expect_tx(&full[stage], STG);
          const size_t tj = (size_t)c * a.T_total + item.z + j;
          uint8_t* sd = sS + stage * STG;
          bulk_g2s(sd, a.XB + tj * XT, XT, &full[stage]);
          bulk_g2s(sd + XT, a.VJ + tj * GT, GT, &full[stage]);
          bulk_g2s(sd + XT + GT, a.BG + tj * BT, BT, &full[stage]);
          ++n_issued;
          if (++stage == (uint32_t)S) { stage = 0; sph ^= 1; }
        }
        ++it;
      }
      if (aborted) {
        for (int k = 1; k <= min(n_issued, S); ++k) {
          const int idx = n_issued - k;
          mbar_drain(&full[idx % S], (idx / S) & 1, 500000000ull);
        }
        for (int k = 1; k <= min(n_a_issued, NA); ++k) {
          const int idx = n_a_issued - k;
          mbar_drain(&a_full[idx % NA], (idx / NA) & 1, 500000000ull);
        }
      }
    }
  } else if (warp == kMmaWarp || warp == kBwdIssue1Warp) {
    if (lane == 0) {
      // ------------------------------------------------------------ MMA issuer of I tile g
      // Half-tile stream k: S, W of half k once half k-1 is loaded by the
      // warpgroup, then the feature sums of half k-1 once its Q is written.
      const int g = warp == kMmaWarp ? 0 : 1;
      const uint32_t idSW = idesc_f16(128, 64, 1, 1);
      const uint32_t idA = idesc_f16(128, a.NB, 0, 0);
      const uint32_t sboX = a.KX * 16u, sboG = a.KG * 16u;
      const int nkx = a.KX / 16, nkg = a.KG / 16;
      const uint64_t dXA = sdesc(smem_u32(sA + g * XT), 128, sboX);
      const uint64_t dGI = sdesc(smem_u32(sA + 2 * XT + g * GT), 128, sboG);
      const uint64_t dXB = sdesc(smem_u32(sS), 128, sboX);
      const uint64_t dVJ = sdesc(smem_u32(sS + XT), 128, sboG);
      const uint64_t dBG = sdesc(smem_u32(sS + XT + GT), 128, 2048);
      const uint32_t tg = tbase + 256 * g;
      int it = 0;
      uint32_t stage = 0, sph = 0, sf_ph = 0, qr_ph = 0, of_ph = 0;
      bool opend = false;
      long long k = 0;
      bool have_prev = false;
      uint32_t prev_stage = 0;
      int prev_h = 0, prev_nH = 0;
      for (int t = blockIdx.x; t < a.n_items; t += gridDim.x) {
        const int4 item = a.items[t];
        if (a.sys_active && !a.sys_active[item.x]) continue;
        const int ab = it % NA;
        const int nH = 2 * item.w;
        for (int h = 0; h < nH; ++h, ++k) {
          const int hh = h & 1;
          // ---- S, W of half k
          if (k > 0) {
            if (!mbar_wait(&s_free[g], sf_ph, abort, a.err, 23)) goto mma_out;
            sf_ph ^= 1;
          }
          if (h == 0 && !mbar_wait(&a_full[ab], (it / NA) & 1, abort, a.err, 24)) goto mma_out;
          if (hh == 0 && !mbar_wait(&full[stage], sph, abort, a.err, 25)) goto mma_out;
          tc_fence_after();
          issue_ss(tg, sdesc_add(dXA, ab * ABUF), sdesc_add(dXB, stage * STG + hh * a.KX * 128u), nkx, idSW);
          issue_ss(tg + 64, sdesc_add(dGI, ab * ABUF), sdesc_add(dVJ, stage * STG + hh * a.KG * 128u), nkg, idSW);
          tc_commit(&s_full[g]);
          // the A buffer is read only by the S, W MMAs: release it after the
          // item's last half, before the next item waits for its own A buffer
          if (h == nH - 1) tc_commit(&a_empty[ab]);
          // ---- feature sums of half k-1
          if (have_prev) {
            if (!mbar_wait(&q_ready[g], qr_ph, abort, a.err, 26)) goto mma_out;
            qr_ph ^= 1;
            tc_fence_after();
            const uint32_t acc = (prev_h % kFoldH) != 0;
            if (!acc && opend) {
              if (!mbar_wait(&o_free[g], of_ph, abort, a.err, 27)) goto mma_out;
              of_ph ^= 1;
              opend = false;
              tc_fence_after();
            }
            issue_ts4(tg + 192, tg + 128, sdesc_add(dBG, prev_stage * STG + (prev_h & 1) * 1024u), idA, acc);
            tc_commit(&q_free[g]);
            if ((prev_h % kFoldH) == kFoldH - 1 || prev_h == prev_nH - 1) {
              tc_commit(&o_ready[g]);
              opend = true;
            }
            if (prev_h & 1) tc_commit(&empty[prev_stage]);
          }
          have_prev = true;
          prev_stage = stage;
          prev_h = h;
          prev_nH = nH;
          if (hh == 1) {
            if (++stage == (uint32_t)S) { stage = 0; sph ^= 1; }
          }
        }
        ++it;
      }
      if (have_prev) {
        if (!mbar_wait(&q_ready[g], qr_ph, abort, a.err, 26)) goto mma_out;
        tc_fence_after();
        const uint32_t acc = (prev_h % kFoldH) != 0;
        if (!acc && opend) {
          if (!mbar_wait(&o_free[g], of_ph, abort, a.err, 27)) goto mma_out;
          tc_fence_after();
        }
        issue_ts4(tg + 192, tg + 128, sdesc_add(dBG, prev_stage * STG + (prev_h & 1) * 1024u), idA, acc);
        tc_commit(&q_free[g]);
        tc_commit(&o_ready[g]);
        tc_commit(&empty[prev_stage]);
      }
    mma_out:
      tc_commit(&done[g]);
      mbar_drain(&done[g], 0, 500000000ull);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ exp warpgroups
    const int g = warp >> 2, w = warp & 3;
    const int row = 32 * w + lane;
    const uint32_t tl = tbase + 256 * g + (static_cast<uint32_t>(32 * w) << 16);
    const int d = a.d;
    uint32_t sph = 0, qf_ph = 0, oph = 0;
    long long k = 0;
    for (int t = blockIdx.x; t < a.n_items; t += gridDim.x) {
      const int4 item = a.items[t];
      if (a.sys_active && !a.sys_active[item.x]) continue;
      const int s = item.x, b = s / a.chains;
      const int64_t nb = a.L.offsets[b + 1] - a.L.offsets[b];
      const int64_t rl = (int64_t)(item.y + g - a.T.inst_tile0[b]) * 128 + row;
      const bool valid = rl < nb;
      const double* th = a.theta + (int64_t)s * a.n_theta;
      float xt[kMaxDB];
      double dacc[kMaxDB];
      double dq = 0.0;
#pragma unroll
      for (int kk = 0; kk < kMaxDB; ++kk) {
        xt[kk] = 0.f;
        dacc[kk] = 0.0;
      }
      if (valid) {
        const int64_t i = a.L.offsets[b] + rl;
#pragma unroll
        for (int kk = 0; kk < kMaxDB; ++kk) {
          if (kk < d) {
            const float sc = (float)(sqrt(2.0 * kHalfLog2e) * exp(-th[1 + (a.ard ? kk : 0)]));
            xt[kk] = xt_of(a.x[i * d + kk], sc);
          }
        }
      }
      const int nH = 2 * item.w;
      for (int h = 0; h < nH; ++h, ++k) {
        bool ok = mbar_wait(&s_full[g], sph, abort, a.err, 28);
        if (!__all_sync(0xffffffffu, ok)) goto exp_out;
        sph ^= 1;
        tc_fence_after();
        {
          uint32_t s0[32], w0[32], s1[32], w1[32], qq[32];
          tmem_ld32(tl, s0);
          tmem_ld32(tl + 64, w0);
          tmem_ld_wait();
          tmem_ld32(tl + 32, s1);
          tmem_ld32(tl + 96, w1);
#pragma unroll
          for (int q = 0; q < 16; ++q)
            qq[q] = pack_f16x2(ex2(__uint_as_float(s0[2 * q])) * __uint_as_float(w0[2 * q]),
                               ex2(__uint_as_float(s0[2 * q + 1])) * __uint_as_float(w0[2 * q + 1]));
          tmem_ld_wait();
          // S, W of this half are in registers: the tensor core may overwrite them
          tc_fence_before();
          mbar_arrive(&s_free[g]);
#pragma unroll
          for (int q = 0; q < 16; ++q)
            qq[16 + q] = pack_f16x2(ex2(__uint_as_float(s1[2 * q])) * __uint_as_float(w1[2 * q]),
                                    ex2(__uint_as_float(s1[2 * q + 1])) * __uint_as_float(w1[2 * q + 1]));
          if (k > 0) {
            // Q of the previous half must have been consumed
            ok = mbar_wait(&q_free[g], qf_ph, abort, a.err, 30);
            if (!__all_sync(0xffffffffu, ok)) goto exp_out;
            qf_ph ^= 1;
            tc_fence_after();
          }
          tmem_st32(tl + 128, qq);
        }
        tmem_st_wait();
        tc_fence_before();
        mbar_arrive(&q_ready[g]);
        if ((h % kFoldH) == kFoldH - 1 || h == nH - 1) {
          ok = mbar_wait(&o_ready[g], oph, abort, a.err, 29);
          if (!__all_sync(0xffffffffu, ok)) goto exp_out;
          oph ^= 1;
          tc_fence_after();
          uint32_t o3[16];
          tmem_ld16(tl + 192 + 48, o3);
          tmem_ld_wait();
          const float qs = __uint_as_float(o3[kQCol - 48]);
          dq += (double)qs;
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4) {
            if (4 * c4 < d) {
              uint32_t o[16];
              if (c4 == 3) {
#pragma unroll
                for (int q = 0; q < 16; ++q) o[q] = o3[q];
              } else {
                tmem_ld16(tl + 192 + 16 * c4, o);
                tmem_ld_wait();
              }
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int kk = 4 * c4 + u;
                if (kk < kMaxDB && kk < d) {
                  const float R = __uint_as_float(o[4 * u]) + __uint_as_float(o[4 * u + 1]);
                  const float T = __uint_as_float(o[4 * u + 2]) + __uint_as_float(o[4 * u + 3]);
                  const float x = xt[kk];
                  dacc[kk] += (double)fmaf(x, fmaf(x, qs, -2.f * R), T);
                }
              }
            }
          }
          tc_fence_before();
          mbar_arrive(&o_free[g]);
        }
      }
      // per-warp partial of this item: [q, contrib_0 .. contrib_{d-1}]
      {
        double* out = a.gpart + ((size_t)t * 8 + g * 4 + w) * kGW;
        double v = dq;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) out[0] = v;
#pragma unroll
        for (int kk = 0; kk < kMaxDB; ++kk) {
          if (kk < d) {
            double u = dacc[kk];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) u += __shfl_down_sync(0xffffffffu, u, o);
            if (lane == 0) out[1 + kk] = u;
          }
        }
      }
    }
  exp_out:;
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) tmem_dealloc(tbase, 512);
}

// max |G_i| and max |V_j| per system (row norms) and sum_i G_i . V_i.
__global__ void tc_bwd_norms_kernel(DevLayout L, int chains, int64_t n_total, const float* V, const float* G,
                                    int m, uint32_t* gmax, uint32_t* vmax, double* gvpart,
                                    const int32_t* sys_active) {
  __shared__ double red[kTile / 32];
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int s = b * chains + c;
  if (sys_active && !sys_active[s]) return;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  double gv = 0.0;
  if (i < L.offsets[b + 1]) {
    float g2 = 0.f, v2 = 0.f;
    for (int q = 0; q < m; ++q) {
      const int64_t idx = ((int64_t)c * n_total + i) * m + q;
      const float gq = G[idx], vq = V[idx];
      g2 = fmaf(gq, gq, g2);
      v2 = fmaf(vq, vq, v2);
      gv += (double)gq * (double)vq;
    }
    atomicMax(&gmax[s], __float_as_uint(sqrtf(g2)));
    atomicMax(&vmax[s], __float_as_uint(sqrtf(v2)));
  }
  const double t = block_sum(gv, red);
  if (threadIdx.x == 0) gvpart[(int64_t)item * chains + c] = t;
}

// GI, VJ and BG operand tiles of every (chain, padded tile).
__global__ void tc_prep_bwd_kernel(DevLayout L, TcTables T, int chains, int d, int ard, int n_theta, int m,
                                   int KG, int NB, int T_total, const float* x, const double* theta,
                                   const float* V, const float* G, int64_t n_total, const uint32_t* gmax,
                                   const uint32_t* vmax, const int32_t* sys_active, uint8_t* GI, uint8_t* VJ,
                                   uint8_t* BG, int* err) {
  const int t = blockIdx.x, c = blockIdx.y, r = threadIdx.x;
  const int b = T.tile_inst[t];
  const int s = b * chains + c;
  if (sys_active && !sys_active[s]) return;
  const int64_t nb = L.offsets[b + 1] - L.offsets[b];
  const int64_t rl = (int64_t)(t - T.inst_tile0[b]) * 128 + r;
  const bool valid = rl < nb;
  const int64_t i = L.offsets[b] + rl;
  const size_t tile = (size_t)c * T_total + t;
  __nv_bfloat16* gi = reinterpret_cast<__nv_bfloat16*>(GI + tile * (size_t)KG * 256);
  __nv_bfloat16* vj = reinterpret_cast<__nv_bfloat16*>(VJ + tile * (size_t)KG * 256);
  __half* bg = reinterpret_cast<__half*>(BG + tile * (size_t)NB * 256);
  const float gs = (float)w_scale(gmax[s], vmax[s]);
  const __nv_bfloat16 zb = __float2bfloat16_rn(0.f);
  for (int q = 0; q < KG; ++q) {
    __nv_bfloat16 gval = zb, vval = zb;
    if (valid && q < 3 * m) {
      const int col = q % m, part = q / m;
      const int64_t idx = ((int64_t)c * n_total + i) * m + col;
      const float gq = G[idx] * gs, vq = V[idx];
      const __nv_bfloat16 gh = __float2bfloat16_rn(gq), vh = __float2bfloat16_rn(vq);
      const __nv_bfloat16 gl = __float2bfloat16_rn(gq - __bfloat162float(gh));
      const __nv_bfloat16 vl = __float2bfloat16_rn(vq - __bfloat162float(vh));
      gval = part < 2 ? gh : gl;        // [gh, gh, gl]
      vval = part == 1 ? vl : vh;       // [vh, vl, vh]
    }
    gi[x_off(r, q, KG) / 2] = gval;
    vj[x_off(r, q, KG) / 2] = vval;
  }
  const double* th = theta + (int64_t)s * n_theta;
  for (int f = 0; f < NB; ++f) bg[t_off(f, r) / 2] = __float2half_rn(0.f);
  if (valid) {
    for (int k = 0; k < d; ++k) {
      const float sc = (float)(sqrt(2.0 * kHalfLog2e) * exp(-th[1 + (ard ? k : 0)]));
      const float xh = x[i * d + k] * sc;
      const __half hi = __float2half_rn(xh);
      const __half lo = __float2half_rn(xh - __half2float(hi));
      const float xtv = __half2float(hi) + __half2float(lo);
      if (!(fabsf(xtv) < 240.f)) atomicCAS(err, 0, 100);
      const float sq = xtv * xtv;
      const __half sh = __float2half_rn(sq);
      const __half sl = __float2half_rn(sq - __half2float(sh));
      bg[t_off(4 * k, r) / 2] = hi;
      bg[t_off(4 * k + 1, r) / 2] = lo;
      bg[t_off(4 * k + 2, r) / 2] = sh;
      bg[t_off(4 * k + 3, r) / 2] = sl;
    }
    bg[t_off(kQCol, r) / 2] = __float2half_rn(1.f);
  }
}

// grad[s, :] from the per-warp partials and sum_i G_i . V_i.  Each thread
// sums a fixed strided subset of the partials, then a fixed-shape tree joins
// the threads, so the result is bitwise reproducible.
constexpr int kFinThreads = 256;

__global__ void __launch_bounds__(kFinThreads) tc_bwd_finalize_kernel(
    DevLayout L, TcTables T, int chains, int n_theta, int ard, int d, const double* theta, const double* gpart,
    const double* gvpart, const uint32_t* gmax, const uint32_t* vmax, const int32_t* sys_active, const int* err,
    double* grad) {
  __shared__ double red[kFinThreads / 32][kGW + 1];
  const int s = blockIdx.x;
  if (sys_active && !sys_active[s]) return;
  const int b = s / chains, c = s - b * chains;
  const int64_t nb = L.offsets[b + 1] - L.offsets[b];
  const int npair = (int)((nb + 255) / 256);
  const int64_t n_rows = (int64_t)npair * T.inst_nk[b] * 8;   // (item, warp) partial rows
  const int64_t r0 = (int64_t)T.sys_item0[s] * 8;
  double acc[kGW + 1];
#pragma unroll
  for (int v = 0; v <= kGW; ++v) acc[v] = 0.0;
  for (int64_t r = threadIdx.x; r < n_rows; r += kFinThreads) {
    const double* row = gpart + (r0 + r) * kGW;
    for (int v = 0; v <= d; ++v) acc[v] += row[v];
  }
  for (int it = L.inst_item0[b] + threadIdx.x; it < L.inst_item0[b + 1]; it += kFinThreads)
    acc[kGW] += gvpart[(int64_t)it * chains + c];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int v = 0; v <= kGW; ++v) {
    double u = acc[v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u += __shfl_down_sync(0xffffffffu, u, o);
    if (lane == 0) red[w][v] = u;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double tot[kGW + 1];
  for (int v = 0; v <= kGW; ++v) {
    tot[v] = 0.0;
    for (int ww = 0; ww < kFinThreads / 32; ++ww) tot[v] += red[ww][v];
  }
  const double* th = theta + (int64_t)s * n_theta;
  const double alpha = exp(th[0]), s2 = exp(th[n_theta - 1]);
  const double gs = w_scale(gmax[s], vmax[s]);
  const bool bad = *err != 0;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  double* out = grad + (int64_t)s * n_theta;
  out[0] = bad ? nan : alpha * tot[0] / gs;
  const double ls = alpha / (gs * 2.0 * kHalfLog2e);
  if (ard) {
    for (int k = 0; k < d; ++k) out[1 + k] = bad ? nan : ls * tot[1 + k];
  } else {
    double sum = 0.0;
    for (int k = 0; k < d; ++k) sum += tot[1 + k];
    out[1] = bad ? nan : ls * sum;
  }
  out[n_theta - 1] = bad ? nan : s2 * tot[kGW];
}

}  // namespace

kmv_status tc_backward(kmv_handle h, const KmvArgs& a, double* grad, cudaStream_t st) {
  const Layout& L = h->layout;
  if (a.d > kMaxDB) return tc_fail(h, KMV_EUNSUPPORTED, "tensor-core adjoint supports d <= 15");
  TcState* S = tc_state(h);
  kmv_status stt = tc_build_plan(h, S, st);
  if (stt != KMV_OK) return stt;
  const int n_sys = L.n_inst * L.chains;
  const int KX = x_width(a.d), KG = round16(3 * a.m), NB = kNB;
  const size_t XT = (size_t)KX * 256, GT = (size_t)KG * 256, BT = (size_t)NB * 256;
  const size_t ABUF = 2 * XT + 2 * GT, STG = XT + GT + BT;
  const size_t fixed = 1024 + 512;
  int NA = 2;
  int stages = (int)std::min<size_t>(6, (kMaxSmem - fixed - NA * ABUF) / STG);
  if (kMaxSmem < fixed + NA * ABUF || stages < 2) {
    NA = 1;
    stages = kMaxSmem > fixed + ABUF ? (int)std::min<size_t>(6, (kMaxSmem - fixed - ABUF) / STG) : 0;
  }
  if (stages < 2) return tc_fail(h, KMV_EUNSUPPORTED, "tensor-core adjoint tiles do not fit in shared memory");
  const size_t smem = std::max(kMinSmem, fixed + NA * ABUF + stages * STG);

  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  const size_t tiles = (size_t)L.chains * S->T_total;
  const size_t o_xa = 0, o_xb = o_xa + al(tiles * XT), o_gi = o_xb + al(tiles * XT);
  const size_t o_vj = o_gi + al(tiles * GT), o_bg = o_vj + al(tiles * GT), o_mx = o_bg + al(tiles * BT);
  const size_t o_gv = o_mx + al(sizeof(uint32_t) * 2 * n_sys);
  const size_t o_gp = o_gv + al(sizeof(double) * (size_t)std::max(1, L.n_items) * L.chains);
  const size_t o_er = o_gp + al(sizeof(double) * (size_t)std::max(1, S->n_items) * 8 * kGW);
  stt = tc_ensure_buf(h, S, o_er + 256);
  if (stt != KMV_OK) return stt;
  uint8_t* base = static_cast<uint8_t*>(S->buf);
  uint32_t* gmax = reinterpret_cast<uint32_t*>(base + o_mx);
  uint32_t* vmax = gmax + n_sys;
  double* gvpart = reinterpret_cast<double*>(base + o_gv);
  double* gpart = reinterpret_cast<double*>(base + o_gp);
  int* err = reinterpret_cast<int*>(base + o_er);

  if (!S->bwd_attr_set) {
    if (cudaFuncSetAttribute(tc_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem) !=
        cudaSuccess)
      return tc_fail(h, KMV_ECUDA, "cudaFuncSetAttribute failed");
    S->bwd_attr_set = true;
  }
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(base + o_mx, 0, o_gv - o_mx, st) != cudaSuccess)
    return tc_fail(h, KMV_ECUDA, "memset failed");
  if (L.n_items > 0)
    tc_bwd_norms_kernel<<<dim3(L.n_items, L.chains), kTile, 0, st>>>(h->dev, L.chains, L.n_total, a.V, a.G, a.m,
                                                                     gmax, vmax, gvpart, a.sys_active);
  if (S->n_items > 0) {
    tc_launch_prep_x(h, S, a, KX, 2, base + o_xa, base + o_xb, st);
    tc_prep_bwd_kernel<<<dim3(S->T_total, L.chains), 128, 0, st>>>(
        h->dev, S->dev, L.chains, a.d, a.ard, a.n_theta, a.m, KG, NB, S->T_total, a.x, a.theta, a.V, a.G,
        L.n_total, gmax, vmax, a.sys_active, base + o_gi, base + o_vj, base + o_bg, err);
    TcBwdArgs ba;
    ba.items = S->d_items;
    ba.n_items = S->n_items;
    ba.chains = L.chains;
    ba.T_total = S->T_total;
    ba.KX = KX;
    ba.KG = KG;
    ba.NB = NB;
    ba.S = stages;
    ba.NA = NA;
    ba.d = a.d;
    ba.n_theta = a.n_theta;
    ba.ard = a.ard;
    ba.L = h->dev;
    ba.T = S->dev;
    ba.x = a.x;
    ba.theta = a.theta;
    ba.XA = base + o_xa;
    ba.XB = base + o_xb;
    ba.GI = base + o_gi;
    ba.VJ = base + o_vj;
    ba.BG = base + o_bg;
    ba.gpart = gpart;
    ba.m = a.m;
    ba.sys_active = a.sys_active;
    ba.err = err;
    const int grid = std::min(S->n_items, S->num_sms);
    tc_bwd_kernel<<<grid, kBwdThreads, smem, st>>>(ba);
  }
  tc_bwd_finalize_kernel<<<n_sys, kFinThreads, 0, st>>>(h->dev, S->dev, L.chains, a.n_theta, a.ard, a.d, a.theta, gpart,
                                                gvpart, gmax, vmax, a.sys_active, err, grad);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return tc_fail(h, KMV_ECUDA, cudaGetErrorString(e));
  if (a.Y != nullptr) {
    // dL/dV = A G: the forward product with G in place of V.  Stream order puts
    // it after the finalize above, so it may reuse the workspace.
    KmvArgs fa = a;
    fa.V = a.G;
    fa.col_shift = nullptr;
    fa.Y64 = nullptr;
    fa.dot_partial = nullptr;
    return tc_forward(h, fa, st);
  }
  return KMV_OK;
}

}  // namespace kmv

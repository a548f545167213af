// Tensor-core (tcgen05) adjoint of L = sum G o (A V), KMV_BF16_HILO.
//
// For every pair the gradient needs W_ij = G_i . V_j, K0_ij and, per input
// dimension, (xt_ik - xt_jk)^2.  Because K0 and (xt_i - xt_j)^2 are symmetric
// in (i, j), W may be replaced by W^s = (W + W^T) / 2, and then the sum over
// tile (J, I) equals the sum over tile (I, J): only the upper triangle of
// tiles (J >= I) is evaluated, off-diagonal tiles weighted twice.
//
// A work item is one I tile of one system against a range of J tiles; each J
// tile is split into two 64-column halves, half b for warpgroup b.  The two
// warpgroups run as independent pipelines, each with its own MMA issuer warp,
// TMEM buffers and accumulator, sharing only the operand stages.  For its half
// of a J tile, issuer b writes into TMEM
//   S = XA_I XB_J^T           the base-2 exponent from F16 hi/lo operands of the
//                             centred points (|dS| ~ 2^-24 |xh|^2); XA from TMEM
//   W = GI_I VJ_J^T           = G_i . V_j + V_i . G_j with GI rows
//                             [gh gh gl vh vh vl] (shared memory, once per item)
//                             and VJ rows [vh vl vh gh gl gh] (F16 hi/lo, G and V
//                             each scaled by a power of two)
// warpgroup b forms Q = W 2^S in FP32 (halved on the diagonal tile, and zero for
// i = j, whose (xt_i - xt_i)^2 is 0), splits it exactly into Q = Qh + Ql with Qh
// holding 11 significant bits (Veltkamp's splitting), stores both as F16, and
// issuer b accumulates, per row i,
//   ACC_b += Qh BG + Ql BG    BG: F16 hi/lo of xt_jk and xt_jk^2 and a ones column
//                             (the hi and lo parts in separate accumulator
//                             columns, or, for large d, in the same columns by
//                             splitting the K dimension), giving
//                             R_ik = sum_j Q_ij xt_jk, T_ik = sum_j Q_ij xt_jk^2, q_i = sum_j Q_ij
// Every kFoldOwn own halves warpgroup b folds its accumulator, per row,
//   sum_j Q_ij (xt_ik - xt_jk)^2 = xt_ik^2 q_i - 2 xt_ik R_ik + T_ik
// summed over the warp's rows into running sums of the item kept as FP32 pairs (TwoSum)
// (short accumulations: the tensor core's FP32 accumulator drops low bits at
// every K step), written as the warp's FP64 partial once per item.  The fold
// reads the accumulator right after
// waiting for the next Q's buffer, which implies its MMAs are complete, so it
// adds no wait of its own.  Because q, R and T are formed from the same Q, its
// rounding cancels in this combination exactly as in the exact sum; leaving
// out the diagonal keeps its large terms out of that cancellation, and its
// share of the alpha gradient, sum_i G_i . V_i, is added exactly in FP64.  The
// scales of G and V are removed at the end; per-warp FP64 partials are reduced
// per system in a fixed order.  G and V enter in blocks of columns and the
// feature sums in blocks of dimensions when the operands would not fit, one
// launch per block pair.
// dL/dV = A G is the forward product with G in place of V (kmv_tc.cu).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <climits>
#include <cmath>

#include "kmv_tc.cuh"
#include "simt_common.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace kmv {
namespace {

// Own halves (64 columns each) a warpgroup accumulates in TMEM before folding
// into its running sums: the tensor core's FP32 accumulation loses low bits at every K
// step (8 per half), so the sums are kept short (4 halves = 256 columns).
#ifndef KMV_BWD_FOLD_HALVES
#define KMV_BWD_FOLD_HALVES 4
#endif
constexpr int kFoldOwn = KMV_BWD_FOLD_HALVES;
static_assert(kFoldOwn >= 1, "at least one half per fold");
constexpr int kGW = 34;        // doubles per (item, warp) gradient partial: [q, contrib_0..d-1]
constexpr int kFoldWarps = 8;  // warps holding gradient partials (both warpgroups fold)

struct TcBwdArgs {
  const int4* items;
  int n_items;
  int chains;
  int T_total;
  int KX, KG, NB, S;
  // Feature-sum layout.  ksplit = 0: BG has NB = NACC features, per dimension
  // kk of the block the columns 4kk..4kk+3 = [xh, xl, sh, sl], and the ones
  // column qcol = 4 dk; the accumulator has the same NACC columns.  ksplit = 1:
  // BG has 2 NACC features, a hi block [xh_kk at kk, sh_kk at toff + kk, 1 at
  // qcol = 2 toff] and a lo block of the same layout at feature NACC; the
  // accumulator has NACC columns.
  int ksplit, NACC, toff, qcol;
  int k0, dk;   // dimensions [k0, k0 + dk) of this launch; q enters the alpha sum when k0 == 0
  int chunk;    // index of this launch's (column block, dimension block) (partials are per chunk)
  int d;
  const uint8_t* XA;
  const uint8_t* XB;
  const uint8_t* GI;
  const uint8_t* VJ;
  const uint8_t* BG;
  double* gpart;   // (chunks, n_items, 8 warps, kGW)
  const int32_t* sys_active;
  int* err;
};

// K = 64 from TMEM (four K = 16 steps of 8 columns each).
__device__ __forceinline__ void issue_ts4(uint32_t d_tmem, uint32_t a_tmem, uint64_t db, uint32_t idesc,
                                          uint32_t acc) {
#pragma unroll
  for (int k = 0; k < 4; ++k) ptx::mma_ts(d_tmem, a_tmem + 8 * k, db + 16 * k, idesc, (k > 0) || acc);
}

// Power-of-two factor putting a largest row norm just below 2^7, so that the
// F16 operands of G and V hold every element and |W^s| <= 2 2^7 2^7 = 2^15.
__device__ __forceinline__ double row_scale(uint32_t bits) {
  const double mx = (double)__uint_as_float(bits);
  if (!(mx > 0.0) || !isfinite(mx)) return 1.0;
  int e;
  frexp(mx, &e);
  return ldexp(1.0, 7 - e);
}

// Exact split q = hi + lo with hi holding 11 significant bits (Veltkamp's
// splitting with the factor 2^13 + 1), so that hi is an F16 value and lo
// carries the next 11 bits when stored as F16.  The rounded intrinsics keep
// the compiler from contracting the steps into FMAs, which would break the
// split.
__device__ __forceinline__ void split_q(float q, float& hi, float& lo) {
  const float t = __fmul_rn(q, 8193.f);
  hi = __fsub_rn(t, __fsub_rn(t, q));
  lo = __fsub_rn(q, hi);
}

// Warps: 0-7 the two warpgroups, 8 the issuer of warpgroup 0 (and TMEM owner),
// 9 the producer, 10 the issuer of warpgroup 1.  TMEM (512 columns):
//   S_b [128 b, +64), W_b [128 b + 64, +64), Qh_b [256 + 64 b, +32), Ql_b [+32, +32),
//   XA [384, 384 + KX/2) unless XS, ACC_b [512 - 2 NACC + b NACC, +NACC).
// Shared memory: the item's GI tile, the item's XA tile when XS (large d), and
// the stages [XB | VJ | BG] of the J tiles.
constexpr int kTsThreads = 352;
constexpr int kBwdIssue1Warp = 10;
constexpr int kMaxDT = 32;     // d <= 32
constexpr int kTsBarBytes = 512;                       // mbarriers, TMEM slot, abort flag
constexpr uint32_t kColXA = 384;

__host__ __device__ constexpr size_t al1k(size_t v) { return (v + 1023) & ~size_t(1023); }

// Sums v[u] over the warp's 32 lanes for u = 0..7 with 9 shuffles (halving
// the vector at offsets 16, 8, 4, then a butterfly over 2 and 1); lanes
// 4u .. 4u + 3 return the sum of v[u].
__device__ __forceinline__ float warp_reduce_scatter8(const float (&v)[8], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  float w4[4], w2[2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    w4[i] = (b4 ? v[i + 4] : v[i]) + __shfl_xor_sync(0xffffffffu, b4 ? v[i] : v[i + 4], 16);
#pragma unroll
  for (int i = 0; i < 2; ++i)
    w2[i] = (b3 ? w4[i + 2] : w4[i]) + __shfl_xor_sync(0xffffffffu, b3 ? w4[i] : w4[i + 2], 8);
  float z = (b2 ? w2[1] : w2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? w2[0] : w2[1], 4);
  z += __shfl_xor_sync(0xffffffffu, z, 2);
  z += __shfl_xor_sync(0xffffffffu, z, 1);
  return z;
}

template <bool XS>
__global__ void __launch_bounds__(kTsThreads, 1) tc_bwd_ts_kernel(TcBwdArgs a) {
  using namespace ptx;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  const uint32_t XT = a.KX * 256u, GT = a.KG * 256u, BT = a.NB * 256u;
  const uint32_t STG = XT + GT + BT;   // one stage: XB, VJ, BG of a J tile
  const int S = a.S;
  uint8_t* sGI = smem;                                            // the item's GI tile
  uint8_t* sXA = sGI + al1k(GT);                                  // XS: the item's XA tile
  uint8_t* sS = sXA + (XS ? al1k(XT) : 0u);                       // stages
  uint64_t* full = reinterpret_cast<uint64_t*>(sS + S * STG);
  uint64_t* empty = full + S;        // both issuers done with the stage (2 commits)
  uint64_t* a_ready = empty + S;     // XA of the item stored in TMEM (128 arrivals of warpgroup 0)
  uint64_t* seg = a_ready + 1;       // both warpgroups finished the previous item (256)
  uint64_t* sw_full = seg + 1;       // [b] S_b, W_b written
  uint64_t* s_free = sw_full + 2;    // [b] S_b, W_b loaded into registers
  uint64_t* q_ready = s_free + 2;    // [b] Q_b written
  uint64_t* q_free = q_ready + 2;    // [b] the feature sums of Q_b done
  uint64_t* done = q_free + 2;       // [issuer b]
  uint64_t* xa_full = done + 2;      // XS: XA tile landed
  uint64_t* xa_empty = xa_full + 1;  // XS: both issuers done with it (2 commits)
  uint64_t* gi_full = xa_empty + 1;  // GI tile landed
  uint64_t* gi_empty = gi_full + 1;  // both issuers done with it (2 commits)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(gi_empty + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 2);
    }
    mbar_init(a_ready, 128);
    mbar_init(seg, 256);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sw_full[b], 1);
      mbar_init(&s_free[b], 128);
      mbar_init(&q_ready[b], 128);
      mbar_init(&q_free[b], 1);
      mbar_init(&done[b], 1);
    }
    mbar_init(xa_full, 1);
    mbar_init(xa_empty, 2);
    mbar_init(gi_full, 1);
    mbar_init(gi_empty, 2);
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
    // ------------------------------------------------------------ producer
    const bool leader = elect_one();
    int n_issued = 0, n_items_done = 0;
    uint32_t stage = 0, sph = 0;
    bool aborted = false;
    for (int t = blockIdx.x; t < a.n_items && !aborted; t += gridDim.x) {
      const int4 item = a.items[t];
      if (a.sys_active && !a.sys_active[item.x]) continue;
      const int c = item.x % a.chains;
      const size_t ti = (size_t)c * a.T_total + item.y;
      const uint32_t ip = (uint32_t)(n_items_done & 1) ^ 1u;
      if (XS) {
        if (!warp_wait(xa_empty, ip, abort, a.err, 33)) { aborted = true; break; }
        if (leader) {
          mbar_arrive_expect_tx(xa_full, XT);
          bulk_g2s(sXA, a.XA + ti * XT, XT, xa_full);
        }
        __syncwarp();
      }
      if (!warp_wait(gi_empty, ip, abort, a.err, 35)) { aborted = true; break; }
      if (leader) {
        mbar_arrive_expect_tx(gi_full, GT);
        bulk_g2s(sGI, a.GI + ti * GT, GT, gi_full);
      }
      __syncwarp();
      ++n_items_done;
      for (int j = 0; j < item.w; ++j) {
        if (!warp_wait(&empty[stage], sph ^ 1, abort, a.err, 22)) { aborted = true; break; }
        if (leader) {
          mbar_arrive_expect_tx(&full[stage], STG);
          const size_t tj = (size_t)c * a.T_total + item.z + j;
          uint8_t* sd = sS + stage * STG;
          bulk_g2s(sd, a.XB + tj * XT, XT, &full[stage]);
          bulk_g2s(sd + XT, a.VJ + tj * GT, GT, &full[stage]);
          bulk_g2s(sd + XT + GT, a.BG + tj * BT, BT, &full[stage]);
        }
        __syncwarp();
        ++n_issued;
        if (++stage == (uint32_t)S) { stage = 0; sph ^= 1; }
      }
    }
    if (aborted) {
      // the copies already issued must land before the CTA exits
      for (int k = 1; k <= min(n_issued, S); ++k) {
        const int idx = n_issued - k;
        mbar_drain(&full[idx % S], (idx / S) & 1, 500000000ull);
      }
      if (n_items_done > 0) {
        if (XS) mbar_drain(xa_full, (uint32_t)(n_items_done - 1) & 1u, 500000000ull);
        mbar_drain(gi_full, (uint32_t)(n_items_done - 1) & 1u, 500000000ull);
      }
    }
  } else if (warp == kMmaWarp || warp == kBwdIssue1Warp) {
    // ------------------------------------------------------------ issuer of warpgroup b
    // Per own half k of the item: S(k), W(k) once the warpgroup has read
    // S(k-1), W(k-1); then the feature sums of Q(k-1) once it is written.
    const bool leader = elect_one();
    const int b = warp == kMmaWarp ? 0 : 1;
    const uint32_t idSW = idesc_f16(128, 64, 0, 0);
    const uint32_t idA = idesc_f16(128, a.NACC, 0, 0);
    const int nkx = a.KX / 16, nkg = a.KG / 16;
    const uint64_t dXA = sdesc(smem_u32(sXA), 128, a.KX * 16u);
    const uint64_t dGI = sdesc(smem_u32(sGI), 128, a.KG * 16u);
    const uint64_t dXB = sdesc(smem_u32(sS + b * a.KX * 128u), 128, a.KX * 16u);
    const uint64_t dVJ = sdesc(smem_u32(sS + XT + b * a.KG * 128u), 128, a.KG * 16u);
    const uint64_t dBG = sdesc(smem_u32(sS + XT + GT + b * 1024u), 128, 2048);
    const uint32_t lo_bytes = (uint32_t)a.NACC * 256u;   // ksplit: the lo block of BG
    const uint32_t tS = tbase + 128 * b, tW = tS + 64, tA = tbase + kColXA;
    const uint32_t tQh = tbase + 256 + 64 * b, tQl = tQh + 32;
    const uint32_t tACC = tbase + 512 - 2 * a.NACC + b * a.NACC;
    int it = 0;
    long long uses = 0, qr = 0;
    uint32_t stage = 0, sph = 0;
    // the feature sums of own half jj (stored in Q_b), from stage st_
    auto issue_acc = [&](uint32_t st_, int jj) -> bool {
      if (!warp_wait(&q_ready[b], (uint32_t)(qr & 1), abort, a.err, 26)) return false;
      ++qr;
      tc_fence_after();
      const uint32_t acc = (jj % kFoldOwn) != 0;
      const uint64_t dbg = sdesc_add(dBG, st_ * STG);
      if (leader) {
        issue_ts4(tACC, tQh, dbg, idA, acc);
        if (a.ksplit) issue_ts4(tACC, tQh, sdesc_add(dbg, lo_bytes), idA, 1);
        issue_ts4(tACC, tQl, dbg, idA, 1);
        tc_commit(&q_free[b]);
        tc_commit(&empty[st_]);
      }
      __syncwarp();
      return true;
    };
    for (int t = blockIdx.x; t < a.n_items; t += gridDim.x) {
      const int4 item = a.items[t];
      if (a.sys_active && !a.sys_active[item.x]) continue;
      const uint32_t ip = (uint32_t)(it & 1);
      if (!warp_wait(XS ? xa_full : a_ready, ip, abort, a.err, XS ? 34 : 31)) goto sw_out;
      if (!warp_wait(gi_full, ip, abort, a.err, 36)) goto sw_out;
      ++it;
      uint32_t prev_stage = 0;
      for (int j = 0; j < item.w; ++j) {
        if (uses > 0 && !warp_wait(&s_free[b], (uint32_t)((uses - 1) & 1), abort, a.err, 23)) goto sw_out;
        if (!warp_wait(&full[stage], sph, abort, a.err, 25)) goto sw_out;
        tc_fence_after();
        // operands computed by the whole warp (warp-uniform), issued by the leader
        const uint64_t db = sdesc_add(dXB, stage * STG);
        const uint64_t dv = sdesc_add(dVJ, stage * STG);
        if (leader) {
#pragma unroll
          for (int q = 0; q < kMaxKX / 16; ++q) {
            if (q < nkx) {
              if (XS)
                mma_ss(tS, dXA + 16 * q, db + 16 * q, idSW, q > 0);
              else
                mma_ts(tS, tA + 8 * q, db + 16 * q, idSW, q > 0);
            }
          }
#pragma unroll 4
          for (int q = 0; q < nkg; ++q) mma_ss(tW, dGI + 16 * q, dv + 16 * q, idSW, q > 0);
          tc_commit(&sw_full[b]);
          // the item's XA and GI tiles are released after its last S, W products
          if (j == item.w - 1) {
            tc_commit(gi_empty);
            if (XS) tc_commit(xa_empty);
          }
        }
        __syncwarp();
        ++uses;
        if (j > 0 && !issue_acc(prev_stage, j - 1)) goto sw_out;
        prev_stage = stage;
        if (++stage == (uint32_t)S) { stage = 0; sph ^= 1; }
      }
      if (item.w > 0 && !issue_acc(prev_stage, item.w - 1)) goto sw_out;
    }
  sw_out:
    if (leader) tc_commit(&done[b]);
    __syncwarp();
    mbar_drain(&done[b], 0, 500000000ull);
  } else {
    // ------------------------------------------------------------ warpgroups
    const int b = warp >> 2, w = warp & 3;
    const int row = 32 * w + lane;
    const uint32_t lofs = static_cast<uint32_t>(32 * w) << 16;
    const uint32_t tS = tbase + lofs + 128 * b, tQh = tbase + lofs + 256 + 64 * b;
    const uint32_t tQl = tQh + 32;
    const uint32_t tACC = tbase + lofs + 512 - 2 * a.NACC + b * a.NACC;
    const int d = a.d, dk = a.dk, k0 = a.k0;
    const int qc = a.qcol;
    long long uses = 0, qf = 0;
    int u = 0;
    for (int t = blockIdx.x; t < a.n_items; t += gridDim.x) {
      const int4 item = a.items[t];
      if (a.sys_active && !a.sys_active[item.x]) continue;
      const int c = item.x % a.chains;
      const size_t ti = (size_t)c * a.T_total + item.y;
      if (u > 0) {
        // both warpgroups are done with the previous item (its last products
        // and folds): nothing reads the TMEM XA rows any more
        mbar_arrive(seg);
        const bool ok = mbar_wait(seg, (uint32_t)(u - 1) & 1u, abort, a.err, 32);
        if (!__all_sync(0xffffffffu, ok)) goto exp_out;
      }
      ++u;
      if (!XS && b == 0) {
        // warpgroup 0 stores the item's XA rows into TMEM
        const uint8_t* src = a.XA + ti * XT + (row >> 3) * (a.KX * 16) + (row & 7) * 16;
        for (int q = 0; q < a.KX / 16; ++q) {
          const uint4 u0 = *reinterpret_cast<const uint4*>(src + 2 * q * 128);
          const uint4 u1 = *reinterpret_cast<const uint4*>(src + (2 * q + 1) * 128);
          const uint32_t v[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
          tmem_st8(tbase + lofs + kColXA + 8 * q, v);
          // v's registers are the next store's source: reused only after the store completes
          tmem_st_wait();
        }
        tc_fence_before();
        mbar_arrive(a_ready);
      }
      // Fold of ACC_b (complete): per row xt^2 q - 2 xt R + T per dimension of
      // the block, xt being the F16 hi + lo of the scaled, centred point as in
      // BG (columns 3k, 3k + 1 of the row's XA operand: from TMEM, or, when XA
      // is a shared-memory tile, from the item's tile in global memory, which
      // the next item cannot overwrite).  The warp's 32 rows are summed in FP32
      // by a reduce-scatter over groups of 8 dimensions, after which lanes
      // 4u .. 4u + 3 hold dimension 8g + u of group g; lane 4u keeps the item's
      // running sum of it (an FP32 pair s + c, TwoSum), lane 0 that of q.  Nothing in the
      // fold touches FP64 or shared memory: the warp's partial is written once
      // per item.
      float accg[kMaxDT / 8], cmpg[kMaxDT / 8], accq = 0.f, cmpq = 0.f;
#pragma unroll
      for (int g = 0; g < kMaxDT / 8; ++g) accg[g] = cmpg[g] = 0.f;
      const uint8_t* gxa = a.XA + ti * XT;
      auto fold = [&]() {
        uint32_t oq[16], xa0[16], xa1[16] = {};
        tmem_ld16(tACC + 16 * (qc >> 4), oq);
        if (!XS) {
          tmem_ld16(tbase + lofs + kColXA, xa0);
          if (3 * d > 32) tmem_ld16(tbase + lofs + kColXA + 16, xa1);
        }
#pragma unroll
        for (int g = 0; g < kMaxDT / 8; ++g) {
          if (8 * g >= dk) break;
          // the group's R and T columns; the first group's wait also covers q
          // and the XA rows
          uint32_t o0[16], o1[16] = {};
          if (!a.ksplit) {
            // dimension kk: columns 4 kk .. 4 kk + 3 = (R hi, R lo, T hi, T lo);
            // only columns below NACC = round16(4 dk + 1) are read: the second
            // load only when the group has a dimension past its fourth
            tmem_ld16(tACC + 32 * g, o0);
            if (8 * g + 4 < dk) tmem_ld16(tACC + 32 * g + 16, o1);
          } else {
            // R of kk at column kk, T at toff + kk
            tmem_ld16(tACC + 16 * (g >> 1), o0);
            tmem_ld16(tACC + a.toff + 16 * (g >> 1), o1);
          }
          float xt[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int kk = 8 * g + u;
            xt[u] = 0.f;
            if (XS && kk < dk) {
              const int k = k0 + kk;
              const uint16_t hb = __ldg(reinterpret_cast<const unsigned short*>(gxa + x_off(row, 3 * k, a.KX)));
              const uint16_t lb = __ldg(reinterpret_cast<const unsigned short*>(gxa + x_off(row, 3 * k + 1, a.KX)));
              xt[u] = __half2float(__ushort_as_half(hb)) + __half2float(__ushort_as_half(lb));
            }
          }
          if (g == 0)
            tmem_ld_wait_regs(o0, o1, oq, xa0, xa1);
          else
            tmem_ld_wait_regs(o0, o1);
          const float qs = __uint_as_float(oq[qc & 15]);
          float e[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int kk = 8 * g + u;
            if (!XS && kk < dk) {
              // one dimension block when XA is in TMEM (k = kk): register
              // indices fixed at compile time
              constexpr int kMaxXtReg = 31;
              const int ih = (3 * kk) >> 1, il = (3 * kk + 1) >> 1;
              if (il <= kMaxXtReg) {
                const uint32_t wh = ih < 16 ? xa0[ih & 15] : xa1[ih & 15];
                const uint32_t wl = il < 16 ? xa0[il & 15] : xa1[il & 15];
                const uint16_t hb = (uint16_t)(((3 * kk) & 1) ? (wh >> 16) : (wh & 0xffffu));
                const uint16_t lb = (uint16_t)(((3 * kk + 1) & 1) ? (wl >> 16) : (wl & 0xffffu));
                xt[u] = __half2float(__ushort_as_half(hb)) + __half2float(__ushort_as_half(lb));
              }
            }
            float R, T;
            if (!a.ksplit) {
              const uint32_t* o = u < 4 ? o0 : o1;
              const int cc = 4 * (u & 3);
              R = __uint_as_float(o[cc]) + __uint_as_float(o[cc + 1]);
              T = __uint_as_float(o[cc + 2]) + __uint_as_float(o[cc + 3]);
            } else {
              R = __uint_as_float(o0[8 * (g & 1) + u]);
              T = __uint_as_float(o1[8 * (g & 1) + u]);
            }
            e[u] = kk < dk ? fmaf(xt[u], fmaf(xt[u], qs, -2.f * R), T) : 0.f;
          }
          const float sum = warp_reduce_scatter8(e, lane);
          two_sum_add(accg[g], cmpg[g], sum);
          if (g == 0 && k0 == 0) {
            float v = qs;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            two_sum_add(accq, cmpq, v);
          }
        }
      };
      for (int j = 0; j < item.w; ++j, ++uses) {
        bool ok = mbar_wait(&sw_full[b], (uint32_t)(uses & 1), abort, a.err, 28);
        if (!__all_sync(0xffffffffu, ok)) goto exp_out;
        tc_fence_after();
        {
          // the whole half of S and W in registers with one wait, so S_b, W_b
          // are released at once and the next products into them can start
          uint32_t s0[32], s1[32], w0[32], w1[32], qq[32];
          tmem_ld32(tS, s0);
          tmem_ld32(tS + 32, s1);
          tmem_ld32(tS + 64, w0);
          tmem_ld32(tS + 96, w1);
          tmem_ld_wait_regs(s0, s1, w0, w1);
          tc_fence_before();
          mbar_arrive(&s_free[b]);
          if (item.z + j == item.y) {
            // diagonal tile of the upper triangle: counted once, off-diagonal
            // tiles twice; the pair i = j is left out (its distance is 0, and its
            // share of the alpha gradient is added exactly at the end)
            const int e = row - 64 * b;
#pragma unroll
            for (int q = 0; q < 32; ++q) {
              w0[q] = __float_as_uint(q == e ? 0.f : 0.5f * __uint_as_float(w0[q]));
              w1[q] = __float_as_uint(q + 32 == e ? 0.f : 0.5f * __uint_as_float(w1[q]));
            }
          }
          // Q = W 2^S split into F16 hi and lo parts
          uint32_t qh[32];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            float h0, l0, h1, l1;
            split_q(ex2(__uint_as_float(s0[2 * q])) * __uint_as_float(w0[2 * q]), h0, l0);
            split_q(ex2(__uint_as_float(s0[2 * q + 1])) * __uint_as_float(w0[2 * q + 1]), h1, l1);
            qh[q] = pack_f16x2(h0, h1);
            qq[q] = pack_f16x2(l0, l1);
          }
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            float h0, l0, h1, l1;
            split_q(ex2(__uint_as_float(s1[2 * q])) * __uint_as_float(w1[2 * q]), h0, l0);
            split_q(ex2(__uint_as_float(s1[2 * q + 1])) * __uint_as_float(w1[2 * q + 1]), h1, l1);
            qh[16 + q] = pack_f16x2(h0, h1);
            qq[16 + q] = pack_f16x2(l0, l1);
          }
          if (j > 0) {
            // the feature sums of Q(j-1) are done: Q_b may be overwritten, and
            // ACC_b is complete up to half j-1
            ok = mbar_wait(&q_free[b], (uint32_t)(qf & 1), abort, a.err, 30);
            if (!__all_sync(0xffffffffu, ok)) goto exp_out;
            ++qf;
            tc_fence_after();
          }
          tmem_st32(tQh, qh);
          tmem_st32(tQl, qq);
        }
        tmem_st_wait();
        // a fold ending at half j-1 reads ACC_b before the sums of Q(j) may
        // restart it (they are issued after q_ready)
        if (j > 0 && ((j - 1) % kFoldOwn) == kFoldOwn - 1) fold();
        tc_fence_before();
        mbar_arrive(&q_ready[b]);
      }
      if (item.w > 0) {
        // the item's last feature sums, then its last fold
        const bool ok = mbar_wait(&q_free[b], (uint32_t)(qf & 1), abort, a.err, 30);
        if (!__all_sync(0xffffffffu, ok)) goto exp_out;
        ++qf;
        tc_fence_after();
        fold();
      }
      {
        // per-warp partial of this item: [q, contrib_0 .. contrib_{d-1}], the
        // entries outside the dimension block zero
        double* out = a.gpart + (((size_t)a.chunk * a.n_items + t) * kFoldWarps + b * 4 + w) * kGW;
        for (int v = lane; v <= d; v += 32) {
          const int kk = v - 1 - k0;
          if (v > 0 && kk >= 0 && kk < dk) continue;
          out[v] = v == 0 && k0 == 0 ? (double)accq + (double)cmpq : 0.0;
        }
        if ((lane & 3) == 0) {
#pragma unroll
          for (int g = 0; g < kMaxDT / 8; ++g) {
            const int kk = 8 * g + (lane >> 2);
            if (kk < dk) out[1 + k0 + kk] = (double)accg[g] + (double)cmpg[g];
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

// max |G_i| and max |V_j| per system (row norms, with the amplitudes),
// sum_i G_i . V_i (the noise gradient) and sum_i amp_i^2 G_i . V_i (the
// diagonal's share of the alpha gradient).
__global__ void tc_bwd_norms_kernel(DevLayout L, int chains, int64_t n_total, const float* V, const float* G,
                                    int m, uint32_t* gmax, uint32_t* vmax, double* gvpart, double* gvdiag,
                                    const int32_t* sys_active, const float* amp) {
  __shared__ double red[kTile / 32];
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int s = b * chains + c;
  if (sys_active && !sys_active[s]) return;
  const int64_t i = L.item_row0[item] + threadIdx.x;
  double gv = 0.0, am2 = 1.0;
  if (i < L.offsets[b + 1]) {
    float g2 = 0.f, v2 = 0.f;
    for (int q = 0; q < m; ++q) {
      const int64_t idx = ((int64_t)c * n_total + i) * m + q;
      const float gq = G[idx], vq = V[idx];
      g2 = fmaf(gq, gq, g2);
      v2 = fmaf(vq, vq, v2);
      gv += (double)gq * (double)vq;
    }
    const float am = amp ? amp[(int64_t)c * n_total + i] : 1.f;
    am2 = (double)am * (double)am;
    atomicMax(&gmax[s], __float_as_uint(sqrtf(g2) * am));
    atomicMax(&vmax[s], __float_as_uint(sqrtf(v2) * am));
  }
  const double t = block_sum(gv, red);
  __syncthreads();
  const double t2 = block_sum(gv * am2, red);
  if (threadIdx.x == 0) {
    gvpart[(int64_t)item * chains + c] = t;
    gvdiag[(int64_t)item * chains + c] = t2;
  }
}

// GI, VJ and BG operand tiles of every (chain, padded tile).
// G and V enter by columns [c0, c0 + mc) of their m; GI rows [gh gh gl vh vh vl],
// VJ rows [vh vl vh gh gl gh] (F16 hi/lo, G and V each scaled by a power of
// two), so that GI VJ^T = G_i . V_j + V_i . G_j over the block.  BG carries the
// F16 hi/lo parts of the centred xt and of xt^2 for the dimensions
// [k0, k0 + dk), in the layout of TcBwdArgs, and the ones column.
__global__ void tc_prep_bwd_kernel(DevLayout L, TcTables T, int n_inst, int chains, int d, int ard, int n_theta,
                                   int m, int c0, int mc, int KG, int NB, int ksplit, int NACC, int toff, int qcol,
                                   int k0, int dk, int T_total, const float* x, const double* theta,
                                   const uint32_t* ckeys,
                                   const float* V, const float* G, int64_t n_total, const uint32_t* gmax,
                                   const uint32_t* vmax, const int32_t* sys_active, const float* amp,
                                   uint8_t* GI, uint8_t* VJ, uint8_t* BG, int* err) {
  __shared__ float s_sc[kMaxDT], s_c[kMaxDT];
  const int t = blockIdx.x, c = blockIdx.y, r = threadIdx.x;
  const int b = T.tile_inst[t];
  const int s = b * chains + c;
  if (sys_active && !sys_active[s]) return;
  // scale sqrt(log2 e) / l_k and centre c_k of the block's dimensions, once
  // per block (exp in FP64)
  if (r < dk) {
    const double* th = theta + (int64_t)s * n_theta;
    const int k = k0 + r;
    s_sc[r] = (float)(sqrt(2.0 * kHalfLog2e) * exp(-th[1 + (ard ? k : 0)]));
    s_c[r] = center_of(ckeys, n_inst, d, b, k);
  }
  __syncthreads();
  const int64_t nb = L.offsets[b + 1] - L.offsets[b];
  const int64_t rl = (int64_t)(t - T.inst_tile0[b]) * 128 + r;
  const bool valid = rl < nb;
  const int64_t i = L.offsets[b] + rl;
  const size_t tile = (size_t)c * T_total + t;
  __half* gi = reinterpret_cast<__half*>(GI + tile * (size_t)KG * 256);
  __half* vj = reinterpret_cast<__half*>(VJ + tile * (size_t)KG * 256);
  __half* bg = reinterpret_cast<__half*>(BG + tile * (size_t)NB * 256);
  const float am = (valid && amp) ? amp[(int64_t)c * n_total + i] : 1.f;
  const float gs = (float)row_scale(gmax[s]) * am, vs = (float)row_scale(vmax[s]) * am;
  const __half zh = __float2half_rn(0.f);
  // feature q = part * mc + col: GI rows [gh, gh, gl | vh, vh, vl], VJ rows
  // [vh, vl, vh | gh, gl, gh] (the second half symmetrises W).  Eight
  // consecutive features of a row are 16 contiguous bytes of the tile: each
  // thread assembles them and writes them with one 16-byte store.
  auto feature = [&](int q, __half& gval, __half& vval) {
    gval = vval = zh;
    if (!valid || q >= 6 * mc) return;
    const int col = q % mc, part = q / mc;
    const int64_t idx = ((int64_t)c * n_total + i) * m + c0 + col;
    const float gq = G[idx] * gs, vq = V[idx] * vs;
    const __half gh = __float2half_rn(gq), vh = __float2half_rn(vq);
    const __half gl = __float2half_rn(gq - __half2float(gh));
    const __half vl = __float2half_rn(vq - __half2float(vh));
    if (part < 3) {
      gval = part < 2 ? gh : gl;
      vval = part == 1 ? vl : vh;
    } else {
      gval = part < 5 ? vh : vl;
      vval = part == 4 ? gl : gh;
    }
  };
  for (int q0 = 0; q0 < KG; q0 += 8) {
    uint32_t gw[4], vw[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      __half g0, v0, g1, v1;
      feature(q0 + 2 * e, g0, v0);
      feature(q0 + 2 * e + 1, g1, v1);
      gw[e] = (uint32_t)__half_as_ushort(g0) | ((uint32_t)__half_as_ushort(g1) << 16);
      vw[e] = (uint32_t)__half_as_ushort(v0) | ((uint32_t)__half_as_ushort(v1) << 16);
    }
    *reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(gi) + x_off(r, q0, KG)) = make_uint4(gw[0], gw[1], gw[2], gw[3]);
    *reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(vj) + x_off(r, q0, KG)) = make_uint4(vw[0], vw[1], vw[2], vw[3]);
  }
  for (int f = 0; f < NB; ++f) bg[t_off(f, r) / 2] = zh;
  if (valid) {
    for (int kk = 0; kk < dk; ++kk) {
      const int k = k0 + kk;
      const float xh = (x[i * d + k] - s_c[kk]) * s_sc[kk];
      const __half hi = __float2half_rn(xh);
      const __half lo = __float2half_rn(xh - __half2float(hi));
      const float xtv = __half2float(hi) + __half2float(lo);
      if (!(fabsf(xtv) < 240.f)) atomicCAS(err, 0, 100);
      const float sq = xtv * xtv;
      const __half sh = __float2half_rn(sq);
      const __half sl = __float2half_rn(sq - __half2float(sh));
      if (!ksplit) {
        bg[t_off(4 * kk, r) / 2] = hi;
        bg[t_off(4 * kk + 1, r) / 2] = lo;
        bg[t_off(4 * kk + 2, r) / 2] = sh;
        bg[t_off(4 * kk + 3, r) / 2] = sl;
      } else {
        bg[t_off(kk, r) / 2] = hi;
        bg[t_off(toff + kk, r) / 2] = sh;
        bg[t_off(NACC + kk, r) / 2] = lo;
        bg[t_off(NACC + toff + kk, r) / 2] = sl;
      }
    }
    bg[t_off(qcol, r) / 2] = __float2half_rn(1.f);
  }
}

// grad[s, :] from the per-warp partials and sum_i G_i . V_i.  Each thread
// sums a fixed strided subset of the partials, then a fixed-shape tree joins
// the threads, so the result is bitwise reproducible.
constexpr int kFinThreads = 256;

// Partial sums of one system's gradient partials over a fixed slice of its
// (item, warp) rows, all chunks, entries 0..d (q and the d dimensions); slice
// 0 also sums the instance's G.V terms.  Grid (systems, slices): the slices
// spread a single large system over many SMs, and the fixed split keeps the
// order of the sums, hence the result, the same on every run.
__global__ void __launch_bounds__(kFinThreads) tc_bwd_fin_part_kernel(
    DevLayout L, const int32_t* pref, int n_items, int n_chunks, int chains, int d, int n_slices,
    const double* gpart, const double* gvpart, const double* gvdiag, const int32_t* sys_active, double* fin) {
  __shared__ double red[kFinThreads / 32][kGW + 2];
  const int s = blockIdx.x, p = blockIdx.y;
  if (sys_active && !sys_active[s]) return;
  const int b = s / chains, c = s - b * chains;
  const int64_t n_rows = (int64_t)(pref[s + 1] - pref[s]) * kFoldWarps;   // (item, warp) partial rows per chunk
  const int64_t q0 = n_rows * p / n_slices, q1 = n_rows * (p + 1) / n_slices;
  double acc[kGW + 2];
#pragma unroll
  for (int v = 0; v <= kGW + 1; ++v) acc[v] = 0.0;
  for (int ch = 0; ch < n_chunks; ++ch) {
    const int64_t r0 = ((int64_t)ch * n_items + pref[s]) * kFoldWarps;
    for (int64_t r = q0 + threadIdx.x; r < q1; r += kFinThreads) {
      const double* row = gpart + (r0 + r) * kGW;
      // compile-time indices keep acc in registers
#pragma unroll
      for (int v = 0; v < kGW; ++v)
        if (v <= d) acc[v] += row[v];
    }
  }
  if (p == 0) {
    for (int it = L.inst_item0[b] + threadIdx.x; it < L.inst_item0[b + 1]; it += kFinThreads) {
      acc[kGW] += gvpart[(int64_t)it * chains + c];
      acc[kGW + 1] += gvdiag[(int64_t)it * chains + c];
    }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int v = 0; v <= kGW + 1; ++v) {
    if (v <= d || v >= kGW) {
      double u = acc[v];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) u += __shfl_down_sync(0xffffffffu, u, o);
      if (lane == 0) red[w][v] = u;
    }
  }
  __syncthreads();
  double* out = fin + ((int64_t)s * n_slices + p) * (kGW + 2);
  for (int v = threadIdx.x; v <= kGW + 1; v += kFinThreads) {
    double tot = 0.0;
    if (v <= d || v >= kGW)
      for (int ww = 0; ww < kFinThreads / 32; ++ww) tot += red[ww][v];
    out[v] = tot;
  }
}

// The gradient of each system from its slices' sums: one block per system,
// thread v sums entry v over the slices in slice order, thread 0 applies the
// scales.
constexpr int kFinalThreads = 64;   // >= kGW + 2
static_assert(kFinalThreads >= kGW + 2, "one thread per entry");
__global__ void __launch_bounds__(kFinalThreads) tc_bwd_finalize_kernel(
    int n_theta, int ard, int d, int n_slices, const double* theta, const double* fin, const uint32_t* gmax,
    const uint32_t* vmax, const int32_t* sys_active, const int* err, double* grad) {
  __shared__ double tot[kGW + 2];
  const int s = blockIdx.x, v = threadIdx.x;
  if (sys_active && !sys_active[s]) return;
  if (v <= kGW + 1) {
    double acc = 0.0;
    if (v <= d || v >= kGW)
      for (int p = 0; p < n_slices; ++p) acc += fin[((int64_t)s * n_slices + p) * (kGW + 2) + v];
    tot[v] = acc;
  }
  __syncthreads();
  if (v != 0) return;
  const double* th = theta + (int64_t)s * n_theta;
  const double alpha = exp(th[0]), s2 = exp(th[n_theta - 1]);
  // W^s carried the scales of G and V
  const double gs = row_scale(gmax[s]) * row_scale(vmax[s]);
  const bool bad = *err != 0;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  double* out = grad + (int64_t)s * n_theta;
  // off-diagonal pairs from the kernel, the pairs i = j (K0_ii = 1) exactly
  out[0] = bad ? nan : alpha * (tot[0] / gs + tot[kGW + 1]);
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
  if (a.d > kMaxDT) return tc_fail(h, KMV_EUNSUPPORTED, "tensor-core adjoint supports d <= 32");
  TcState* S = tc_state(h);
  const TcTiles tl = tc_tiles_for(h, kTilesAdjoint, a.d, a.m);
  kmv_status stt = tc_build_plan(h, S, 0, tl.items_per_sm, st);
  if (stt != KMV_OK) return stt;
  const int n_sys = L.n_inst * L.chains;
  const int KX = x_width(a.d, kSplitF16);
  const size_t max_stages = tl.stages > 0 ? (size_t)std::max(2, std::min(tl.stages, 6)) : 6;
  const size_t fixed = 1024 + kTsBarBytes;
  // Feature-sum layout, dimensions per launch (dk), columns of G, V per launch
  // (mc) and where XA lives: the two accumulators and (unless XS) the XA rows
  // must fit the TMEM columns left by S, W and Q (128), and the GI tile, the
  // XA tile (XS) and at least two stages shared memory.  Fewest launches
  // first, then XA in TMEM, then the wide layout (fewer MMAs per half tile).
  struct Choice {
    int ksplit, NACC, toff, qcol, NB, dk, n_dblk, mc, n_cblk, stages;
    bool xs;
    long long launches;
  };
  auto make = [&](int ksplit, bool xs, int n_dblk) -> Choice {
    Choice c{};
    c.ksplit = ksplit;
    c.xs = xs;
    c.n_dblk = n_dblk;
    c.dk = (a.d + n_dblk - 1) / n_dblk;
    c.launches = LLONG_MAX;
    // XA in TMEM: one dimension block (the fold's register indices are fixed),
    // and a row's split values in at most two loads
    if (!xs && (n_dblk != 1 || 3 * a.d > 64)) return c;
    if (!ksplit) {
      c.toff = 0;
      c.qcol = 4 * c.dk;
      c.NACC = round16(4 * c.dk + 1);
      c.NB = c.NACC;
    } else {
      c.toff = round16(c.dk);
      c.qcol = 2 * c.toff;
      c.NACC = round16(c.qcol + 1);
      c.NB = 2 * c.NACC;
    }
    if ((int)kColXA + (xs ? 0 : KX / 2) + 2 * c.NACC > 512) return c;
    for (int mc = a.m; mc >= 1; --mc) {
      const size_t KG = round16(6 * mc);
      const size_t stg = (size_t)(KX + KG + c.NB) * 256;
      const size_t base = fixed + al1k(KG * 256) + (xs ? al1k((size_t)KX * 256) : 0);
      if (base + 2 * stg > kMaxSmem) continue;
      c.mc = mc;
      c.n_cblk = (a.m + mc - 1) / mc;
      c.stages = (int)std::min<size_t>(max_stages, (kMaxSmem - base) / stg);
      c.launches = (long long)c.n_cblk * n_dblk;
      return c;
    }
    return c;
  };
  Choice best{};
  best.launches = LLONG_MAX;
  for (int n_dblk = 1; n_dblk <= a.d; ++n_dblk) {
    if (n_dblk > 1 && (a.d + n_dblk - 1) / n_dblk == (a.d + n_dblk - 2) / (n_dblk - 1)) continue;
    for (bool xs : {false, true})
      for (int ksplit : {0, 1}) {
        const Choice c = make(ksplit, xs, n_dblk);
        if (c.launches < best.launches) best = c;
      }
    if (best.launches < LLONG_MAX) break;
  }
  if (best.launches == LLONG_MAX)
    return tc_fail(h, KMV_EUNSUPPORTED, "tensor-core adjoint operands do not fit in tensor/shared memory");
  const bool xs = best.xs;
  const int mc = best.mc, NB = best.NB, n_chunks = (int)best.launches;
  const int KG = round16(6 * mc);
  const size_t XT = (size_t)KX * 256, GT = (size_t)KG * 256, BT = (size_t)NB * 256;
  const size_t STG = XT + GT + BT;
  const size_t smem = std::max(kMinSmem, fixed + al1k(GT) + (xs ? al1k(XT) : 0) + best.stages * STG);
  const int n_items = S->sym_n_items;

  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  const size_t tiles = (size_t)L.chains * S->T_total;
  const size_t gvb = al(sizeof(double) * (size_t)std::max(1, L.n_items) * L.chains);
  const size_t o_xa = 0, o_xb = o_xa + al(tiles * XT), o_gi = o_xb + al(tiles * XT);
  const size_t o_vj = o_gi + al(tiles * GT), o_bg = o_vj + al(tiles * GT), o_mx = o_bg + al(tiles * BT);
  const size_t o_gv = o_mx + al(sizeof(uint32_t) * 2 * n_sys);
  const size_t o_gd = o_gv + gvb;
  const size_t o_ck = o_gd + gvb;
  const size_t o_gp = o_ck + al(tc_center_bytes(L));
  // slices of the finalize: about kFinThreads partial rows per slice on
  // average, at most 32 per system
  const int64_t rows_per_sys = (int64_t)std::max(1, n_items) * kFoldWarps / std::max(1, n_sys);
  const int n_slices = (int)std::max<int64_t>(1, std::min<int64_t>(32, (rows_per_sys + kFinThreads - 1) / kFinThreads));
  const size_t o_fn = o_gp + al(sizeof(double) * (size_t)n_chunks * std::max(1, n_items) * kFoldWarps * kGW);
  const size_t o_er = o_fn + al(sizeof(double) * (size_t)n_sys * n_slices * (kGW + 2));
  stt = tc_ensure_buf(h, S, o_er + 256);
  if (stt != KMV_OK) return stt;
  uint8_t* base = static_cast<uint8_t*>(S->buf);
  uint32_t* gmax = reinterpret_cast<uint32_t*>(base + o_mx);
  uint32_t* vmax = gmax + n_sys;
  double* gvpart = reinterpret_cast<double*>(base + o_gv);
  double* gvdiag = reinterpret_cast<double*>(base + o_gd);
  uint32_t* ckeys = reinterpret_cast<uint32_t*>(base + o_ck);
  double* gpart = reinterpret_cast<double*>(base + o_gp);
  double* fin = reinterpret_cast<double*>(base + o_fn);
  int* err = reinterpret_cast<int*>(base + o_er);

  if (!S->bwd_attr_set) {
    if (cudaFuncSetAttribute(tc_bwd_ts_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kMaxSmem) != cudaSuccess ||
        cudaFuncSetAttribute(tc_bwd_ts_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kMaxSmem) != cudaSuccess)
      return tc_fail(h, KMV_ECUDA, "cudaFuncSetAttribute failed");
    S->bwd_attr_set = true;
  }
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(base + o_mx, 0, o_gv - o_mx, st) != cudaSuccess)
    return tc_fail(h, KMV_ECUDA, "memset failed");
  if (L.n_items > 0)
    tc_bwd_norms_kernel<<<dim3(L.n_items, L.chains), kTile, 0, st>>>(h->dev, L.chains, L.n_total, a.V, a.G, a.m,
                                                                     gmax, vmax, gvpart, gvdiag, a.sys_active,
                                                                     a.amp);
  // the adjoint's operand tiles overwrite the forward's
  S->prep_valid = false;
  if (n_items > 0) {
    tc_launch_center(h, a, ckeys, st);
    tc_launch_prep_x(h, S, a, KX, kSplitF16, ckeys, base + o_xa, base + o_xb, err, st);
    TcBwdArgs ba;
    ba.items = S->d_sym_items;
    ba.n_items = n_items;
    ba.chains = L.chains;
    ba.T_total = S->T_total;
    ba.KX = KX;
    ba.KG = KG;
    ba.NB = NB;
    ba.ksplit = best.ksplit;
    ba.NACC = best.NACC;
    ba.toff = best.toff;
    ba.qcol = best.qcol;
    ba.S = best.stages;
    ba.d = a.d;
    ba.XA = base + o_xa;
    ba.XB = base + o_xb;
    ba.GI = base + o_gi;
    ba.VJ = base + o_vj;
    ba.BG = base + o_bg;
    ba.gpart = gpart;
    ba.sys_active = a.sys_active;
    ba.err = err;
    const int grid = std::min(n_items, S->num_sms);
    // One launch per (block of mc columns of G, V, block of dk dimensions): the
    // gradient is a sum over columns, and the dimensions are separate entries
    // (q enters once, from the first dimension block), so the finalize sums
    // every launch's partials.  Stream order keeps each block's operand tiles
    // until its launch has read them.
    for (int cb = 0; cb < best.n_cblk; ++cb) {
      const int c0 = cb * mc, mcc = std::min(mc, a.m - c0);
      for (int db = 0; db < best.n_dblk; ++db) {
        const int k0 = db * best.dk, dkk = std::min(best.dk, a.d - k0);
        if (dkk <= 0) continue;
        tc_prep_bwd_kernel<<<dim3(S->T_total, L.chains), 128, 0, st>>>(
            h->dev, S->dev, L.n_inst, L.chains, a.d, a.ard, a.n_theta, a.m, c0, mcc, KG, NB, best.ksplit,
            best.NACC, best.toff, best.qcol, k0, dkk, S->T_total, a.x, a.theta, ckeys, a.V, a.G, L.n_total, gmax,
            vmax, a.sys_active, a.amp, base + o_gi, base + o_vj, base + o_bg, err);
        ba.chunk = cb * best.n_dblk + db;
        ba.k0 = k0;
        ba.dk = dkk;
        ProfScope prof(h, KMV_KERNEL_ADJOINT, st);
        if (xs)
          tc_bwd_ts_kernel<true><<<grid, kTsThreads, smem, st>>>(ba);
        else
          tc_bwd_ts_kernel<false><<<grid, kTsThreads, smem, st>>>(ba);
      }
    }
  }
  tc_bwd_fin_part_kernel<<<dim3(n_sys, n_slices), kFinThreads, 0, st>>>(
      h->dev, S->dev.sym_pref, n_items, n_chunks, L.chains, a.d, n_slices, gpart, gvpart, gvdiag, a.sys_active, fin);
  tc_bwd_finalize_kernel<<<n_sys, kFinalThreads, 0, st>>>(a.n_theta, a.ard, a.d, n_slices, a.theta, fin, gmax, vmax,
                                                           a.sys_active, err, grad);
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

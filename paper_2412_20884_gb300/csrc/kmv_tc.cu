// Tensor-core (tcgen05) form of Y = A(theta) V, KMV_BF16_HILO.
//
// Layout in HBM (written per call by the prep kernels, per chain c, in
// 128-row tiles that are byte-for-byte the shared-memory operand layout, so
// each tile moves with one bulk copy):
//   XA[c][t] : 128 x KX BF16, rows i:  per dimension [hi, lo, hi] of xh, then 1, 1, 1, bh, bm, bl, 0..
//   XB[c][t] : 128 x KX BF16, rows j:  per dimension [hi, hi, lo] of xh, then bh, bm, bl, 1, 1, 1, 0..
//   VT[c][t] : MP x 128 F16, V^T of the tile scaled by a per-column power of two
// with xh = x sqrt(log2(e)) / l and b = -|xh|^2/2 (computed from the split
// values, so the diagonal exponent is 0) split into three BF16 terms.  One
// K = KX contraction then gives the base-2 exponent of K0 directly:
//   S_ij = hi_i.hi_j + hi_i.lo_j + lo_i.hi_j + b_i + b_j = -|xh_i - xh_j|^2/2 + O(2^-16 |xh|^2)
// and K0_ij = 2^S_ij.  Core matrices are 8 rows x 16 bytes, no swizzle.
//
// Main kernel (one CTA per SM, persistent over work items): an item is one
// pair of 128-row I tiles of one system against a contiguous range of J tiles.
//   warp 9       : bulk-copy producer (A tiles per item, XB/VT tiles per J step)
//   warps 8, 10  : one MMA issuer per I tile g: S_g = A_g XB^T into TMEM (a
//                  128x128 FP32 accumulator), then O_g += P_g VT^T with P_g
//                  read from TMEM.  Two issuers let the two tiles' thin P.V
//                  MMAs overlap in the tensor pipe and keep the warpgroups
//                  independent of each other.
//   warps 0-7    : two exp warpgroups, one per I tile: TMEM S -> ex2 -> F16 P
//                  written to its own TMEM columns (the second half tile's
//                  TMEM loads overlap the first half's exps), and every kFold
//                  J tiles the FP32 O accumulator is folded into per-column
//                  FP32 pair sums (TwoSum), written in FP64 once per item.
// An epilogue kernel sums the per-item partials in a fixed order and applies
// Y = alpha O + (sigma^2 + shift) V.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "cg_common.cuh"
#include "kmv_tc.cuh"
#include "simt_common.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace kmv {

namespace {

// J tiles accumulated in FP32 in TMEM before each fold (4096 columns) into
// the per-column TwoSum pairs.
constexpr int kFold = 32;
// Forward warp roles: warps 0-7 two exp warpgroups, warp 8 MMA issuer for I
// tile 0 (and TMEM owner), warp 9 producer, warp 10 MMA issuer for I tile 1.
constexpr int kFwdThreads = 352;
constexpr int kIssue1Warp = 10;
// FMA-pipe forward warp roles: warps 0-15 four exp warpgroups (I tile
// (w >> 2) & 1, S columns 64 (w >> 3) .. + 63), warp 16 MMA issuer for I
// tile 0 (and TMEM owner), warp 17 producer, warp 18 MMA issuer for I tile 1.
constexpr int kFmaThreads = 608;
constexpr int kFmaMmaWarp = 16, kFmaLoadWarp = 17, kFmaIssue1Warp = 18;

// Issues S = A B^T (K = 16 nk) and O (+)= P VT^T (K = 128 from TMEM).
__device__ __forceinline__ void issue_s(uint32_t d_tmem, uint64_t da, uint64_t db, int nk, uint32_t idesc) {
  for (int k = 0; k < nk; ++k) ptx::mma_ss(d_tmem, da + 16 * k, db + 16 * k, idesc, k > 0);
}
__device__ __forceinline__ void issue_pv(uint32_t d_tmem, uint32_t a_tmem, uint64_t db, uint32_t idesc,
                                         uint32_t acc) {
#pragma unroll
  for (int k = 0; k < 8; ++k) ptx::mma_ts(d_tmem, a_tmem + 8 * k, db + 16 * k, idesc, (k > 0) || acc);
}

// 2^s for element e of a 32-element chunk (e is a compile-time constant once
// the loops are unrolled): one element in POLY on the FMA pipe (degree-DEG
// polynomial), the rest on the MUFU; POLY = 0 puts every exp on the MUFU.
template <int POLY, int DEG>
__device__ __forceinline__ float exp2_mix(float s, int e) {
  if constexpr (POLY > 0) {
    if ((e % POLY) == POLY - 1) return exp2_fma<DEG>(s);
  }
  return ptx::ex2(s);
}

// FP64 partial of (item t, column q, row rowp in the item's 256 rows): column
// by column, so that the kernels' writes and the epilogue's reads are coalesced.
__host__ __device__ __forceinline__ size_t part_idx(int t, int mz, int q, int rowp) {
  return ((size_t)t * mz + q) * 256 + rowp;
}

struct TcFwdArgs {
  const int4* items;       // {system, I tile (first of 2), first J tile, number of J tiles}
  int n_items;
  int chains;
  int T_total;             // padded tiles per chain
  int KX, MP, S;
  const uint8_t* XA;
  const uint8_t* XB;
  const uint8_t* VT;
  double* part;            // (n_items, mz, 256) FP64, part_idx
  int mz;                  // columns of this pass
  const int32_t* sys_active;
  int* err;
};

// RM > 0: the FP64 fold accumulators of up to RM columns live in registers;
// RM == 0: they live in the per-item partial (global read-modify-write).
template <int RM, int POLY>
__global__ void __launch_bounds__(kFwdThreads, 1) tc_fwd_kernel(TcFwdArgs a) {
  using namespace ptx;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  const uint32_t A_TILE = a.KX * 256u, V_TILE = a.MP * 256u;
  const int S = a.S;
  uint8_t* sA = smem;                       // [buffer 2][tile 2]
  uint8_t* sB = sA + 4 * A_TILE;            // [stage]
  uint8_t* sV = sB + S * A_TILE;            // [stage]
  uint64_t* full = reinterpret_cast<uint64_t*>(sV + S * V_TILE);
  uint64_t* empty = full + S;
  uint64_t* a_full = empty + S;
  uint64_t* a_empty = a_full + 2;
  uint64_t* s_full = a_empty + 2;    // [g] S_g written by the tensor core
  uint64_t* s_free = s_full + 2;     // [g] S_g read into registers by warpgroup g
  uint64_t* p_ready = s_free + 2;    // [g] P_g written by warpgroup g
  uint64_t* p_free = p_ready + 2;    // [g] P_g consumed by the P.V MMAs
  uint64_t* o_ready = p_free + 2;
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
      mbar_init(&p_ready[g], 128);
      mbar_init(&p_free[g], 1);
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
  // TMEM columns: S_g [128 g, 128 g + 128), P_g [256 + 64 g, +64), O_g [384 + 64 g, +MP)

  // The producer and issuer warps run their loops with all 32 lanes, so that
  // addresses and descriptors stay warp-uniform, and one elected lane issues
  // the copies, MMAs and commits: issuing from a lone lane was measured at
  // 2-3x the cost per tcgen05.mma.
  if (warp == kLoadWarp) {
    const bool leader = elect_one();
    {
      // ------------------------------------------------------------ producer
      int it = 0;
      uint32_t stage = 0, sph = 0;
      int n_issued = 0, n_a_issued = 0;
      bool aborted = false;
      for (int t = blockIdx.x; t < a.n_items && !aborted; t += gridDim.x) {
        const int4 item = a.items[t];
        if (a.sys_active && !a.sys_active[item.x]) continue;
        const int c = item.x % a.chains;
        const int ab = it & 1;
        if (!warp_wait(&a_empty[ab], ((it >> 1) & 1) ^ 1, abort, a.err, 1)) { aborted = true; break; }
        if (leader) {
          mbar_arrive_expect_tx(&a_full[ab], 2 * A_TILE);
          bulk_g2s(sA + (2 * ab) * A_TILE, a.XA + ((size_t)c * a.T_total + item.y) * A_TILE, 2 * A_TILE,
                   &a_full[ab]);
        }
        __syncwarp();
        ++n_a_issued;
        for (int j = 0; j < item.w; ++j) {
          if (!warp_wait(&empty[stage], sph ^ 1, abort, a.err, 2)) { aborted = true; break; }
          if (leader) {
            mbar_arrive_expect_tx(&full[stage], A_TILE + V_TILE);
            const size_t tj = (size_t)c * a.T_total + item.z + j;
            bulk_g2s(sB + stage * A_TILE, a.XB + tj * A_TILE, A_TILE, &full[stage]);
            bulk_g2s(sV + stage * V_TILE, a.VT + tj * V_TILE, V_TILE, &full[stage]);
          }
          __syncwarp();
          ++n_issued;
          if (++stage == (uint32_t)S) { stage = 0; sph ^= 1; }
        }
        ++it;
      }
      if (aborted) {
        // drain: the copies already issued must land before the CTA exits
        for (int k = 1; k <= min(n_issued, S); ++k) {
          const int idx = n_issued - k;
          mbar_drain(&full[idx % S], (idx / S) & 1, 500000000ull);
        }
        for (int k = 1; k <= min(n_a_issued, 2); ++k) {
          const int idx = n_a_issued - k;
          mbar_drain(&a_full[idx & 1], (idx >> 1) & 1, 500000000ull);
        }
      }
    }
  } else if (warp == kMmaWarp || warp == kIssue1Warp) {
    const bool leader = elect_one();
    {
      // ------------------------------------------------------------ MMA issuer of I tile g
      // Tile stream k = 0, 1, ... over this CTA's items.  For tile k it issues
      // S(k) once warpgroup g has read S(k-1), then P.V of tile k-1 once P(k-1)
      // is written, so the tensor core computes the next S while the
      // warpgroup computes exps, and P.V runs during the next tile's exps.
      const int g = warp == kMmaWarp ? 0 : 1;
      const uint32_t idS = idesc_f16(128, 128, 1, 1);
      const uint32_t idP = idesc_f16(128, a.MP, 0, 0);
      const uint32_t sboX = a.KX * 16u;
      const int nkx = a.KX / 16;
      const uint64_t dA = sdesc(smem_u32(sA + g * A_TILE), 128, sboX);
      const uint64_t dB = sdesc(smem_u32(sB), 128, sboX);
      const uint64_t dV = sdesc(smem_u32(sV), 128, 2048);
      const uint32_t s_tmem = tbase + g * 128, p_tmem = tbase + 256 + g * 64, o_tmem = tbase + 384 + g * 64;
      int it = 0;
      uint32_t stage = 0, sph = 0;
      uint32_t sf_ph = 0, pr_ph = 0, of_ph = 0;
      bool opend = false;
      long long k = 0;
      // the previous tile, whose P.V is still to be issued
      bool have_prev = false;
      uint32_t prev_stage = 0;
      int prev_j = 0, prev_nJ = 0, prev_ab = 0;
      for (int t = blockIdx.x; t < a.n_items; t += gridDim.x) {
        const int4 item = a.items[t];
        if (a.sys_active && !a.sys_active[item.x]) continue;
        const int ab = it & 1;
        const uint64_t dAg = sdesc_add(dA, 2 * ab * A_TILE);
        for (int j = 0; j < item.w; ++j, ++k) {
          // ---- S(k)
          if (k > 0) {
            if (!warp_wait(&s_free[g], sf_ph, abort, a.err, 3)) goto mma_out;
            sf_ph ^= 1;
          }
          if (j == 0 && !warp_wait(&a_full[ab], (it >> 1) & 1, abort, a.err, 4)) goto mma_out;
          if (!warp_wait(&full[stage], sph, abort, a.err, 5)) goto mma_out;
          tc_fence_after();
          // operands computed by the whole warp (warp-uniform), issued by the leader
          const uint64_t db = sdesc_add(dB, stage * A_TILE);
          if (leader) {
            issue_s(s_tmem, dAg, db, nkx, idS);
            tc_commit(&s_full[g]);
          }
          __syncwarp();
          // ---- P.V of tile k-1
          if (have_prev) {
            if (!warp_wait(&p_ready[g], pr_ph, abort, a.err, 6)) goto mma_out;
            pr_ph ^= 1;
            tc_fence_after();
            const uint32_t acc = (prev_j % kFold) != 0;
            if (!acc && opend) {
              if (!warp_wait(&o_free[g], of_ph, abort, a.err, 7)) goto mma_out;
              of_ph ^= 1;
              opend = false;
              tc_fence_after();
            }
            const bool fold_end = (prev_j % kFold) == kFold - 1 || prev_j == prev_nJ - 1;
            const uint64_t dv = sdesc_add(dV, prev_stage * V_TILE);
            if (leader) {
              issue_pv(o_tmem, p_tmem, dv, idP, acc);
              tc_commit(&p_free[g]);
              if (fold_end) tc_commit(&o_ready[g]);
              tc_commit(&empty[prev_stage]);
              if (prev_j == prev_nJ - 1) tc_commit(&a_empty[prev_ab]);
            }
            __syncwarp();
            if (fold_end) opend = true;
          }
          have_prev = true;
          prev_stage = stage;
          prev_j = j;
          prev_nJ = item.w;
          prev_ab = ab;
          if (++stage == (uint32_t)S) { stage = 0; sph ^= 1; }
        }
        ++it;
      }
      if (have_prev) {
        if (!warp_wait(&p_ready[g], pr_ph, abort, a.err, 6)) goto mma_out;
        tc_fence_after();
        const uint32_t acc = (prev_j % kFold) != 0;
        if (!acc && opend) {
          if (!warp_wait(&o_free[g], of_ph, abort, a.err, 7)) goto mma_out;
          tc_fence_after();
        }
        const uint64_t dv = sdesc_add(dV, prev_stage * V_TILE);
        if (leader) {
          issue_pv(o_tmem, p_tmem, dv, idP, acc);
          tc_commit(&p_free[g]);
          tc_commit(&o_ready[g]);
          tc_commit(&empty[prev_stage]);
          tc_commit(&a_empty[prev_ab]);
        }
        __syncwarp();
      }
    mma_out:
      if (leader) tc_commit(&done[g]);
      __syncwarp();
      mbar_drain(&done[g], 0, 500000000ull);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ exp warpgroups
    const int g = warp >> 2, w = warp & 3;
    const int row = 32 * w + lane;
    const uint32_t tl = tbase + (static_cast<uint32_t>(32 * w) << 16);
    const uint32_t s_col = g * 128, p_col = 256 + g * 64, o_col = 384 + g * 64;
    uint32_t sph = 0, pf_ph = 0, oph = 0;
    long long k = 0;
    for (int t = blockIdx.x; t < a.n_items; t += gridDim.x) {
      const int4 item = a.items[t];
      if (a.sys_active && !a.sys_active[item.x]) continue;
      const int rowp = g * 128 + row;
      // the item's O sums per column as FP32 pairs (TwoSum; the FP64 pipe is a
      // small fraction of the FP32 rate on this GPU), written in FP64
      float rs[RM > 0 ? RM : 1], rc[RM > 0 ? RM : 1];
#pragma unroll
      for (int q = 0; q < (RM > 0 ? RM : 1); ++q) rs[q] = rc[q] = 0.f;
      bool first = true;
      for (int j = 0; j < item.w; ++j, ++k) {
        bool ok = mbar_wait(&s_full[g], sph, abort, a.err, 8);
        if (!__all_sync(0xffffffffu, ok)) goto exp_out;
        sph ^= 1;
        tc_fence_after();
        {
          uint32_t a0[32], a1[32], b0[32], b1[32], pk[32];
          tmem_ld32(tl + s_col, a0);
          tmem_ld32(tl + s_col + 32, a1);
          tmem_ld_wait_regs(a0, a1);
          tmem_ld32(tl + s_col + 64, b0);
          tmem_ld32(tl + s_col + 96, b1);
#pragma unroll
          for (int q = 0; q < 16; ++q)
            pk[q] = pack_f16x2(exp2_mix<POLY, 3>(__uint_as_float(a0[2 * q]), 2 * q),
                               exp2_mix<POLY, 3>(__uint_as_float(a0[2 * q + 1]), 2 * q + 1));
#pragma unroll
          for (int q = 0; q < 16; ++q)
            pk[16 + q] = pack_f16x2(exp2_mix<POLY, 3>(__uint_as_float(a1[2 * q]), 2 * q),
                               exp2_mix<POLY, 3>(__uint_as_float(a1[2 * q + 1]), 2 * q + 1));
          tmem_ld_wait_regs(b0, b1);
          // S(k) is fully in registers: the tensor core may overwrite it
          tc_fence_before();
          mbar_arrive(&s_free[g]);
          if (k > 0) {
            // P(k-1) must have been consumed before P(k) overwrites it
            ok = mbar_wait(&p_free[g], pf_ph, abort, a.err, 10);
            if (!__all_sync(0xffffffffu, ok)) goto exp_out;
            pf_ph ^= 1;
            tc_fence_after();
          }
          tmem_st32(tl + p_col, pk);
          // the second half's exps in place; pk, the source of the store just
          // issued, is rewritten only after tcgen05.wait::st
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            b0[e] = __float_as_uint(exp2_mix<POLY, 3>(__uint_as_float(b0[e]), e));
            b1[e] = __float_as_uint(exp2_mix<POLY, 3>(__uint_as_float(b1[e]), e));
          }
          tmem_st_wait();
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            pk[q] = pack_f16x2(__uint_as_float(b0[2 * q]), __uint_as_float(b0[2 * q + 1]));
            pk[16 + q] = pack_f16x2(__uint_as_float(b1[2 * q]), __uint_as_float(b1[2 * q + 1]));
          }
          tmem_st32(tl + p_col + 32, pk);
        }
        tmem_st_wait();
        tc_fence_before();
        mbar_arrive(&p_ready[g]);
        if ((j % kFold) == kFold - 1 || j == item.w - 1) {
          ok = mbar_wait(&o_ready[g], oph, abort, a.err, 9);
          if (!__all_sync(0xffffffffu, ok)) goto exp_out;
          oph ^= 1;
          tc_fence_after();
          if (RM > 0) {
#pragma unroll
            for (int c0 = 0; c0 < (RM > 0 ? RM : 16); c0 += 16) {
              if (c0 < a.MP) {
                uint32_t o[16];
                tmem_ld16(tl + o_col + c0, o);
                tmem_ld_wait_regs(o);
#pragma unroll
                for (int q = 0; q < 16; ++q) two_sum_add(rs[c0 + q], rc[c0 + q], __uint_as_float(o[q]));
              }
            }
          } else {
            for (int c0 = 0; c0 < a.MP; c0 += 16) {
              uint32_t o[16];
              tmem_ld16(tl + o_col + c0, o);
              tmem_ld_wait_regs(o);
#pragma unroll
              for (int q = 0; q < 16; ++q) {
                const int col = c0 + q;
                if (col < a.mz) {
                  const double v = (double)__uint_as_float(o[q]);
                  double& pv = a.part[part_idx(t, a.mz, col, rowp)];
                  pv = first ? v : pv + v;
                }
              }
            }
          }
          first = false;
          tc_fence_before();
          mbar_arrive(&o_free[g]);
        }
      }
      if (RM > 0) {
#pragma unroll
        for (int q = 0; q < (RM > 0 ? RM : 1); ++q)
          if (q < a.mz) a.part[part_idx(t, a.mz, q, rowp)] = (double)rs[q] + (double)rc[q];
      }
    }
  exp_out:;
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) tmem_dealloc(tbase, 512);
}

// Forward for one or two columns (the CG product): S = XA XB^T on the tensor
// core as above, but P.v on the FMA pipe with P kept in FP32 and v in FP32
// (tile VF: MZ x 128 floats), so the tensor pipe only computes S and the
// kernel is bound by the exps.  S is double buffered in TMEM (512 columns), so
// the issuers run one tile ahead.  Each I tile's S is read by two exp
// warpgroups, one per 64-column half, so that four warps per scheduler hide
// the exp and FMA latencies; the second half's row sums reach the first
// through shared memory at the end of each item and are added in that order.
template <int MZ, int POLY>
__global__ void __launch_bounds__(kFmaThreads, 1) tc_fwd_fma_kernel(TcFwdArgs a) {
  using namespace ptx;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  const uint32_t A_TILE = a.KX * 256u, V_TILE = MZ * 512u;
  const int S = a.S;
  uint8_t* sA = smem;
  uint8_t* sB = sA + 4 * A_TILE;
  uint8_t* sV = sB + S * A_TILE;
  uint64_t* full = reinterpret_cast<uint64_t*>(sV + S * V_TILE);
  uint64_t* empty = full + S;        // released by the 2 issuers (S read XB) and 16 exp warps (read VF)
  uint64_t* a_full = empty + S;
  uint64_t* a_empty = a_full + 2;
  uint64_t* s_full = a_empty + 2;   // [g][buffer]
  uint64_t* s_free = s_full + 4;    // [g][buffer]
  uint64_t* done = s_free + 4;
  uint64_t* comb_full = done + 2;       // [g][item parity] second half's row sums written
  uint64_t* comb_free = comb_full + 4;  // [g][item parity] ... and read by the first half
  uint32_t* tslot = reinterpret_cast<uint32_t*>(comb_free + 4);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  double* s_comb = reinterpret_cast<double*>(tslot + 2);  // [g][item parity][MZ][128 rows]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 2 + 16);
    }
    for (int g = 0; g < 2; ++g) {
      mbar_init(&a_full[g], 1);
      mbar_init(&a_empty[g], 2);
      mbar_init(&done[g], 1);
    }
    for (int q = 0; q < 4; ++q) {
      mbar_init(&s_full[q], 1);
      mbar_init(&s_free[q], 256);
      mbar_init(&comb_full[q], 128);
      mbar_init(&comb_free[q], 128);
    }
    *abort = 0;
    fence_barrier_init();
  }
  if (warp == kFmaMmaWarp) {
    tmem_alloc(tslot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;

  if (warp == kFmaLoadWarp) {
    const bool leader = elect_one();
    {
      int it = 0;
      uint32_t stage = 0, sph = 0;
      int n_issued = 0, n_a_issued = 0;
      bool aborted = false;
      for (int t = blockIdx.x; t < a.n_items && !aborted; t += gridDim.x) {
        const int4 item = a.items[t];
        if (a.sys_active && !a.sys_active[item.x]) continue;
        const int c = item.x % a.chains;
        const int ab = it & 1;
        if (!warp_wait(&a_empty[ab], ((it >> 1) & 1) ^ 1, abort, a.err, 11)) { aborted = true; break; }
        if (leader) {
          mbar_arrive_expect_tx(&a_full[ab], 2 * A_TILE);
          bulk_g2s(sA + (2 * ab) * A_TILE, a.XA + ((size_t)c * a.T_total + item.y) * A_TILE, 2 * A_TILE,
                   &a_full[ab]);
        }
        __syncwarp();
        ++n_a_issued;
        for (int j = 0; j < item.w; ++j) {
          if (!warp_wait(&empty[stage], sph ^ 1, abort, a.err, 12)) { aborted = true; break; }
          if (leader) {
            mbar_arrive_expect_tx(&full[stage], A_TILE + V_TILE);
            const size_t tj = (size_t)c * a.T_total + item.z + j;
            bulk_g2s(sB + stage * A_TILE, a.XB + tj * A_TILE, A_TILE, &full[stage]);
            bulk_g2s(sV + stage * V_TILE, a.VT + tj * V_TILE, V_TILE, &full[stage]);
          }
          __syncwarp();
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
        for (int k = 1; k <= min(n_a_issued, 2); ++k) {
          const int idx = n_a_issued - k;
          mbar_drain(&a_full[idx & 1], (idx >> 1) & 1, 500000000ull);
        }
      }
    }
  } else if (warp == kFmaMmaWarp || warp == kFmaIssue1Warp) {
    const bool leader = elect_one();
    {
      const int g = warp == kFmaMmaWarp ? 0 : 1;
      const uint32_t idS = idesc_f16(128, 128, 1, 1);
      const uint32_t sboX = a.KX * 16u;
      const int nkx = a.KX / 16;
      const uint64_t dA = sdesc(smem_u32(sA + g * A_TILE), 128, sboX);
      const uint64_t dB = sdesc(smem_u32(sB), 128, sboX);
      // S of I tile g, double-buffered: tile k goes to columns [256 (k & 1) + 128 g, +128),
      // so the next tile's S is computed while the warpgroup still reads this one
      const uint32_t s_tmem = tbase + g * 128;
      int it = 0;
      uint32_t stage = 0, sph = 0;
      uint32_t sf_ph[2] = {0u, 0u};
      long long k = 0;
      for (int t = blockIdx.x; t < a.n_items; t += gridDim.x) {
        const int4 item = a.items[t];
        if (a.sys_active && !a.sys_active[item.x]) continue;
        const int ab = it & 1;
        const uint64_t dAg = sdesc_add(dA, 2 * ab * A_TILE);
        for (int j = 0; j < item.w; ++j, ++k) {
          const int buf = (int)(k & 1);
          if (k >= 2) {
            if (!warp_wait(&s_free[2 * g + buf], sf_ph[buf], abort, a.err, 13)) goto fma_mma_out;
            sf_ph[buf] ^= 1;
          }
          if (j == 0 && !warp_wait(&a_full[ab], (it >> 1) & 1, abort, a.err, 14)) goto fma_mma_out;
          if (!warp_wait(&full[stage], sph, abort, a.err, 15)) goto fma_mma_out;
          tc_fence_after();
          const uint64_t db = sdesc_add(dB, stage * A_TILE);
          if (leader) {
            issue_s(s_tmem + 256 * buf, dAg, db, nkx, idS);
            tc_commit(&s_full[2 * g + buf]);
            tc_commit(&empty[stage]);
            if (j == item.w - 1) tc_commit(&a_empty[ab]);
          }
          __syncwarp();
          if (++stage == (uint32_t)S) { stage = 0; sph ^= 1; }
        }
        ++it;
      }
    fma_mma_out:
      if (leader) tc_commit(&done[g]);
      __syncwarp();
      mbar_drain(&done[g], 0, 500000000ull);
    }
    __syncwarp();
  } else {
    const int g = (warp >> 2) & 1, w = warp & 3, hf = warp >> 3;
    const int row = 32 * w + lane;
    const uint32_t tl = tbase + (static_cast<uint32_t>(32 * w) << 16);
    // barrier phases as bits (bit b: S buffer b; item parity b), kept in registers
    uint32_t sph = 0, stage = 0, fph = 0;
    // phases of comb_full (first half) or comb_free (second half)
    uint32_t cph = 0;
    long long k = 0;
    int it = 0;
    for (int t = blockIdx.x; t < a.n_items; t += gridDim.x) {
      const int4 item = a.items[t];
      if (a.sys_active && !a.sys_active[item.x]) continue;
      const int rowp = g * 128 + row;
      // four independent FP32 chains per column (short FMA dependency chains)
      double acc64[MZ];
      float acc[MZ][4];
#pragma unroll
      for (int q = 0; q < MZ; ++q) {
        acc64[q] = 0.0;
        acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
      }
      for (int j = 0; j < item.w; ++j, ++k) {
        const int buf = (int)(k & 1);
        const uint32_t s_col = 256 * buf + g * 128 + 64 * hf;
        bool ok = mbar_wait(&s_full[2 * g + buf], (sph >> buf) & 1u, abort, a.err, 16);
        // the VF tile of this stage is visible once its copy has completed
        ok = ok && mbar_wait(&full[stage], fph, abort, a.err, 17);
        if (!__all_sync(0xffffffffu, ok)) goto fma_exp_out;
        sph ^= 1u << buf;
        tc_fence_after();
        // this half's 64 columns of v: float4 16 hf .. 16 hf + 15 of each column's 32
        const float4* vs = reinterpret_cast<const float4*>(sV + stage * V_TILE) + 16 * hf;
        {
          // 32 columns at a time (registers are 96 a thread at 608 threads; the
          // other warps of the scheduler cover the second load)
          uint32_t a0[32];
          tmem_ld32(tl + s_col, a0);
          tmem_ld_wait_regs(a0);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float p0 = exp2_mix<POLY, 5>(__uint_as_float(a0[4 * u]), 4 * u);
            const float p1 = exp2_mix<POLY, 5>(__uint_as_float(a0[4 * u + 1]), 4 * u + 1);
            const float p2 = exp2_mix<POLY, 5>(__uint_as_float(a0[4 * u + 2]), 4 * u + 2);
            const float p3 = exp2_mix<POLY, 5>(__uint_as_float(a0[4 * u + 3]), 4 * u + 3);
#pragma unroll
            for (int q = 0; q < MZ; ++q) {
              const float4 v = vs[q * 32 + u];
              acc[q][0] = fmaf(p0, v.x, acc[q][0]);
              acc[q][1] = fmaf(p1, v.y, acc[q][1]);
              acc[q][2] = fmaf(p2, v.z, acc[q][2]);
              acc[q][3] = fmaf(p3, v.w, acc[q][3]);
            }
          }
          uint32_t a1[32];
          tmem_ld32(tl + s_col + 32, a1);
          tmem_ld_wait_regs(a1);
          // this half of S(k) is in registers: once both halves are, the tensor core may overwrite it
          tc_fence_before();
          mbar_arrive(&s_free[2 * g + buf]);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float p0 = exp2_mix<POLY, 5>(__uint_as_float(a1[4 * u]), 4 * u);
            const float p1 = exp2_mix<POLY, 5>(__uint_as_float(a1[4 * u + 1]), 4 * u + 1);
            const float p2 = exp2_mix<POLY, 5>(__uint_as_float(a1[4 * u + 2]), 4 * u + 2);
            const float p3 = exp2_mix<POLY, 5>(__uint_as_float(a1[4 * u + 3]), 4 * u + 3);
#pragma unroll
            for (int q = 0; q < MZ; ++q) {
              const float4 v = vs[q * 32 + 8 + u];
              acc[q][0] = fmaf(p0, v.x, acc[q][0]);
              acc[q][1] = fmaf(p1, v.y, acc[q][1]);
              acc[q][2] = fmaf(p2, v.z, acc[q][2]);
              acc[q][3] = fmaf(p3, v.w, acc[q][3]);
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[stage]);
        if (++stage == (uint32_t)S) { stage = 0; fph ^= 1; }
        if ((j % kFold) == kFold - 1) {
#pragma unroll
          for (int q = 0; q < MZ; ++q) {
            acc64[q] += (double)((acc[q][0] + acc[q][1]) + (acc[q][2] + acc[q][3]));
            acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
          }
        }
      }
      // the row sums of the two halves, first + second, through shared memory
      // (a buffer per item parity; each wait bounded like the others)
      const int par = it & 1;
      double* cb = s_comb + (size_t)(2 * g + par) * MZ * 128;
      if (hf == 1) {
        if (it >= 2) {
          // the buffer's previous contents (item it - 2) must have been read
          const bool okf = mbar_wait(&comb_free[2 * g + par], (cph >> par) & 1u, abort, a.err, 18);
          if (!__all_sync(0xffffffffu, okf)) goto fma_exp_out;
          cph ^= 1u << par;
        }
#pragma unroll
        for (int q = 0; q < MZ; ++q)
          cb[q * 128 + row] = acc64[q] + (double)((acc[q][0] + acc[q][1]) + (acc[q][2] + acc[q][3]));
        mbar_arrive(&comb_full[2 * g + par]);
      } else {
        const bool okc = mbar_wait(&comb_full[2 * g + par], (cph >> par) & 1u, abort, a.err, 18);
        if (!__all_sync(0xffffffffu, okc)) goto fma_exp_out;
        cph ^= 1u << par;
#pragma unroll
        for (int q = 0; q < MZ; ++q)
          a.part[part_idx(t, a.mz, q, rowp)] =
              (acc64[q] + (double)((acc[q][0] + acc[q][1]) + (acc[q][2] + acc[q][3]))) + cb[q * 128 + row];
        mbar_arrive(&comb_free[2 * g + par]);
      }
      ++it;
    }
  fma_exp_out:;
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kFmaMmaWarp) tmem_dealloc(tbase, 512);
}

// V tiles as FP32 columns for the FMA-pipe product: VF[c][t] = MZ x 128 floats.
__global__ void tc_prep_vf_kernel(DevLayout L, TcTables T, int chains, int64_t n_total, const float* V, int m,
                                  int mz, int T_total, const int32_t* sys_active, const float* amp, float* VF,
                                  const CgSys* cg_sys, const MscgSys* ms_sys, const MscgShift* ms_sh, int ms_m,
                                  float* ms_ps, const float* cg_r, float* cg_p) {
  const int t = blockIdx.x, c = blockIdx.y, r = threadIdx.x;
  const int b = T.tile_inst[t];
  const int s = b * chains + c;
  if (sys_active && !sys_active[s]) return;
  const int64_t nb = L.offsets[b + 1] - L.offsets[b];
  const int64_t rl = (int64_t)(t - T.inst_tile0[b]) * 128 + r;
  const bool valid = rl < nb;
  const int64_t i = L.offsets[b] + rl;
  float* dst = VF + ((size_t)c * T_total + t) * (size_t)mz * 128;
  const float am = (valid && amp) ? amp[(int64_t)c * n_total + i] : 1.f;
  if (cg_sys || ms_sys) {
    // one column inside a (multi-shift) CG iteration (V is p): p = r + beta p
    // first, as the direction update does, and the shifted directions
    // p_j = zeta_j r + beta_j p_j of the active shifts; then the tile of p
    float pv = 0.f;
    if (valid) {
      const int64_t v = (int64_t)c * n_total + i;
      const float rv = cg_r[v];
      pv = fmaf((float)(cg_sys ? cg_sys[s].beta : ms_sys[s].beta), cg_p[v], rv);
      cg_p[v] = pv;
      if (ms_sys) {
        const MscgShift* k = ms_sh + (int64_t)s * ms_m;
        for (int j = 0; j < ms_m; ++j)
          if (k[j].active) ms_ps[v * ms_m + j] = fmaf((float)k[j].beta_s, ms_ps[v * ms_m + j], (float)k[j].zeta * rv);
      }
    }
    dst[r] = valid ? pv * am : 0.f;
    return;
  }
  for (int q = 0; q < mz; ++q) dst[q * 128 + r] = valid ? V[((int64_t)c * n_total + i) * m + q] * am : 0.f;
}

// ------------------------------------------------------------------ prep kernels

// Per (instance, dimension) min and max of x as order-preserving keys; one
// block per 128-row item of the layout: a warp reduction, then a block
// reduction in shared memory, then one atomic pair per block and dimension.
__global__ void tc_center_kernel(DevLayout L, int n_inst, int d, const float* x, uint32_t* keys) {
  __shared__ uint32_t smin[kTile / 32], smax[kTile / 32];
  const int item = blockIdx.x;
  const int b = L.item_inst[item];
  const int64_t i = L.item_row0[item] + threadIdx.x;
  const bool valid = i < L.offsets[b + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < d; ++k) {
    uint32_t kmin = 0xffffffffu, kmax = 0u;
    if (valid) kmin = kmax = fkey(x[i * d + k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
      kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }
    if (lane == 0) {
      smin[w] = kmin;
      smax[w] = kmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 1; q < kTile / 32; ++q) {
        kmin = min(kmin, smin[q]);
        kmax = max(kmax, smax[q]);
      }
      if (kmax != 0u) {
        atomicMin(&keys[(size_t)b * d + k], kmin);
        atomicMax(&keys[((size_t)n_inst + b) * d + k], kmax);
      }
    }
    __syncthreads();
  }
}

// One thread per padded row: the A-side and B-side operand rows (16-bit
// elements, BF16 or F16 by split mode) of the centred, scaled points.
__global__ void tc_prep_x_kernel(DevLayout L, TcTables T, int n_inst, int chains, int d, int ard, int n_theta,
                                 int KX, int nsplit, int T_total, const float* x, const double* theta,
                                 const uint32_t* ckeys, uint8_t* XA, uint8_t* XB, int* err) {
  __shared__ float s_sc[kMaxD], s_c[kMaxD];
  const int t = blockIdx.x, c = blockIdx.y, r = threadIdx.x;
  const int b = T.tile_inst[t];
  const int s = b * chains + c;
  // scale sqrt(log2 e) / l_k and centre c_k of the tile's system, once per
  // dimension (exp in FP64, once per block, not per point)
  if (r < d) {
    const double* th = theta + (int64_t)s * n_theta;
    s_sc[r] = (float)(sqrt(2.0 * kHalfLog2e) * exp(-th[1 + (ard ? r : 0)]));
    s_c[r] = center_of(ckeys, n_inst, d, b, r);
  }
  __syncthreads();
  const int64_t nb = L.offsets[b + 1] - L.offsets[b];
  const int64_t rl = (int64_t)(t - T.inst_tile0[b]) * 128 + r;
  const bool valid = rl < nb;
  const size_t base = ((size_t)c * T_total + t) * (size_t)KX * 256;
  uint16_t* A = reinterpret_cast<uint16_t*>(XA + base);
  uint16_t* B = reinterpret_cast<uint16_t*>(XB + base);
  auto putA = [&](int kk, uint16_t v) { A[x_off(r, kk, KX) / 2] = v; };
  auto putB = [&](int kk, uint16_t v) { B[x_off(r, kk, KX) / 2] = v; };
  const bool f16 = nsplit == kSplitF16;
  // 16-bit encodings of the operand type and their values back in FP32
  auto enc = [&](float v) -> uint16_t {
    return f16 ? __half_as_ushort(__float2half_rn(v)) : __bfloat16_as_ushort(__float2bfloat16_rn(v));
  };
  auto dec = [&](uint16_t u) -> float {
    return f16 ? __half2float(__ushort_as_half(u)) : __bfloat162float(__ushort_as_bfloat16(u));
  };
  const uint16_t zero = 0, one = enc(1.f);
  if (!valid) {
    for (int kk = 0; kk < KX; ++kk) {
      putA(kk, zero);
      putB(kk, zero);
    }
    return;
  }
  const int64_t i = L.offsets[b] + rl;
  double nrm = 0.0;
  bool range_ok = true;
  for (int k = 0; k < d; ++k) {
    // xh = (x - centre) sqrt(log2 e) / l, so that -|xh_i - xh_j|^2 / 2 = -log2(e) r^2 / 2
    const float xh = (x[i * d + k] - s_c[k]) * s_sc[k];
    if (f16 && !(fabsf(xh) < 240.f)) range_ok = false;
    const uint16_t hi = enc(xh);
    const float r1 = xh - dec(hi);
    const uint16_t mid = enc(r1);
    const double hd = dec(hi), md = dec(mid);
    if (nsplit != kSplitBf3) {
      // per dimension a triple, A: [hi, lo, hi]  B: [hi, hi, lo], so that
      // column 3k of an A row holds hi and 3k + 1 holds lo of dimension k
      nrm += hd * hd + 2.0 * hd * md;
      putA(3 * k, hi);
      putA(3 * k + 1, mid);
      putA(3 * k + 2, hi);
      putB(3 * k, hi);
      putB(3 * k + 1, hi);
      putB(3 * k + 2, mid);
    } else {
      // A: [h, h, m, h, l, m]  B: [h, m, h, l, h, m]
      const uint16_t lo = enc(r1 - dec(mid));
      const double ld = dec(lo);
      nrm += hd * hd + 2.0 * hd * md + 2.0 * hd * ld + md * md;
      putA(k, hi);
      putA(d + k, hi);
      putA(2 * d + k, mid);
      putA(3 * d + k, hi);
      putA(4 * d + k, lo);
      putA(5 * d + k, mid);
      putB(k, hi);
      putB(d + k, mid);
      putB(2 * d + k, hi);
      putB(3 * d + k, lo);
      putB(4 * d + k, hi);
      putB(5 * d + k, mid);
    }
  }
  const double bias = -0.5 * nrm;
  if (f16 && !(-bias < (double)kF16BiasMax)) range_ok = false;
  if (!range_ok && err) atomicCAS(err, 0, 101);
  const uint16_t bh = enc((float)bias);
  const double r1 = bias - (double)dec(bh);
  const uint16_t bm = enc((float)r1);
  const uint16_t bl = enc((float)(r1 - (double)dec(bm)));
  const int o = (nsplit == kSplitBf3 ? 6 : 3) * d;
  putA(o + 0, one);
  putA(o + 1, one);
  putA(o + 2, one);
  putA(o + 3, bh);
  putA(o + 4, bm);
  putA(o + 5, bl);
  putB(o + 0, bh);
  putB(o + 1, bm);
  putB(o + 2, bl);
  putB(o + 3, one);
  putB(o + 4, one);
  putB(o + 5, one);
  for (int kk = o + 6; kk < KX; ++kk) {
    putA(kk, zero);
    putB(kk, zero);
  }
}

// Per (system, column) max |V| over the instance (as float bits; values >= 0 order like uints).
__global__ void tc_vmax_kernel(DevLayout L, int chains, int64_t n_total, const float* V, int m, int c0,
                               int mz, const int32_t* sys_active, const float* amp, uint32_t* vmax) {
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int s = b * chains + c;
  if (sys_active && !sys_active[s]) return;
  __shared__ uint32_t smx[kTile / 32];
  const int64_t i = L.item_row0[item] + threadIdx.x;
  const bool valid = i < L.offsets[b + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const float am = (valid && amp) ? amp[(int64_t)c * n_total + i] : 1.f;
  // per column: the block's maximum (as order-preserving bits of a
  // non-negative float) by a warp and a block reduction, then one atomic
  for (int q = 0; q < mz; ++q) {
    const float v = valid ? fabsf(V[((int64_t)c * n_total + i) * m + c0 + q] * am) : 0.f;
    const uint32_t u = __reduce_max_sync(0xffffffffu, __float_as_uint(v));
    if (lane == 0) smx[w] = u;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t mx = smx[0];
      for (int k = 1; k < kTile / 32; ++k) mx = max(mx, smx[k]);
      if (mx != 0u) atomicMax(&vmax[(int64_t)s * mz + q], mx);
    }
    __syncthreads();
  }
}

__global__ void tc_prep_v_kernel(DevLayout L, TcTables T, int chains, int64_t n_total, const float* V, int m,
                                 int c0, int mz, int MP, int T_total, const uint32_t* vmax,
                                 const int32_t* sys_active, const float* amp, uint8_t* VT) {
  const int t = blockIdx.x, c = blockIdx.y, r = threadIdx.x;
  const int b = T.tile_inst[t];
  const int s = b * chains + c;
  if (sys_active && !sys_active[s]) return;
  const int64_t nb = L.offsets[b + 1] - L.offsets[b];
  const int64_t rl = (int64_t)(t - T.inst_tile0[b]) * 128 + r;
  const bool valid = rl < nb;
  __half* dst = reinterpret_cast<__half*>(VT + ((size_t)c * T_total + t) * (size_t)MP * 256);
  const int64_t i = L.offsets[b] + rl;
  const float am = (valid && amp) ? amp[(int64_t)c * n_total + i] : 1.f;
  for (int q = 0; q < MP; ++q) {
    float v = 0.f;
    if (valid && q < mz)
      v = V[((int64_t)c * n_total + i) * m + c0 + q] * am * col_scale(vmax[(int64_t)s * mz + q]);
    dst[t_off(q, r) / 2] = __float2half_rn(v);
  }
}

// Y = alpha * sum_k part + (sigma^2 + shift) V, per 128-row tile of the product layout.
__global__ void tc_fwd_epilogue_kernel(DevLayout L, TcTables T, KmvArgs a, int c0, int mz, const double* part,
                                       const uint32_t* vmax, const int* err) {
  __shared__ double red[kTile / 32];
  __shared__ double s_alpha, s_s2;
  const int item = blockIdx.x, c = blockIdx.y;
  const int b = L.item_inst[item];
  const int s = b * a.chains + c;
  if (a.sys_active && !a.sys_active[s]) return;
  if (threadIdx.x == 0) {
    // alpha and sigma^2 of the system (FP64 exp once per block)
    const double* th = a.theta + (int64_t)s * a.n_theta;
    s_alpha = exp(th[0]);
    s_s2 = exp(th[a.n_theta - 1]);
  }
  __syncthreads();
  const int64_t i = L.item_row0[item] + threadIdx.x;
  const bool valid = i < L.offsets[b + 1];
  const int tile_in_inst = (int)((L.item_row0[item] - L.offsets[b]) / 128);
  const int p = tile_in_inst >> 1, half = tile_in_inst & 1;
  const int nk = T.inst_nk[b];
  const int64_t it0 = T.sys_item0[s] + (int64_t)p * nk;
  const int rowp = half * 128 + threadIdx.x;
  const double alpha = s_alpha, s2 = s_s2;
  const bool bad = *err != 0;
  double dot = 0.0;
  if (valid) {
    const double ai = a.amp ? alpha * (double)a.amp[(int64_t)c * a.n_total + i] : alpha;
    for (int q = 0; q < mz; ++q) {
      double acc = 0.0;
      for (int k = 0; k < nk; ++k) acc += part[part_idx((int)(it0 + k), mz, q, rowp)];
      const int col = c0 + q;
      const int64_t idx = ((int64_t)c * a.n_total + i) * a.m + col;
      const double shift = a.col_shift ? (double)a.col_shift[(int64_t)s * a.col_shift_stride + col] : 0.0;
      const double vi = (double)a.V[idx];
      // the column scale is a power of two: multiplying by its reciprocal is
      // exact, and avoids an FP64 divide per element (no column maxima: the
      // FMA-pipe product, whose probabilities and vectors are not scaled)
      const double inv_sc = vmax ? col_scale_inv(vmax[(int64_t)s * mz + q]) : 1.0;
      double y = ai * acc * inv_sc + (a.no_diag ? 0.0 : (s2 + shift) * vi);
      if (bad) y = __longlong_as_double(0x7ff8000000000000ll);
      a.Y[idx] = (float)y;
      if (a.Y64) a.Y64[idx] = y;
      dot += vi * y;
    }
  }
  if (a.dot_partial) {
    const double tsum = block_sum(dot, red);
    if (threadIdx.x == 0) {
      a.dot_partial[(int64_t)item * a.chains + c] = tsum;
      // inside a (multi-shift) CG iteration: the system's last CTA takes its
      // p.q (alpha) step
      if ((a.cg_sys || a.ms_sys) &&
          last_block_of_system(a.cg_count, s, (uint32_t)(L.inst_item0[b + 1] - L.inst_item0[b]))) {
        const double pq = sys_sum(L, b, c, a.chains, a.dot_partial, 1, 0);
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

// ------------------------------------------------------------------ host side

}  // namespace

TcState* tc_state(kmv_handle h) {
  if (!h->tc) h->tc = new TcState();
  return static_cast<TcState*>(h->tc);
}

kmv_status tc_fail(kmv_handle h, kmv_status s, const char* msg) {
  h->last_error = msg;
  return s;
}

int size_class(const Layout& L) {
  int64_t mx = 1;
  for (int b = 0; b < L.n_inst; ++b) mx = std::max<int64_t>(mx, L.offsets[b + 1] - L.offsets[b]);
  int k = 0;
  while ((int64_t(1) << (k + 1)) <= mx) ++k;
  return k;
}

TcTiles tc_tiles_for(kmv_handle h, int kind, int d, int m) {
  TcState* S = tc_state(h);
  const int nl = size_class(h->layout);
  for (const TcTuned& e : S->tuned)
    if (e.kind == kind && e.d == d && e.m == m && e.nlog2 == nl) return e.t;
  return S->tiles[kind];
}

kmv_status tc_build_plan(kmv_handle h, TcState* S, int ipsm_fwd, int ipsm_adj, cudaStream_t st) {
  const Layout& L = h->layout;
  if (ipsm_fwd <= 0) ipsm_fwd = S->plan_ipsm_fwd > 0 ? S->plan_ipsm_fwd : S->tiles[kTilesForward].items_per_sm;
  if (ipsm_adj <= 0) ipsm_adj = S->plan_ipsm_adj > 0 ? S->plan_ipsm_adj : S->tiles[kTilesAdjoint].items_per_sm;
  if (S->chains == L.chains && S->offsets == L.offsets && S->tables && S->plan_ipsm_fwd == ipsm_fwd &&
      S->plan_ipsm_adj == ipsm_adj)
    return KMV_OK;
  if (h->capturing)
    return tc_fail(h, KMV_EINVAL, "new work plan during stream capture: make the same call once before capturing");
  if (S->num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int n_inst = L.n_inst, chains = L.chains;
  S->inst_tile0.assign(n_inst + 1, 0);
  S->inst_nk.assign(n_inst, 1);
  S->tile_inst.clear();
  int64_t units = 0;
  for (int b = 0; b < n_inst; ++b) {
    const int64_t nb = L.offsets[b + 1] - L.offsets[b];
    const int ntP = (int)(2 * ((nb + 255) / 256));
    S->inst_tile0[b] = (int32_t)S->tile_inst.size();
    for (int k = 0; k < ntP; ++k) S->tile_inst.push_back(b);
    units += (int64_t)chains * (ntP / 2);
  }
  S->inst_tile0[n_inst] = (int32_t)S->tile_inst.size();
  S->T_total = (int)S->tile_inst.size();
  const int64_t target = (int64_t)S->num_sms * ipsm_fwd;
  const int64_t nk_all = units > 0 ? std::max<int64_t>(1, (target + units - 1) / units) : 1;
  S->items.clear();
  S->sys_item0.assign((size_t)n_inst * chains, 0);
  for (int b = 0; b < n_inst; ++b) {
    const int64_t nb = L.offsets[b + 1] - L.offsets[b];
    const int ntJ = (int)((nb + 127) / 128);
    const int npair = (int)((nb + 255) / 256);
    const int nk = (int)std::max<int64_t>(1, std::min<int64_t>(nk_all, ntJ));
    S->inst_nk[b] = nk;
    for (int c = 0; c < chains; ++c) {
      const int s = b * chains + c;
      S->sys_item0[s] = (int32_t)S->items.size();
      for (int p = 0; p < npair; ++p)
        for (int k = 0; k < nk; ++k) {
          const int j0 = (int)((int64_t)k * ntJ / nk), j1 = (int)((int64_t)(k + 1) * ntJ / nk);
          S->items.push_back(make_int4(s, S->inst_tile0[b] + 2 * p, S->inst_tile0[b] + j0, j1 - j0));
        }
    }
  }
  S->n_items = (int)S->items.size();
  if ((int64_t)S->items.size() > (int64_t(1) << 30)) return tc_fail(h, KMV_EINVAL, "too many tensor-core work items");
  S->sys_pref.assign((size_t)n_inst * chains + 1, 0);
  for (size_t q = 0; q < S->sys_item0.size(); ++q) S->sys_pref[q] = S->sys_item0[q];
  S->sys_pref[S->sys_item0.size()] = S->n_items;
  // Upper-triangle plan (J >= I) for the symmetric adjoint: row I of an instance
  // with T tiles has T - I tile pairs, cut into near-equal chunks of at most C
  // tiles; a system's items are ordered longest first, which the round-robin
  // assignment of items to CTAs then balances.
  {
    int64_t pairs = 0;
    for (int b = 0; b < n_inst; ++b) {
      const int64_t T = (L.offsets[b + 1] - L.offsets[b] + 127) / 128;
      pairs += (int64_t)chains * T * (T + 1) / 2;
    }
    const int64_t target_adj = (int64_t)S->num_sms * ipsm_adj;
    const int64_t C = std::max<int64_t>(8, (pairs + target_adj - 1) / std::max<int64_t>(1, target_adj));
    S->sym_items.clear();
    S->sym_pref.assign((size_t)n_inst * chains + 1, 0);
    std::vector<int4> row;
    for (int b = 0; b < n_inst; ++b) {
      const int T = (int)((L.offsets[b + 1] - L.offsets[b] + 127) / 128);
      for (int c = 0; c < chains; ++c) {
        const int s = b * chains + c;
        S->sym_pref[s] = (int32_t)S->sym_items.size();
        row.clear();
        for (int I = 0; I < T; ++I) {
          const int len = T - I;
          const int nc = (int)((len + C - 1) / C);
          for (int k = 0; k < nc; ++k) {
            const int j0 = I + (int)((int64_t)k * len / nc), j1 = I + (int)((int64_t)(k + 1) * len / nc);
            row.push_back(make_int4(s, S->inst_tile0[b] + I, S->inst_tile0[b] + j0, j1 - j0));
          }
        }
        std::stable_sort(row.begin(), row.end(), [](const int4& x, const int4& y) { return x.w > y.w; });
        S->sym_items.insert(S->sym_items.end(), row.begin(), row.end());
      }
    }
    S->sym_pref[(size_t)n_inst * chains] = (int32_t)S->sym_items.size();
    S->sym_n_items = (int)S->sym_items.size();
    if ((int64_t)S->sym_items.size() > (int64_t(1) << 30))
      return tc_fail(h, KMV_EINVAL, "too many tensor-core work items");
  }
  // upload tables
  const size_t b_items = sizeof(int4) * std::max<size_t>(1, S->items.size());
  const size_t b_ti = sizeof(int32_t) * std::max<size_t>(1, S->tile_inst.size());
  const size_t b_it0 = sizeof(int32_t) * (n_inst + 1);
  const size_t b_si = sizeof(int32_t) * std::max<size_t>(1, S->sys_item0.size());
  const size_t b_nk = sizeof(int32_t) * n_inst;
  const size_t b_pref = sizeof(int32_t) * ((size_t)n_inst * chains + 1);
  const size_t b_sym = sizeof(int4) * std::max<size_t>(1, S->sym_items.size());
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  const size_t total = al(b_items) + al(b_ti) + al(b_it0) + al(b_si) + al(b_nk) + 2 * al(b_pref) + al(b_sym);
  if (total > S->tables_bytes) {
    if (S->tables) {
      cudaDeviceSynchronize();
      cudaFree(S->tables);
      S->tables = nullptr;
      S->tables_bytes = 0;
    }
    if (cudaMalloc(&S->tables, total) != cudaSuccess) {
      cudaGetLastError();
      return tc_fail(h, KMV_ENOMEM, "tensor-core table allocation failed");
    }
    S->tables_bytes = total;
  }
  char* p = static_cast<char*>(S->tables);
  size_t o = 0;
  auto up = [&](const void* src, size_t bytes, size_t slot) -> char* {
    char* dst = p + o;
    if (bytes) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    o += al(slot);
    return dst;
  };
  S->d_items = reinterpret_cast<const int4*>(up(S->items.data(), sizeof(int4) * S->items.size(), b_items));
  S->dev.tile_inst = reinterpret_cast<const int32_t*>(up(S->tile_inst.data(), sizeof(int32_t) * S->tile_inst.size(), b_ti));
  S->dev.inst_tile0 = reinterpret_cast<const int32_t*>(up(S->inst_tile0.data(), b_it0, b_it0));
  S->dev.sys_item0 = reinterpret_cast<const int32_t*>(up(S->sys_item0.data(), sizeof(int32_t) * S->sys_item0.size(), b_si));
  S->dev.inst_nk = reinterpret_cast<const int32_t*>(up(S->inst_nk.data(), b_nk, b_nk));
  S->dev.sys_pref = reinterpret_cast<const int32_t*>(up(S->sys_pref.data(), b_pref, b_pref));
  S->dev.sym_pref = reinterpret_cast<const int32_t*>(up(S->sym_pref.data(), b_pref, b_pref));
  S->d_sym_items = reinterpret_cast<const int4*>(up(S->sym_items.data(), sizeof(int4) * S->sym_items.size(), b_sym));
  if (cudaStreamSynchronize(st) != cudaSuccess) return tc_fail(h, KMV_ECUDA, "table upload failed");
  S->offsets = L.offsets;
  S->chains = L.chains;
  S->prep_valid = false;
  S->plan_ipsm_fwd = ipsm_fwd;
  S->plan_ipsm_adj = ipsm_adj;
  return KMV_OK;
}

kmv_status tc_ensure_buf(kmv_handle h, TcState* S, size_t bytes) {
  if (bytes <= S->buf_bytes) return KMV_OK;
  if (h->capturing)
    return tc_fail(h, KMV_EINVAL,
                   "workspace would grow during stream capture: make the same call once before capturing");
  if (S->buf) {
    cudaDeviceSynchronize();
    cudaFree(S->buf);
    S->buf = nullptr;
    S->buf_bytes = 0;
  }
  S->prep_valid = false;
  const size_t want = bytes + bytes / 8 + (1 << 20);
  if (cudaMalloc(&S->buf, want) != cudaSuccess) {
    cudaGetLastError();
    return tc_fail(h, KMV_ENOMEM, "tensor-core workspace allocation failed");
  }
  S->buf_bytes = want;
  return KMV_OK;
}

size_t tc_center_bytes(const Layout& L) { return sizeof(uint32_t) * 2 * (size_t)L.n_inst * std::max(1, L.d); }

void tc_launch_center(kmv_handle h, const KmvArgs& a, uint32_t* keys, cudaStream_t st) {
  const Layout& L = h->layout;
  const size_t half = sizeof(uint32_t) * (size_t)L.n_inst * a.d;
  cudaMemsetAsync(keys, 0xff, half, st);
  cudaMemsetAsync(reinterpret_cast<uint8_t*>(keys) + half, 0, half, st);
  if (L.n_items > 0) tc_center_kernel<<<L.n_items, kTile, 0, st>>>(h->dev, L.n_inst, a.d, a.x, keys);
}

void tc_launch_prep_x(kmv_handle h, TcState* S, const KmvArgs& a, int KX, int nsplit, const uint32_t* ckeys,
                      uint8_t* XA, uint8_t* XB, int* err, cudaStream_t st) {
  tc_prep_x_kernel<<<dim3(S->T_total, h->layout.chains), 128, 0, st>>>(
      h->dev, S->dev, h->layout.n_inst, h->layout.chains, a.d, a.ard, a.n_theta, KX, nsplit, S->T_total, a.x,
      a.theta, ckeys, XA, XB, err);
}

void tc_launch_epilogue(kmv_handle h, TcState* S, const KmvArgs& a, int c0, int mz, const double* part,
                        const uint32_t* colmax, const int* err, cudaStream_t st) {
  tc_fwd_epilogue_kernel<<<dim3(h->layout.n_items, h->layout.chains), kTile, 0, st>>>(h->dev, S->dev, a, c0, mz,
                                                                                      part, colmax, err);
}

using FwdKernel = void (*)(TcFwdArgs);

// The instantiation for RM (16: register fold accumulators, 0: global) or MZ
// (FMA path) and the exp split; exp splits other than 0, 4 and 8 take the
// nearest built one.
FwdKernel fwd_kernel(bool fma, int cols, int split) {
  const int sp = split <= 0 ? 0 : (split <= 5 ? 4 : 8);
  if (fma) {
    if (cols == 1) return sp == 0 ? tc_fwd_fma_kernel<1, 0> : sp == 4 ? tc_fwd_fma_kernel<1, 4> : tc_fwd_fma_kernel<1, 8>;
    return sp == 0 ? tc_fwd_fma_kernel<2, 0> : sp == 4 ? tc_fwd_fma_kernel<2, 4> : tc_fwd_fma_kernel<2, 8>;
  }
  if (cols == 16) return sp == 0 ? tc_fwd_kernel<16, 0> : sp == 4 ? tc_fwd_kernel<16, 4> : tc_fwd_kernel<16, 8>;
  return sp == 0 ? tc_fwd_kernel<0, 0> : sp == 4 ? tc_fwd_kernel<0, 4> : tc_fwd_kernel<0, 8>;
}

cudaError_t fwd_kernels_set_smem() {
  for (bool fma : {false, true})
    for (int cols : {0, 1, 2, 16})
      for (int sp : {0, 4, 8}) {
        if (fma != (cols == 1 || cols == 2)) continue;
        const cudaError_t e =
            cudaFuncSetAttribute(fwd_kernel(fma, cols, sp), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
        if (e != cudaSuccess) return e;
      }
  return cudaSuccess;
}

kmv_status tc_forward(kmv_handle h, const KmvArgs& a, cudaStream_t st) {
  const Layout& L = h->layout;
  // one or two columns (the CG / energy products) take the FMA-pipe P.v path,
  // where the tensor pipe has room for the three-way split of the exponent
  const bool fma_path = a.m <= 2 && x_width(a.d, kSplitBf3) <= kMaxKX;
  // the CG-iteration hooks (p update, p.q step) live in the one-column FMA path
  if ((a.cg_sys || a.ms_sys) && !(fma_path && a.m == 1 && a.dot_partial))
    return tc_fail(h, KMV_EINVAL, "internal: fused CG step needs the one-column FMA-pipe product");
  const int nsplit = fma_path ? kSplitBf3 : kSplitBf2;
  const int KX = x_width(a.d, nsplit);
  if (KX > kMaxKX) return tc_fail(h, KMV_EUNSUPPORTED, "KMV_BF16_HILO supports d <= 35");
  TcState* S = tc_state(h);
  const TcTiles tl = tc_tiles_for(h, fma_path ? kTilesForwardFma : kTilesForward, a.d, a.m);
  kmv_status stt = tc_build_plan(h, S, tl.items_per_sm, 0, st);
  if (stt != KMV_OK) return stt;
  if (S->n_items == 0) return KMV_OK;
  const int n_sys = L.n_inst * L.chains;
  const size_t max_stages = tl.stages > 0 ? (size_t)std::max(2, std::min(tl.stages, 8)) : 8;
  const size_t A_TILE = (size_t)KX * 256;
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  // column chunk: as wide as shared memory allows (at least two pipeline stages)
  const size_t fixed = 1024 + 4 * A_TILE + 256;
  int mz_max = std::min(a.m, kMaxMP);
  auto stages_for = [&](int mz) {
    const size_t vt = (size_t)std::max(16, (mz + 15) / 16 * 16) * 256;
    return (int)std::min<size_t>(max_stages, (kMaxSmem - fixed - 20 * 8) / (A_TILE + vt + 16));
  };
  while (stages_for(mz_max) < 2 && mz_max > 16) mz_max = std::max(16, mz_max / 2);
  if (stages_for(mz_max) < 2) return tc_fail(h, KMV_EUNSUPPORTED, "tensor-core tiles do not fit in shared memory");
  const int MPmax = std::max(16, (mz_max + 15) / 16 * 16);
  const size_t xbytes = al((size_t)L.chains * S->T_total * A_TILE);
  const size_t vbytes = al((size_t)L.chains * S->T_total * MPmax * 256);
  const size_t mbytes = al(sizeof(uint32_t) * (size_t)n_sys * mz_max);
  const size_t pbytes = al(sizeof(double) * (size_t)S->n_items * 256 * mz_max);
  const size_t cbytes = al(tc_center_bytes(L));
  const size_t total = 2 * xbytes + vbytes + mbytes + pbytes + cbytes + 256;
  stt = tc_ensure_buf(h, S, total);
  if (stt != KMV_OK) return stt;
  uint8_t* base = static_cast<uint8_t*>(S->buf);
  uint8_t* XA = base;
  uint8_t* XB = XA + xbytes;
  uint8_t* VT = XB + xbytes;
  uint32_t* vmax = reinterpret_cast<uint32_t*>(VT + vbytes);
  double* part = reinterpret_cast<double*>(reinterpret_cast<uint8_t*>(vmax) + mbytes);
  uint32_t* ckeys = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(part) + pbytes);
  int* err = reinterpret_cast<int*>(reinterpret_cast<uint8_t*>(ckeys) + cbytes);
  if (!S->attr_set) {
    if (fwd_kernels_set_smem() != cudaSuccess) return tc_fail(h, KMV_ECUDA, "cudaFuncSetAttribute failed");
    S->attr_set = true;
  }
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return tc_fail(h, KMV_ECUDA, "memset failed");
  // the operand tiles depend on theta and x only: a solve's later products
  // reuse those of its first one
  const bool reuse = a.reuse_prep && S->prep_valid && S->prep_theta == a.theta && S->prep_x == a.x &&
                     S->prep_nsplit == nsplit && S->prep_d == a.d;
  if (!reuse) {
    tc_launch_center(h, a, ckeys, st);
    tc_launch_prep_x(h, S, a, KX, nsplit, ckeys, XA, XB, nullptr, st);
    S->prep_valid = true;
    S->prep_theta = a.theta;
    S->prep_x = a.x;
    S->prep_nsplit = nsplit;
    S->prep_d = a.d;
  }
  if (fma_path) {
    // one or two columns: P.v on the FMA pipe (FP32 P and v, no scaling)
    const int mz = a.m;
    const size_t V_TILE = (size_t)mz * 512;
    // barriers (2 per stage + 22), the TMEM slot and abort flag, and the two
    // column halves' row-sum buffers (2 I tiles x 2 item parities x mz x 128 FP64)
    const size_t tail = 24 * 8 + (size_t)4 * mz * 128 * 8;
    const int stages =
        (int)std::max<size_t>(2, std::min<size_t>(max_stages, (kMaxSmem - fixed - tail) / (A_TILE + V_TILE + 16)));
    const size_t smem = std::max(kMinSmem, fixed + stages * (A_TILE + V_TILE + 16) + tail);
    tc_prep_vf_kernel<<<dim3(S->T_total, L.chains), 128, 0, st>>>(
        h->dev, S->dev, L.chains, L.n_total, a.V, a.m, mz, S->T_total, a.sys_active, a.amp,
        reinterpret_cast<float*>(VT), a.cg_sys, a.ms_sys, a.ms_sh, a.ms_m, a.ms_ps, a.cg_r,
        const_cast<float*>(a.V));
    TcFwdArgs fa;
    fa.items = S->d_items;
    fa.n_items = S->n_items;
    fa.chains = L.chains;
    fa.T_total = S->T_total;
    fa.KX = KX;
    fa.MP = 16;
    fa.S = stages;
    fa.XA = XA;
    fa.XB = XB;
    fa.VT = VT;
    fa.part = part;
    fa.mz = mz;
    fa.sys_active = a.sys_active;
    fa.err = err;
    const int grid = std::min(S->n_items, S->num_sms);
    {
      ProfScope prof(h, KMV_KERNEL_FORWARD, st);
      fwd_kernel(true, mz, tl.exp_split)<<<grid, kFmaThreads, smem, st>>>(fa);
    }
    // no column maxima: the epilogue's column scale is 1
    tc_launch_epilogue(h, S, a, 0, mz, part, nullptr, err, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tc_fail(h, KMV_ECUDA, cudaGetErrorString(e));
    return KMV_OK;
  }
  for (int c0 = 0; c0 < a.m; c0 += mz_max) {
    const int mz = std::min(mz_max, a.m - c0);
    const int MP = std::max(16, (mz + 15) / 16 * 16);
    const size_t V_TILE = (size_t)MP * 256;
    const int stages = stages_for(mz);
    const size_t smem = std::max(kMinSmem, fixed + stages * (A_TILE + V_TILE) + (2 * stages + 20) * 8);
    if (cudaMemsetAsync(vmax, 0, sizeof(uint32_t) * (size_t)n_sys * mz, st) != cudaSuccess)
      return tc_fail(h, KMV_ECUDA, "memset failed");
    tc_vmax_kernel<<<dim3(L.n_items, L.chains), kTile, 0, st>>>(h->dev, L.chains, L.n_total, a.V, a.m, c0, mz,
                                                                a.sys_active, a.amp, vmax);
    tc_prep_v_kernel<<<dim3(S->T_total, L.chains), 128, 0, st>>>(h->dev, S->dev, L.chains, L.n_total, a.V, a.m, c0,
                                                                 mz, MP, S->T_total, vmax, a.sys_active, a.amp, VT);
    TcFwdArgs fa;
    fa.items = S->d_items;
    fa.n_items = S->n_items;
    fa.chains = L.chains;
    fa.T_total = S->T_total;
    fa.KX = KX;
    fa.MP = MP;
    fa.S = stages;
    fa.XA = XA;
    fa.XB = XB;
    fa.VT = VT;
    fa.part = part;
    fa.mz = mz;
    fa.sys_active = a.sys_active;
    fa.err = err;
    const int grid = std::min(S->n_items, S->num_sms);
    {
      ProfScope prof(h, KMV_KERNEL_FORWARD, st);
      fwd_kernel(false, MP <= 16 ? 16 : 0, tl.exp_split)<<<grid, kFwdThreads, smem, st>>>(fa);
    }
    tc_launch_epilogue(h, S, a, c0, mz, part, vmax, err, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tc_fail(h, KMV_ECUDA, cudaGetErrorString(e));
  }
  return KMV_OK;
}

bool x_width_fma_ok(int d) { return x_width(d, kSplitBf3) <= kMaxKX; }

void tc_release(kmv_handle h) {
  if (!h->tc) return;
  TcState* S = static_cast<TcState*>(h->tc);
  if (S->buf) cudaFree(S->buf);
  if (S->tables) cudaFree(S->tables);
  delete S;
  h->tc = nullptr;
}

size_t tc_workspace_bytes(kmv_handle h) {
  if (!h->tc) return 0;
  const TcState* S = static_cast<const TcState*>(h->tc);
  return S->buf_bytes + S->tables_bytes;
}

}  // namespace kmv

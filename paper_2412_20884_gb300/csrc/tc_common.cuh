// Host plan, shared state and device helpers of the tensor-core kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "exp2_poly.cuh"
#include "kmv_internal.cuh"

namespace kmv {

constexpr int kThreads = 320;      // 2 exp warpgroups + MMA warp + producer warp
constexpr int kMmaWarp = 8;
constexpr int kLoadWarp = 9;
constexpr int kMaxKX = 112;        // d <= 35 (X operand width, BF16 elements)
constexpr int kMaxMP = 64;         // forward columns per pass (O_g holds 64 TMEM columns)
constexpr size_t kMinSmem = 120 * 1024;  // keeps one CTA (and one TMEM allocation) per SM
constexpr size_t kMaxSmem = 227 * 1024;

__host__ __device__ constexpr int round16(int v) { return (v + 15) / 16 * 16; }
// How the X operand tiles carry xh (the scaled, centred point):
//   kSplitBf2: xh = hi + lo in BF16, products hi.hi + hi.lo + lo.hi (|dS| ~ 2^-16 |xh|^2)
//   kSplitBf3: xh = h + m + l in BF16, six products (|dS| ~ 2^-24 |xh|^2)
//   kSplitF16: xh = hi + lo in F16, three products (|dS| ~ 2^-24 |xh|^2 at the
//              depth of kSplitBf2; needs |xh_k| < 240 and |xh|^2 / 2 < 2^15)
constexpr int kSplitBf2 = 2, kSplitBf3 = 3, kSplitF16 = 4;
// X operand width: 3 d (two-way splits) or 6 d (three-way split) product terms
// + 6 bias/one columns, rounded to the MMA K step.
__host__ __device__ constexpr int x_width(int d, int nsplit = kSplitBf2) {
  return round16((nsplit == kSplitBf3 ? 6 : 3) * d + 6);
}
// Largest |xh|^2 / 2 the F16 operands hold (the bias is split in three F16 terms).
constexpr float kF16BiasMax = 32768.f;

struct TcTables {
  const int32_t* tile_inst;    // T_total
  const int32_t* inst_tile0;   // n_inst + 1 (padded tiles)
  const int32_t* sys_item0;    // n_sys
  const int32_t* inst_nk;      // n_inst
  const int32_t* sys_pref;     // n_sys + 1: items of system s are [sys_pref[s], sys_pref[s + 1])
  const int32_t* sym_pref;     // n_sys + 1, the same for the upper-triangle plan
};



// Tile choices of one tensor-core kernel (kmv_tiles of the C ABI).
struct TcTiles {
  int stages = 0;        // operand-ring stages, 0 = as many as shared memory holds
  int items_per_sm = 6;  // work items per SM the plan aims at
  int exp_split = 0;     // 0: every exp on the MUFU; k: one element in k on the FMA pipe
};
// kernel kinds of the tile table (kmv_tile_kernel)
constexpr int kTilesForward = 0, kTilesForwardFma = 1, kTilesAdjoint = 2, kTilesKinds = 3;
// A tuned choice for one call shape: kernel kind, d, columns per launch and
// the largest instance's size class (floor(log2 N_b)).
struct TcTuned {
  int kind, d, m, nlog2;
  TcTiles t;
  double ms;
};

struct TcState {
  // tile choices: per-kernel defaults, and tuned entries matched by shape
  TcTiles tiles[kTilesKinds];
  std::vector<TcTuned> tuned;
  // plan key
  std::vector<int64_t> offsets;
  int chains = -1;
  int plan_ipsm_fwd = -1, plan_ipsm_adj = -1;
  // plan
  int T_total = 0, n_items = 0;
  std::vector<int4> items;
  std::vector<int32_t> tile_inst, inst_tile0, sys_item0, inst_nk, sys_pref;
  // upper-triangle plan of the symmetric adjoint: {system, I tile, first J tile >= I, J tiles}
  int sym_n_items = 0;
  std::vector<int4> sym_items;
  std::vector<int32_t> sym_pref;
  const int4* d_sym_items = nullptr;
  void* tables = nullptr;
  size_t tables_bytes = 0;
  TcTables dev{};
  const int4* d_items = nullptr;
  // buffers
  void* buf = nullptr;
  size_t buf_bytes = 0;
  int* err = nullptr;
  // what the XA / XB tiles at the start of the workspace hold (tc_forward):
  // valid only until another tensor-core call or a workspace change
  bool prep_valid = false;
  const double* prep_theta = nullptr;
  const float* prep_x = nullptr;
  int prep_nsplit = 0, prep_d = 0;
  int num_sms = 0;
  bool attr_set = false;
  bool bwd_attr_set = false;
  bool fma_attr_set = false;
};


TcState* tc_state(kmv_handle h);
// The tiles a call of the given kernel kind and shape runs with: a tuned entry
// for (kind, d, m, size class of the largest instance), else the default.
TcTiles tc_tiles_for(kmv_handle h, int kind, int d, int m);
kmv_status tc_fail(kmv_handle h, kmv_status s, const char* msg);
// Builds (or keeps) the work plans of the forward and the symmetric adjoint for
// the handle's layout, aiming at ipsm_* work items per SM (<= 0: keep the
// current value, else the default).
kmv_status tc_build_plan(kmv_handle h, TcState* S, int ipsm_fwd, int ipsm_adj, cudaStream_t st);
kmv_status tc_ensure_buf(kmv_handle h, TcState* S, size_t bytes);
// Per-instance centre of the points: c_k = (min_k + max_k) / 2 over the
// instance's rows.  The kernel depends on differences only, so centring is
// exact; it shrinks |xh| and with it the rounding of the expanded exponent
// S = xh_i.xh_j - |xh_i|^2/2 - |xh_j|^2/2.  Min and max are kept as
// order-preserving integer keys, so the atomics give the same centre in any
// order.  keys: 2 n_inst d words, [min keys | max keys].
size_t tc_center_bytes(const Layout& L);
void tc_launch_center(kmv_handle h, const KmvArgs& a, uint32_t* keys, cudaStream_t st);
// Writes the XA / XB operand tiles of every (chain, padded tile) in the given
// split mode (kSplit*), from the centred points.  err (kSplitF16 only): set to
// 101 when a row leaves the F16 range.
void tc_launch_prep_x(kmv_handle h, TcState* S, const KmvArgs& a, int KX, int nsplit, const uint32_t* ckeys,
                      uint8_t* XA, uint8_t* XB, int* err, cudaStream_t st);
// Y = alpha * sum_k part / colscale + (sigma^2 + shift) V over the product rows of a.
void tc_launch_epilogue(kmv_handle h, TcState* S, const KmvArgs& a, int c0, int mz, const double* part,
                        const uint32_t* colmax, const int* err, cudaStream_t st);

// Order-preserving map float -> uint32 (larger float, larger key), and back.
__device__ __forceinline__ uint32_t fkey(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_dec(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
// Centre of dimension k of instance b from the keys of tc_launch_center.
__device__ __forceinline__ float center_of(const uint32_t* keys, int n_inst, int d, int b, int k) {
  return 0.5f * (fkey_dec(keys[(size_t)b * d + k]) + fkey_dec(keys[((size_t)n_inst + b) * d + k]));
}

// 2^s for s <= 0 on the FMA pipe, the companion of the MUFU ex2 for a share of
// the elements.  s = n + f with n = round(s) and |f| <= 1/2 (the reduction of
// Cody and Waite; for base 2 it is exact), n taken from the low bits of
// s + 1.5 2^23, 2^f from the degree-DEG minimax polynomial of exp2_poly.cuh
// (Horner), and 2^n added to the exponent field.  Arguments below -125 give
// 2^-125 or less (the products treat them as 0).
template <int DEG>
__device__ __forceinline__ float exp2_fma(float s) {
  static_assert(DEG == 3 || DEG == 5, "exp2_poly.cuh holds degrees 3 and 5");
  const float t = fmaxf(s, -125.f);
  const float r = __fadd_rn(t, 12582912.f);
  const float f = __fsub_rn(t, __fsub_rn(r, 12582912.f));
  const float p = DEG == 3 ? exp2_poly3(f) : exp2_poly5(f);
  return __uint_as_float(__float_as_uint(p) + (__float_as_uint(r) << 23));
}

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// Byte offset of element (row r, K index kk) in a K-major, no-swizzle operand
// tile of 128 rows and K = width elements of 16 bits.
__device__ __forceinline__ uint32_t x_off(int r, int kk, int width) {
  return (r & 7) * 16 + (r >> 3) * (width * 16) + (kk & 7) * 2 + (kk >> 3) * 128;
}
// Byte offset of element (row q, K index j) in a K-major tile whose K is the
// 128 rows of a point tile (V^T-like operands): 16 K chunks per 8-row group.
__device__ __forceinline__ uint32_t t_off(int q, int j) {
  return (q & 7) * 16 + (q >> 3) * 2048 + (j & 7) * 2 + (j >> 3) * 128;
}

// Power-of-two scale putting the column's max |V| just below 2^14 (F16 range).
__device__ __forceinline__ float col_scale(uint32_t bits) {
  const float mx = __uint_as_float(bits);
  if (!(mx > 0.f) || !isfinite(mx)) return 1.f;
  int e;
  frexpf(mx, &e);  // mx = f 2^e, f in [0.5, 1)
  return ldexpf(1.f, 14 - e);
}

// Running sum as an unevaluated pair s + c: each addition's rounding error,
// recovered exactly by Knuth's TwoSum, is added to c, so (double)s + (double)c
// differs from the exact sum of the terms by about u^2 times the sum of their
// magnitudes (u = 2^-24) instead of u times it.
__device__ __forceinline__ void two_sum_add(float& s, float& c, float x) {
  const float t = __fadd_rn(s, x);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
  c = __fadd_rn(c, err);
  s = t;
}

// 1 / col_scale(bits), exactly (a power of two, formed from its exponent).
__device__ __forceinline__ double col_scale_inv(uint32_t bits) {
  const float mx = __uint_as_float(bits);
  if (!(mx > 0.f) || !isfinite(mx)) return 1.0;
  int e;
  frexpf(mx, &e);
  return __longlong_as_double((long long)(1023 + e - 14) << 52);
}


}  // namespace kmv

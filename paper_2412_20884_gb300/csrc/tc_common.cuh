// Host plan, shared state and device helpers of the tensor-core kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

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
// X operand width: 3 d (two-way split) or 6 d (three-way split) product terms
// + 6 bias/one columns, rounded to the MMA K step.
__host__ __device__ constexpr int x_width(int d, int nsplit = 2) { return round16((nsplit == 3 ? 6 : 3) * d + 6); }

struct TcTables {
  const int32_t* tile_inst;    // T_total
  const int32_t* inst_tile0;   // n_inst + 1 (padded tiles)
  const int32_t* sys_item0;    // n_sys
  const int32_t* inst_nk;      // n_inst
  const int32_t* sys_pref;     // n_sys + 1: items of system s are [sys_pref[s], sys_pref[s + 1])
  const int32_t* sym_pref;     // n_sys + 1, the same for the upper-triangle plan
};



struct TcState {
  // plan key
  std::vector<int64_t> offsets;
  int chains = -1;
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
  int num_sms = 0;
  bool attr_set = false;
  bool bwd_attr_set = false;
  bool fma_attr_set = false;
};


TcState* tc_state(kmv_handle h);
kmv_status tc_fail(kmv_handle h, kmv_status s, const char* msg);
kmv_status tc_build_plan(kmv_handle h, TcState* S, cudaStream_t st);
kmv_status tc_ensure_buf(kmv_handle h, TcState* S, size_t bytes);
// Writes the XA / XB operand tiles of every (chain, padded tile).
// nsplit = 2: x = hi + lo, products hi.hi + hi.lo + lo.hi (|dS| ~ 2^-16 |x|^2);
// nsplit = 3: x = h + m + l, products hh + hm + mh + hl + lh + mm (|dS| ~ 2^-24 |x|^2).
void tc_launch_prep_x(kmv_handle h, TcState* S, const KmvArgs& a, int KX, int nsplit, uint8_t* XA, uint8_t* XB,
                      cudaStream_t st);
// Y = alpha * sum_k part / colscale + (sigma^2 + shift) V over the product rows of a.
void tc_launch_epilogue(kmv_handle h, TcState* S, const KmvArgs& a, int c0, int mz, const double* part,
                        const uint32_t* colmax, const int* err, cudaStream_t st);

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


}  // namespace kmv

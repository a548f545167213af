// Internal declarations shared by the CUDA translation units of libkmv.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "kmv.h"

namespace kmv {

// Rows per work item of the SIMT kernels and of the reductions built on them.
constexpr int kTile = 128;
constexpr int kMaxD = 64;
// Columns of V handled by one SIMT pass (forward / backward).
constexpr int kMaxMPFwd = 64;
constexpr int kMaxJSplit = 16;   // J-range chunks of the FP32 forward at small sizes
constexpr int kMaxMPBwd = 32;
// exp(-r^2/2) = 2^(-h r^2) with h = log2(e)/2; points are pre-scaled by sqrt(h)/l.
constexpr double kHalfLog2e = 0.72134752044448170368;
// The SIMT kernels fold FP32 partial sums into FP64 accumulators every
// kFoldTiles * kTile columns.
constexpr int kFoldTiles = 4;

// Host description of one call's point set and its row-tile work items.
struct Layout {
  int n_inst = 0, chains = 0, d = 0, ard = 0, n_theta = 0;
  // Chebyshev-amplitude family (Sec. 4): N_cheb (0: the SE kernel of Sec. 1),
  // N_cheb^d coefficients, and the stationary parameter count used inside
  int cheb = 0, n_coef = 0, n_theta_int = 0;
  int64_t n_total = 0;
  int n_items = 0;
  int max_items_per_inst = 0;
  std::vector<int64_t> offsets;     // n_inst + 1
  std::vector<int32_t> item_inst;   // n_items
  std::vector<int64_t> item_row0;   // n_items
  std::vector<int32_t> inst_item0;  // n_inst + 1 prefix over items
};

// Device copies of a Layout's tables (owned by the handle, cached).
struct DevLayout {
  const int64_t* offsets = nullptr;
  const int32_t* item_inst = nullptr;
  const int64_t* item_row0 = nullptr;
  const int32_t* inst_item0 = nullptr;
};

// Per-(system, column) state of the multi-column CG (kmv_mcg.cu).
struct McgCol {
  double rr, bb, alpha, beta, rz;   // rz: r.z of the preconditioned form
  int32_t iters, status, active;
  int32_t pad;  // refinement: 1 when the column's last correction is to be taken back
};

// Multi-shift CG state (kmv_mscg.cu): per system, and per (system, shift).
constexpr int kMaxShifts = 32;
struct MscgSys {
  double rr, bb, alpha, beta, alpha_prev, beta_prev;
  int32_t iters, pad;
};
struct MscgShift {
  double sigma, zeta, zeta_prev, zeta_next, alpha_s, beta_s;
  int32_t active, iters, status, pad;
};

// Per-system CG state, kept in the handle workspace.
struct CgSys {
  double rr, bb, pq, alpha, beta;
  int32_t iters, status;
};

// ---------------------------------------------------------------------------
// Kernel argument blocks
// ---------------------------------------------------------------------------
struct KmvArgs {
  DevLayout L;
  int chains, d, ard, n_theta;
  int64_t n_total;
  const float* x;
  const double* theta;
  const float* V;       // (chains, N, m)
  const float* G;       // backward seed (chains, N, m)
  int m;
  const float* col_shift;
  int col_shift_stride;  // 0: col_shift[c] for every system; else col_shift[s * stride + c]
  float* Y;             // forward output / backward dL/dV
  double* Y64;
  const int32_t* sys_active;   // optional mask: skip systems with 0
  double* dot_partial;         // forward m == 1: per-item sum_i V_i Y_i
  double* grad_partial;        // backward: per-(item, chain, z) partial sums
  int n_z;                     // column chunks
  // Chebyshev-amplitude family (Sec. 4): K_ij = amp_i amp_j K0_ij with
  // amp = exp(C_theta(x)) per (chain, point), laid out (chains, N_total); NULL = 1.
  const float* amp;
  int no_diag;                 // forward: leave out the (sigma^2 + shift) V term
  // forward, tensor-core form: the operand tiles of (theta, x) prepared by the
  // previous product of the same solve may be reused (theta and x unchanged)
  int reuse_prep;
  // forward, one-column product inside a CG iteration (cg_sys set): the CTA of
  // each system that finishes its epilogue last takes the system's p.q step
  // (alpha, or stopping it: cg_active, cg_n_active; cg_count holds one zeroed
  // counter per system), and the tensor-core FMA-pipe product first forms
  // p = r + beta p in place (V is p, r is cg_r).
  CgSys* cg_sys;
  int32_t* cg_active;
  int32_t* cg_n_active;
  uint32_t* cg_count;
  const float* cg_r;
  // the same inside a multi-shift CG iteration (ms_sys set; cg_active,
  // cg_n_active, cg_count and cg_r as above): the last CTA takes the system's
  // alpha step for its ms_m shifts, and the tensor-core FMA-pipe product first
  // forms p = r + beta p and p_j = zeta_j r + beta_j p_j (ms_ps, (chains,
  // N_total, ms_m)).
  MscgSys* ms_sys;
  MscgShift* ms_sh;
  int ms_m;
  float* ms_ps;
};

// The argument rules of a point set and chain count shared by every entry
// point (kmv_api.cu): nullptr when they hold, else what is wrong.
const char* points_error(const kmv_points* pts, int32_t chains);

// SIMT kernels (kmv_simt.cu)
// jsplit > 1 splits each system's J range into jsplit chunks of whole J
// tiles, with per-chunk FP64 row sums in jpart (jsplit * chains * N_total * m
// doubles) added in chunk order by a combine kernel.
cudaError_t launch_forward_simt(const KmvArgs& a, int n_items, int jsplit, double* jpart, cudaStream_t st);
// The J split for a grid of n_items * chains * column chunks CTAs: 1 from two
// CTAs per SM up, else about two CTAs per SM with at least two J tiles (of
// the largest instance, max_rows) per chunk, at most kMaxJSplit.
int forward_jsplit(int n_items, int chains, int m, int64_t max_rows, int num_sms);
cudaError_t launch_backward_simt(const KmvArgs& a, int n_items, cudaStream_t st);
int backward_mp(int m);      // columns per backward pass
int forward_mp(int m);

// Gradient finalisation: sums partials per system in a fixed order and scales.
cudaError_t launch_grad_finalize(const DevLayout& L, int n_inst, int chains, int n_theta,
                                 int ard, int d, int n_z, const double* theta,
                                 const double* partial, double* grad, cudaStream_t st);

// CG / leapfrog / energy kernels (kmv_cg.cu)
cudaError_t launch_cg_init(const DevLayout& L, int n_items, int chains, int64_t n_total,
                           const float* rhs, int64_t rhs_stride, const float* q,
                           float* x, float* r, float* p, int warm, double* partial2, cudaStream_t st);
cudaError_t launch_cg_reduce_init(const DevLayout& L, int n_inst, int chains, const double* partial2,
                                  double tol, CgSys* sys, int32_t* active, int32_t* n_active,
                                  cudaStream_t st);
cudaError_t launch_cg_reduce_pq(const DevLayout& L, int n_inst, int chains, const double* partial,
                                CgSys* sys, int32_t* active, cudaStream_t st);
// cg_update_xr followed, per system, by the r.r step of cg_reduce_rr in the CTA
// that finishes last (count: one zeroed counter per system).
cudaError_t launch_cg_update_xr_rr(const DevLayout& L, int n_items, int chains, int64_t n_total, CgSys* sys,
                                   int32_t* active, float* x, float* r, const float* p, const float* q,
                                   double* partial, uint32_t* count, double tol, int maxiter, int32_t* n_active,
                                   cudaStream_t st);
cudaError_t launch_cg_update_xr(const DevLayout& L, int n_items, int chains, int64_t n_total,
                                const CgSys* sys, const int32_t* active, float* x, float* r,
                                const float* p, const float* q, double* partial, cudaStream_t st);
cudaError_t launch_cg_reduce_rr(const DevLayout& L, int n_inst, int chains, const double* partial,
                                double tol, int maxiter, CgSys* sys, int32_t* active,
                                int32_t* n_active, cudaStream_t st);
cudaError_t launch_cg_update_p(const DevLayout& L, int n_items, int chains, int64_t n_total,
                               const CgSys* sys, const int32_t* active, const float* r, float* p,
                               cudaStream_t st);
cudaError_t launch_cg_finish(int n_sys, const CgSys* sys, int32_t* status, int32_t* iters,
                             cudaStream_t st);
// Sets the value of a graph's conditional handle to (*n_active > 0): the test
// of a captured solver loop (a WHILE node repeats its body while it is 1).
cudaError_t launch_loop_cond(cudaGraphConditionalHandle cond, const int32_t* n_active, cudaStream_t st);

cudaError_t launch_mask_rows(const DevLayout& L, int n_items, int chains, int64_t n_total, const int32_t* active,
                             float* r, cudaStream_t st);
cudaError_t launch_axpy(int64_t n, const float* dx, float* x, cudaStream_t st);
cudaError_t launch_refine_merge(int n_sys, const int32_t* in_status, const int32_t* in_iters, int32_t* status,
                                int32_t* iters, cudaStream_t st);
cudaError_t launch_refine_stagnation(int n_sys, int outer, const CgSys* sys, double* prev_rr, int32_t* active,
                                     int32_t* n_active, double* worst, cudaStream_t st);
cudaError_t launch_refine_finish(int n_sys, const int32_t* active, const CgSys* sys, double tol, int32_t* status,
                                 cudaStream_t st);
// phi refresh (kmv_phi.cu): spectral interval, pole weights/shifts, weighted
// sum of the shifted solutions, per-system status
cudaError_t launch_phi_fill(float* v, int64_t n, float val, cudaStream_t st);
cudaError_t launch_phi_bounds(DevLayout L, int n_sys, int chains, int64_t n_total, const float* Y, double slack,
                              double* bounds, cudaStream_t st);
cudaError_t launch_phi_poles(int n_sys, int n_theta, int n_poles, const double* theta, const double* bounds,
                             float* shifts, double* weights, double* poles_out, cudaStream_t st);
cudaError_t launch_phi_combine(DevLayout L, int n_items, int chains, int n_poles, int64_t n_total,
                               const double* weights, const float* x_p, float* phi, cudaStream_t st);
cudaError_t launch_phi_status(int n_sys, int n_poles, const int32_t* col_status, const int32_t* col_iters,
                              int32_t* status, int32_t* iters, cudaStream_t st);

// Randomized Nystrom preconditioner (kmv_nystrom.cu) and preconditioned CG (kmv_pcg.cu)
constexpr int kMaxRank = 128;
struct PcgSys {
  double rr, bb, rz, alpha, beta;
  int32_t iters, status;
};
struct PcgPrecond {
  int rank;
  const float* U;     // (chains, rank, N_total)
  const double* lam;  // (n_sys, rank), descending
};
cudaError_t launch_nystrom_finish(const DevLayout& L, int n_items, int n_inst, int chains, int64_t n_total, int r,
                                  const float* Om, const float* Y, double* grams, double* scratch, double* T,
                                  double* nu, float* U, double* lam, int32_t* status, cudaStream_t st);
cudaError_t launch_pcg_init(const DevLayout& L, int n_items, int chains, int64_t n_total, const float* rhs,
                            int64_t rhs_stride, const float* q, float* x, float* r, int warm, double* partial2,
                            cudaStream_t st);
cudaError_t launch_pcg_precond(const DevLayout& L, int n_items, int n_inst, int chains, int64_t n_total,
                               const PcgPrecond& P, const double* theta, int n_theta, const float* r, float* z,
                               const int32_t* active, double* proj, double* coef, double* prz, cudaStream_t st);
cudaError_t launch_pcg_setup(const DevLayout& L, int n_inst, int chains, const double* partial2, const double* prz,
                             double tol, PcgSys* sys, int32_t* active, int32_t* n_active, cudaStream_t st);
cudaError_t launch_pcg_alpha(const DevLayout& L, int n_inst, int chains, const double* partial, PcgSys* sys,
                             int32_t* active, cudaStream_t st);
cudaError_t launch_pcg_update_xr(const DevLayout& L, int n_items, int chains, int64_t n_total, const PcgSys* sys,
                                 const int32_t* active, float* x, float* r, const float* p, const float* q,
                                 double* partial, cudaStream_t st);
cudaError_t launch_pcg_beta(const DevLayout& L, int n_inst, int chains, const double* prr, const double* prz,
                            double tol, int maxiter, PcgSys* sys, int32_t* active, int32_t* n_active,
                            cudaStream_t st);
cudaError_t launch_pcg_update_p(const DevLayout& L, int n_items, int chains, int64_t n_total, const PcgSys* sys,
                                const int32_t* active, const float* z, float* p, cudaStream_t st);
cudaError_t launch_pcg_finish(int n_sys, const PcgSys* sys, const int32_t* active, int32_t* status, int32_t* iters,
                              cudaStream_t st);

// Metropolis test (kmv_cg.cu)
cudaError_t launch_status_merge(int n, const int32_t* src, int32_t* dst, cudaStream_t st);
cudaError_t launch_accept(int n_sys, int n_theta, const double* H_old, const double* H_new, const double* u,
                          const int32_t* status, const double* theta_old, double* theta, int32_t* accepted,
                          cudaStream_t st);

// Implicit midpoint step by Anderson acceleration (kmv_implicit.cu)
constexpr int kMaxAA = 16;
cudaError_t launch_fill_i32(int32_t* v, int n, int32_t val, cudaStream_t st);
cudaError_t launch_imp_mid(int n, const double* th0, const double* th, double* tb, cudaStream_t st);
cudaError_t launch_imp_resid(const DevLayout& L, int n_items, int chains, int64_t n_total, const float* y,
                             const float* q, const int32_t* active, float* r, double* partial2, cudaStream_t st);
cudaError_t launch_imp_x(const DevLayout& L, int n_items, int chains, int64_t n_total, int k, int slot, int cnt,
                         const float* x, const float* z, const double* cscale, const int32_t* active, float* Gx,
                         float* Fx, double* partial, cudaStream_t st);
cudaError_t launch_imp_aa(const DevLayout& L, int n_inst, int chains, int n, int k, int slot, int cnt,
                          const double* th0, const double* pi0, const double* th, const double* pi,
                          const double* grad, const double* mu, const double* prec, const uint8_t* mask, double dt,
                          const double* xpart, const double* rpart, double tol, int iter, int maxiter, double* Gtp,
                          double* Ftp, double* H, double* alpha, int32_t* active, int32_t* done_now, int32_t* status,
                          int32_t* iters, int32_t* n_active, double* best_rr, int32_t* best_it, cudaStream_t st);
cudaError_t launch_imp_mix(const DevLayout& L, int n_items, int n_inst, int chains, int64_t n_total, int n, int k,
                           int slot, int cnt, const double* Gtp, const float* Gx, const double* alpha,
                           const int32_t* active, const int32_t* done_now, double* th, double* pi, float* x,
                           cudaStream_t st);
cudaError_t launch_imp_scale(const DevLayout& L, int n_items, int chains, int64_t n_total, const double* norm,
                             const float* w, float* v, double* partial, cudaStream_t st);
cudaError_t launch_imp_norm(const DevLayout& L, int n_inst, int chains, const double* partial, double* cscale,
                            cudaStream_t st);
cudaError_t launch_imp_cfinal(int n_sys, double safety, double* cscale, cudaStream_t st);

// Chebyshev-amplitude kernel family (kmv_cheb.cu)
constexpr int kMaxChebOrder = 32;   // N_cheb
constexpr int kMaxChebDims = 8;     // d when N_cheb >= 2
constexpr int kMaxChebCoef = 1024;  // N_cheb^d
int cheb_n_coef(int n_cheb, int d);  // N_cheb^d, or -1 above kMaxChebCoef
cudaError_t launch_cheb_prepare(const DevLayout& L, int n_items, int n_sys, int chains, int64_t n_total, int d,
                                int n_cheb, int n_coef, int n_theta, int n_theta_int, const float* x,
                                const double* theta, double* theta_int, float* amp, cudaStream_t st);
cudaError_t launch_cheb_grad(const DevLayout& L, int n_items, int n_inst, int chains, int64_t n_total, int d,
                             int n_cheb, int n_coef, int n_theta, int n_theta_int, int m, const float* x,
                             const float* V, const float* G, const float* KV, const float* KG,
                             const int32_t* sys_active, double* partial, const double* grad_int, double* grad,
                             cudaStream_t st);

// multi-shift CG (kmv_mscg.cu)
cudaError_t launch_mscg_init(const DevLayout& L, int n_items, int chains, int64_t n_total, int m, const float* b,
                             float* r, float* p, float* xs, float* ps, double* partial, cudaStream_t st);
cudaError_t launch_mscg_setup(const DevLayout& L, int n_inst, int chains, int m, const double* partial,
                              const float* shifts, double tol, MscgSys* sys, MscgShift* sh, float* base_shift,
                              int32_t* sys_active, int32_t* n_active, cudaStream_t st);
cudaError_t launch_mscg_alpha(const DevLayout& L, int n_inst, int chains, int m, const double* partial, MscgSys* sys,
                              MscgShift* sh, int32_t* sys_active, cudaStream_t st);
cudaError_t launch_mscg_update_xr(const DevLayout& L, int n_items, int chains, int64_t n_total, int m,
                                  const MscgSys* sys, const MscgShift* sh, const int32_t* sys_active, float* r,
                                  const float* q, float* xs, const float* ps, double* partial, cudaStream_t st);
cudaError_t launch_mscg_beta(const DevLayout& L, int n_inst, int chains, int m, const double* partial, double tol,
                             int maxiter, MscgSys* sys, MscgShift* sh, int32_t* sys_active, int32_t* n_active,
                             cudaStream_t st);
// mscg_update_xr followed, per system, by the beta step in the CTA that
// finishes last (count: one zeroed counter per system; n_active decremented).
cudaError_t launch_mscg_update_xr_beta(const DevLayout& L, int n_items, int chains, int64_t n_total, int m,
                                       MscgSys* sys, MscgShift* sh, int32_t* sys_active, float* r, const float* q,
                                       float* xs, const float* ps, double* partial, uint32_t* count, double tol,
                                       int maxiter, int32_t* n_active, cudaStream_t st);
cudaError_t launch_mscg_update_p(const DevLayout& L, int n_items, int chains, int64_t n_total, int m,
                                 const MscgSys* sys, const MscgShift* sh, const int32_t* sys_active, const float* r,
                                 float* p, float* ps, cudaStream_t st);
cudaError_t launch_mscg_finish(int64_t n_cols, const MscgShift* sh, int32_t* col_status, int32_t* col_iters,
                               cudaStream_t st);

// multi-column CG (kmv_mcg.cu)
cudaError_t launch_mcg_init(const DevLayout& L, int n_items, int chains, int64_t n_total, int m, const float* b,
                            int b_cols, const float* q, int warm, float* x, float* r, float* p, double* partial2,
                            cudaStream_t st);
cudaError_t launch_mcg_reduce_init(const DevLayout& L, int n_inst, int chains, int m, const double* partial2,
                                   double tol, McgCol* st, int32_t* sys_any, int32_t* n_active, cudaStream_t s);
cudaError_t launch_mcg_dot(const DevLayout& L, int n_items, int chains, int64_t n_total, int m, const float* p,
                           const float* q, const int32_t* sys_any, double* partial, cudaStream_t st);
cudaError_t launch_mcg_alpha(const DevLayout& L, int n_inst, int chains, int m, const double* partial, McgCol* st,
                             const int32_t* sys_any, int pre, cudaStream_t s);
cudaError_t launch_mcg_update_xr(const DevLayout& L, int n_items, int chains, int64_t n_total, int m,
                                 const McgCol* stt, const int32_t* sys_any, float* x, float* r, const float* p,
                                 const float* q, double* partial, cudaStream_t st);
cudaError_t launch_mcg_beta(const DevLayout& L, int n_inst, int chains, int m, const double* partial,
                            const double* prz, double tol, int maxiter, McgCol* st, int32_t* sys_any,
                            int32_t* n_active, cudaStream_t s);
cudaError_t launch_mcg_finish(int64_t n_cols, const McgCol* cols, int accumulate, int32_t* col_status,
                              int32_t* col_iters, cudaStream_t st);
cudaError_t launch_mcg_mask(const DevLayout& L, int n_items, int chains, int64_t n_total, int m, const McgCol* cols,
                            float* r, cudaStream_t st);
cudaError_t launch_mcg_refine(int64_t n_cols, int outer, McgCol* cols, double* prev_rr, int32_t* n_active,
                              double* worst, cudaStream_t st);
cudaError_t launch_mcg_undo(const DevLayout& L, int n_items, int chains, int64_t n_total, int m, const McgCol* cols,
                            const float* dx, float* x, cudaStream_t st);
cudaError_t launch_mcg_refine_finish(int64_t n_cols, const McgCol* cols, int32_t* col_status, cudaStream_t st);
// preconditioned multi-column CG: z_q = r_q + U (d_q o (U^T r_q)), d from mu_q = sigma^2 + shift_q
cudaError_t launch_mcg_precond(const DevLayout& L, int n_items, int n_inst, int chains, int64_t n_total, int m,
                               const PcgPrecond& P, const double* theta, int n_theta, const float* shifts,
                               const float* r, float* z, const int32_t* sys_any, double* proj, double* coef,
                               double* prz, cudaStream_t st);
cudaError_t launch_mcg_set_rz(const DevLayout& L, int n_inst, int chains, int m, const double* prz, McgCol* cols,
                              cudaStream_t st);
cudaError_t launch_mcg_update_p(const DevLayout& L, int n_items, int chains, int64_t n_total, int m,
                                const McgCol* stt, const int32_t* sys_any, const float* r, float* p,
                                cudaStream_t st);


cudaError_t launch_lf_drift(int n_sys, int n_theta, const double* theta, const double* pi,
                            const uint8_t* mask, double half_dt, double* theta_h, cudaStream_t st);
cudaError_t launch_pack_force(int chains, int64_t n_total, const float* xsol, const float* phi,
                              float* Vf, float* Gf, cudaStream_t st);
cudaError_t launch_lf_kick_drift(int n_sys, int n_theta, const double* theta_h, const double* grad,
                                 const double* mu, const double* prec, const uint8_t* mask,
                                 const int32_t* status, double dt, double* theta, double* pi,
                                 cudaStream_t st);
cudaError_t launch_dot_partial(const DevLayout& L, int n_items, int chains, int64_t n_total,
                               const float* a, int64_t a_stride, const float* b32, const double* b64,
                               double* partial, cudaStream_t st);
cudaError_t launch_energy_finalize(const DevLayout& L, int n_inst, int chains, int n_theta,
                                   const double* theta, const double* pi, const double* mu,
                                   const double* prec, const double* partial_yx,
                                   const double* partial_pap, int32_t* status, double* H,
                                   double* terms, cudaStream_t st);

}  // namespace kmv

// Handle definition (C ABI opaque type).
struct kmv_handle_s {
  int device = 0;
  std::string last_error;
  // cached device tables for the last layout
  std::vector<int64_t> cached_offsets;
  int cached_d = -1;
  void* tables = nullptr;
  size_t tables_bytes = 0;
  kmv::DevLayout dev;
  kmv::Layout layout;
  // grow-only workspace arena
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int32_t* host_flag = nullptr;   // pinned, for convergence checks
  void* tc = nullptr;             // tensor-core path state (kmv_tc.cu)
  // Chebyshev-amplitude family: internal parameters, amplitudes and the
  // backward's scratch for the current theta (kmv_api.cu, cheb_prepare)
  void* cheb_buf = nullptr;
  size_t cheb_bytes = 0;
  double* cheb_theta = nullptr;
  float* cheb_amp = nullptr;
  float *cheb_kv = nullptr, *cheb_kg = nullptr;
  int cheb_mcap = 0;   // columns cheb_kv / cheb_kg hold
  double *cheb_part = nullptr, *cheb_gint = nullptr;
  // preconditioner set by kmv_set_preconditioner (caller-owned arrays)
  bool pc_on = false;
  kmv_nystrom pc = {};
  // true while the current call's stream is being captured into a CUDA graph:
  // no allocation, no table upload, no host synchronisation may happen then
  bool capturing = false;
  // stream on which the bodies of conditional (WHILE) graph nodes are captured
  cudaStream_t side = nullptr;
  // FP32 forward's J-range split (kmv_simt_fwd.cu): per-chunk FP64 row sums,
  // grown on first use (not under capture); the device's SM count
  double* simt_part = nullptr;
  size_t simt_part_bytes = 0;
  int num_sms = 0;
  // kernel timing (kmv_profile_enable): event pairs around the main product kernels
  bool prof = false;
  std::vector<cudaEvent_t> prof_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_rec[2];
};

namespace kmv {
// Brackets one main-kernel launch with events on `st` while timing is enabled
// and the stream is not being captured.
struct ProfScope {
  kmv_handle h;
  int kind;
  cudaStream_t st;
  cudaEvent_t e1 = nullptr;
  ProfScope(kmv_handle h_, int kind_, cudaStream_t st_);
  ~ProfScope();
};
}  // namespace kmv

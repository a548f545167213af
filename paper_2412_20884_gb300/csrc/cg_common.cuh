// Per-system CG steps shared by the CG kernels (kmv_cg.cu) and the products'
// epilogues when they carry the p.q step of a CG iteration (kmv_tc.cu,
// kmv_simt_fwd.cu), so that every path takes the same arithmetic in the same
// order.
#pragma once

#include "kmv_internal.cuh"

namespace kmv {

// Sum of a system's per-item partials in item order (fixed order: bitwise
// reproducible).
__device__ __forceinline__ double sys_sum(const DevLayout& L, int b, int c, int chains,
                                          const double* partial, int stride, int k) {
  double acc = 0.0;
  for (int it = L.inst_item0[b]; it < L.inst_item0[b + 1]; ++it)
    acc += partial[((int64_t)it * chains + c) * stride + k];
  return acc;
}

// alpha = r.r / p.q of one system; false when the system stops here (a
// non-finite p.q, or a breakdown: the operator is not positive definite along
// p, which a perturbed operator can be; the current iterate is kept).
__device__ __forceinline__ bool cg_pq_step(CgSys& S, double pq) {
  S.pq = pq;
  if (!isfinite(pq)) {
    S.status = KMV_ENONFINITE;
    S.alpha = 0.0;
    return false;
  }
  if (!(pq > 0.0)) {
    S.status = KMV_ENOTCONV;
    S.alpha = 0.0;
    return false;
  }
  S.alpha = S.rr / pq;
  return true;
}

// The new r.r of one system: beta, the iteration count and the stopping
// tests (converged at rr <= tol^2 b.b, or out of iterations); false when the
// system stops.
__device__ __forceinline__ bool cg_rr_step(CgSys& S, double rr, double tol, int maxiter) {
  bool active = true;
  S.iters += 1;
  if (!isfinite(rr)) {
    S.status = KMV_ENONFINITE;
    active = false;
  } else if (rr <= tol * tol * S.bb) {
    active = false;
  } else if (S.iters >= maxiter) {
    S.status = KMV_ENOTCONV;
    active = false;
  }
  S.beta = rr / S.rr;
  S.rr = rr;
  return active;
}

// Called by thread 0 of each of the n_blocks CTAs that write one partial of
// system s, after writing it: true for the CTA that arrives last, which then
// sees every partial of the system.  Resets the counter for the next use.
__device__ __forceinline__ bool last_block_of_system(uint32_t* count, int s, uint32_t n_blocks) {
  __threadfence();
  const bool last = atomicAdd(&count[s], 1u) == n_blocks - 1;
  if (last) {
    __threadfence();
    count[s] = 0;
  }
  return last;
}

}  // namespace kmv

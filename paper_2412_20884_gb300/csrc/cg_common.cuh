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

// Multi-shift CG (kmv_mscg.cu, whose header gives the recurrences): alpha of
// the base system and, per active shift j, zeta_j' and alpha_j.  false when
// the base recurrence breaks down (p.Bp not positive or not finite), which
// stops every shift still running.
__device__ __forceinline__ bool mscg_alpha_step(MscgSys& y, MscgShift* sh, int m, double pq) {
  if (!(pq > 0.0) || !isfinite(pq)) {
    for (int j = 0; j < m; ++j) {
      MscgShift& k = sh[j];
      if (!k.active) continue;
      k.active = 0;
      k.status = isfinite(pq) ? KMV_ENOTCONV : KMV_ENONFINITE;
    }
    return false;
  }
  const double alpha = y.rr / pq;
  y.alpha = alpha;
  for (int j = 0; j < m; ++j) {
    MscgShift& k = sh[j];
    if (!k.active) {
      k.alpha_s = 0.0;
      continue;
    }
    const double den = alpha * y.beta_prev * (k.zeta_prev - k.zeta) +
                       k.zeta_prev * y.alpha_prev * (1.0 + k.sigma * alpha);
    const double zn = k.zeta * k.zeta_prev * y.alpha_prev / den;
    if (!isfinite(zn) || k.zeta == 0.0) {
      k.active = 0;
      k.status = KMV_ENONFINITE;
      k.alpha_s = 0.0;
      continue;
    }
    k.zeta_next = zn;
    k.alpha_s = alpha * zn / k.zeta;
  }
  return true;
}

// Multi-shift CG: beta of the base system from the new r.r, and per active
// shift the stopping test (|zeta_j'|^2 r.r <= tol^2 b.b, or out of
// iterations), beta_j and the advance of zeta.  false when no shift is left.
__device__ __forceinline__ bool mscg_beta_step(MscgSys& y, MscgShift* sh, int m, double rr, double tol,
                                               int maxiter) {
  const double beta = rr / y.rr;
  const double lim = tol * tol * y.bb;
  y.iters += 1;
  int any = 0;
  for (int j = 0; j < m; ++j) {
    MscgShift& k = sh[j];
    if (!k.active) continue;
    k.iters += 1;
    const double ratio = k.zeta_next / k.zeta;
    const double res2 = k.zeta_next * k.zeta_next * rr;
    if (!isfinite(res2) || !isfinite(beta)) {
      k.active = 0;
      k.status = KMV_ENONFINITE;
    } else if (res2 <= lim) {
      k.active = 0;
    } else if (k.iters >= maxiter) {
      k.active = 0;
      k.status = KMV_ENOTCONV;
    } else {
      k.beta_s = beta * ratio * ratio;
      k.zeta_prev = k.zeta;
      k.zeta = k.zeta_next;
    }
    any |= k.active;
  }
  y.rr = rr;
  y.beta = beta;
  y.alpha_prev = y.alpha;
  y.beta_prev = beta;
  return any != 0;
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

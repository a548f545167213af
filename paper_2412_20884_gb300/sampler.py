"""One iteration of Algorithm 1 (pseudofermion HMC) composed from the library's
entry points; every arithmetic step runs in the library's kernels, this module
only orders the calls."""
from __future__ import annotations

import torch

from .binding import Kmv, Points, accept, status_merge


def hmc_update(h: Kmv, pts: Points, y, theta, dt: float, n_int: int, xi, pi, u, prior=None, free_mask=None,
               prec: str = "fp32", cg_tol: float = 1e-6, cg_maxiter: int = 2000, n_poles: int = 15,
               integrator: str = "leapfrog", aa_depth: int = 10, aa_tol: float = 1e-5, aa_maxiter: int = 500,
               energy_prec: str = "fp32"):
    """Algorithm 1 for every (instance, chain) system:
      phi = A(theta)^{-1/2} xi            (kmv_phi_refresh, Sec. 3.1)
      H_old = H(theta, pi)                (kmv_energy)
      n_int integrator steps              (leapfrog_step, Sec. 3.2.2, or kmv_implicit_step, Sec. 3.2.3)
      H_new = H(theta', pi')
      accept iff log u <= H_old - H_new   (kmv_accept); a rejected system keeps theta.
    xi (chains, N_total) ~ N(0, 1), pi (n_sys, n_theta) ~ N(0, I) (M = I) and u (n_sys)
    ~ U(0, 1] are the caller's draws.  theta is updated in place; the first failure of
    any step (a solve that did not converge, a non-finite energy) rejects the system.
    Returns (accepted (n_sys int32), fail status (n_sys int32))."""
    if integrator not in ("leapfrog", "implicit"):
        raise ValueError("integrator must be 'leapfrog' or 'implicit'")
    phi, st, _ = h.phi_refresh(pts, theta, xi, n_poles=n_poles, cg_tol=cg_tol, cg_maxiter=cg_maxiter, prec=prec)
    fail = st.clone()
    theta_old = theta.clone()
    pi = pi.clone()
    x = torch.zeros_like(phi)
    H_old, _, st, _ = h.kmv_energy(pts, y, phi, theta, pi, prior=prior, cg_tol=cg_tol, cg_maxiter=cg_maxiter,
                                   x_work=x, prec=energy_prec)
    status_merge(st, fail)
    for _ in range(n_int):
        if integrator == "leapfrog":
            st, _, _ = h.leapfrog_step(pts, y, phi, theta, pi, dt, prior=prior, free_mask=free_mask, cg_tol=cg_tol,
                                       cg_maxiter=cg_maxiter, x_work=x, prec=prec)
        else:
            st, _, _ = h.implicit_step(pts, y, phi, theta, pi, dt, prior=prior, free_mask=free_mask,
                                       aa_depth=aa_depth, tol=aa_tol, maxiter=aa_maxiter, x_work=x, prec=prec)
        status_merge(st, fail)
    H_new, _, st, _ = h.kmv_energy(pts, y, phi, theta, pi, prior=prior, cg_tol=cg_tol, cg_maxiter=cg_maxiter,
                                   prec=energy_prec)
    status_merge(st, fail)
    acc = accept(H_old, H_new, u, theta_old, theta, status=fail)
    return acc, fail

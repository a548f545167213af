"""FP64 implicit-midpoint HMC step solved by Anderson-accelerated fixed-point
iteration (test infrastructure only).

Definitions followed:
  * Sec. 3.2.3, Eq. implicitsystem: the unknowns (theta_1, pi_1, x) of one
    implicit midpoint step satisfy, with theta_bar = (theta_0 + theta_1)/2 and M = I,
        theta_1 = theta_0 + dt (pi_0 + pi_1)/2,
        pi_1    = pi_0 - dt f_phi(theta_bar, x),
        A(theta_bar) x = y,
    f_phi(theta, x) = grad S(theta) - x^T (dA/dtheta) x / 2 + phi^T (dA/dtheta) phi / 2
    (the force with x held fixed, Sec. 3.2.1).
  * Eq. Phi: the fixed-point map
        Phi(theta, pi, x) = (theta_0 + dt (pi_0 + pi)/2,
                             pi_0 - dt f_phi((theta_0 + theta)/2, x),
                             x + R [y - A((theta_0 + theta)/2) x]),
    R a preconditioner for A(theta_0) scaled so that rho(R A) <= 1.
  * App. B (Anderson acceleration): with residuals f(z) = z - Phi(z) of the
    last k iterates, coefficients alpha minimising |sum_i alpha_i f_i|^2 subject
    to sum_i alpha_i = 1, and the next iterate sum_i alpha_i Phi(z_i); theta,
    pi and x form one vector.
  * free components: entries of theta with free = 0 keep theta_0 and pi_0.

Parity status: pinned (Anderson acceleration with full history on a linear map
against GMRES (the Walker-Ni equivalence the appendix cites), the fixed point
against the implicit equations evaluated with Cholesky solves, the symmetry of
the midpoint map (reversibility), and second-order agreement with the leapfrog
map as dt -> 0) - see tests/test_oracle_implicit.py.
"""
from __future__ import annotations

import numpy as np

from .hmc import _A, _dA, prior_grad


def force_frozen(X, phi, theta, x, ard, prior=None, kern=None):
    """f_phi(theta, x) with x held fixed (Sec. 3.2.1)."""
    F = prior_grad(theta, prior)
    for p, M in enumerate(_dA(X, theta, ard, kern)):
        F[p] += -0.5 * float(x @ M @ x) + 0.5 * float(phi @ M @ phi)
    return F


def phi_map(z, theta0, pi0, dt, X, y, phi, R, ard, prior=None, free=None, kern=None):
    """Phi of Eq. Phi on the stacked vector z = [theta, pi, x]."""
    n = theta0.size
    theta, pi, x = z[:n], z[n:2 * n], z[2 * n:]
    mask = np.ones(n) if free is None else np.asarray(free, np.float64)
    tbar = 0.5 * (theta0 + theta)
    t_new = theta0 + dt * 0.5 * (pi0 + pi) * mask
    p_new = pi0 - dt * force_frozen(X, phi, tbar, x, ard, prior, kern) * mask
    x_new = x + R @ (y - _A(X, tbar, ard, kern) @ x)
    return np.concatenate([t_new, p_new, x_new])


def anderson(g, z0, k: int, tol: float, maxiter: int, converged=None):
    """Anderson acceleration of z = g(z) (App. B).  Returns (z, g(z), iterations).

    converged(z, gz) decides when to stop (default: |z - g(z)| <= tol |g(z)|)."""
    if converged is None:
        converged = lambda z, gz: np.linalg.norm(z - gz) <= tol * max(np.linalg.norm(gz), 1e-300)
    Z, G = [], []
    z = np.array(z0, np.float64)
    for it in range(maxiter):
        gz = g(z)
        if converged(z, gz):
            return z, gz, it
        Z.append(z)
        G.append(gz)
        Z, G = Z[-k:], G[-k:]
        F = np.array([zi - gi for zi, gi in zip(Z, G)])          # residuals f_i, newest last
        H = F @ F.T
        ones = np.ones(len(Z))
        a = np.linalg.lstsq(H, ones, rcond=None)[0]
        alpha = a / a.sum()
        z = alpha @ np.array(G)
    return z, g(z), maxiter


def implicit_midpoint(X, y, phi, theta0, pi0, dt, ard, R, k: int = 10, tol: float = 1e-10, maxiter: int = 500,
                      x0=None, prior=None, free=None, kern=None):
    """One implicit midpoint step by Anderson-accelerated iteration of Phi.
    Returns (theta_1, pi_1, x, iterations)."""
    theta0 = np.asarray(theta0, np.float64)
    pi0 = np.asarray(pi0, np.float64)
    n = theta0.size
    x0 = np.zeros(len(y)) if x0 is None else np.asarray(x0, np.float64)
    z0 = np.concatenate([theta0, pi0, x0])
    g = lambda z: phi_map(z, theta0, pi0, dt, X, y, phi, R, ard, prior, free, kern)
    z, gz, it = anderson(g, z0, k, tol, maxiter)
    return gz[:n], gz[n:2 * n], gz[2 * n:], it

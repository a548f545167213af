"""Pole expansion of the inverse square root, App. A (test infrastructure only).

Eq. msqdisc gives A^{1/2} ~ (2 K' m^{1/2} A / (pi N_p)) sum_j cn(t_j) dn(t_j) (A - w(t_j)^2 I)^{-1}
with t_j = i (j - 1/2) K' / N_p, w(t) = m^{1/2} sn(t | k^2), k^2 = m / M,
K = K(k^2), K' = K(1 - k^2).  Dropping the leading A gives A^{-1/2} (Eq. pex).
The sum in the printed formula runs to "N"; it is read as j = 1..N_p.

The t_j are purely imaginary.  Jacobi's imaginary transformation,
  sn(i u | k^2) = i sn(u | k'^2) / cn(u | k'^2),
  cn(i u | k^2) = 1 / cn(u | k'^2),
  dn(i u | k^2) = dn(u | k'^2) / cn(u | k'^2),
turns every term real:
  shift  lambda_j = -w(t_j)^2 = m (sn_j / cn_j)^2 >= 0
  weight w_j      = (2 K' sqrt(m) / (pi N_p)) dn_j / cn_j^2
with (sn_j, cn_j, dn_j) evaluated at u_j = (j - 1/2) K' / N_p, parameter 1 - k^2.
Then A^{-1/2} xi ~ sum_j w_j (A + lambda_j I)^{-1} xi.

m is a lower bound on the spectrum of A (the noise variance sigma^2; App. A
prints min sigma, read as min sigma^2, since lambda_min(A) >= sigma^2).

Spectral interval (Sec. 3.1 / App. A): m = sigma^2; M = the largest row sum of
A, max_i (A 1)_i = alpha max_i sum_j K0_ij + sigma^2.  Because K0 >= 0
entrywise, the largest row sum (the infinity norm of A) bounds lambda_max from
above, where the power iteration App. A mentions approaches it from below.

Parity status: pinned (scalar function against x^{-1/2}, the matrix form
against an exact eigendecomposition, the spectral interval against the
eigenvalues) - see tests/test_oracle_poles_diag.py.
"""
from __future__ import annotations

import numpy as np
from scipy.special import ellipj, ellipk

from .se_kernel import A_matrix, unpack_theta


def pole_weights_shifts(m_lo: float, M_hi: float, n_poles: int = 15):
    k2 = m_lo / M_hi
    Kp = float(ellipk(1.0 - k2))
    u = (np.arange(1, n_poles + 1) - 0.5) * Kp / n_poles
    sn, cn, dn, _ = ellipj(u, 1.0 - k2)
    shifts = m_lo * (sn / cn) ** 2
    weights = (2.0 * Kp * np.sqrt(m_lo) / (np.pi * n_poles)) * dn / cn ** 2
    return weights, shifts


def inv_sqrt_scalar(lam, weights, shifts):
    lam = np.asarray(lam, np.float64)
    return np.sum(weights[None, :] / (lam[:, None] + shifts[None, :]), axis=1)


def inv_sqrt_apply(A, xi, m_lo, M_hi, n_poles: int = 15):
    """sum_j w_j (A + lambda_j I)^{-1} xi with exact dense solves."""
    w, s = pole_weights_shifts(m_lo, M_hi, n_poles)
    n = A.shape[0]
    out = np.zeros_like(np.asarray(xi, np.float64))
    for wj, sj in zip(w, s):
        out += wj * np.linalg.solve(A + sj * np.eye(n), xi)
    return out


def spectral_interval(X, theta, ard: bool):
    """(m, M): sigma^2 and the largest row sum of A(theta)."""
    A = A_matrix(X, theta, ard)
    _, _, s2 = unpack_theta(theta, np.asarray(X).shape[1], ard)
    return float(s2), float(np.max(A.sum(axis=1)))


def phi_pole(X, theta, xi, ard: bool, n_poles: int = 15):
    """The Gibbs draw of Sec. 3.1, phi = A^{-1/2} xi, by the pole expansion of
    App. A on the interval of spectral_interval, with dense solves."""
    m_lo, M_hi = spectral_interval(X, theta, ard)
    return inv_sqrt_apply(A_matrix(X, theta, ard), xi, m_lo, M_hi, n_poles)

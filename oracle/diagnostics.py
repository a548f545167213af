"""Chain diagnostics of Sec. 4.1 and App. C (test infrastructure only).

  * moving_window_mean : T_i = mean(X_floor(i/2) .. X_i) (Sec. 4.1).
  * autocov            : C_hat(j) = 1/(N-j) sum_i (f_i - mean)(f_{i+j} - mean) (App. C).
  * iat                : tau_hat = 1 + 2 sum_{j=1}^{M} C_hat(j)/C_hat(0), with the
                         window M the smallest value satisfying M >= c tau_hat(M),
                         c = 5 (App. C).
  * marginal_cdf_grid  : trapezoid-rule marginal CDFs of P(theta) on a grid (Sec. 4.1).

Parity status: pinned (AR(1) autocorrelation time (1+rho)/(1-rho); the CDF of
a Gaussian density) - see tests/test_oracle_poles_diag.py.
"""
from __future__ import annotations

import numpy as np


def moving_window_mean(xs):
    xs = np.asarray(xs, np.float64)
    out = np.empty(len(xs))
    c = np.concatenate([[0.0], np.cumsum(xs)])
    for i in range(len(xs)):
        lo = i // 2
        out[i] = (c[i + 1] - c[lo]) / (i + 1 - lo)
    return out


def autocov(f):
    f = np.asarray(f, np.float64)
    n = len(f)
    g = f - f.mean()
    return np.array([np.dot(g[:n - j], g[j:]) / (n - j) for j in range(n)])


def iat(f, c: float = 5.0):
    C = autocov(f)
    rho = C / C[0]
    tau = 1.0
    for M in range(1, len(f)):
        tau = 1.0 + 2.0 * np.sum(rho[1:M + 1])
        if M >= c * tau:
            return float(tau)
    return float(tau)


def trapezoid_weights(n):
    w = np.ones(n)
    w[0] = w[-1] = 0.5
    return w


def marginal_cdf_grid(logp_grid, axis_vals, axis: int):
    """Marginal CDF along ``axis`` of exp(logp) tabulated on a tensor grid.

    logp_grid has one dimension per parameter; axis_vals are the equispaced
    coordinates of that axis.  Integrals use the trapezoid rule (Sec. 4.1).
    """
    p = np.exp(logp_grid - logp_grid.max())
    other = tuple(a for a in range(p.ndim) if a != axis)
    for a in sorted(other, reverse=True):
        w = trapezoid_weights(p.shape[a])
        p = np.tensordot(p, w, axes=([a], [0]))
    h = axis_vals[1] - axis_vals[0]
    cum = np.concatenate([[0.0], np.cumsum(0.5 * h * (p[1:] + p[:-1]))])
    return cum / cum[-1]

"""FP64 HMC pieces for the determinant-free posterior (test infrastructure only).

Definitions followed:
  * Eq. P            : P(theta) ~ |A|^{-1/2} exp(-y^T A^{-1} y / 2) p(theta).
  * Eq. extendeddensity / Eq. U : U_phi(theta) = S(theta) + y^T A^{-1} y / 2 + phi^T A phi / 2,
                       with p(theta) ~ exp(-S(theta)).
  * Sec. 3.1         : the Gibbs draw phi = A^{-1/2} xi, xi ~ N(0, I); computed here
                       exactly by a symmetric eigendecomposition.
  * Sec. 3.2         : H = U + pi^T M^{-1} pi / 2 with M = I; acceptance with
                       probability min(1, exp(H_old - H_new)).
  * Sec. 3.2.1       : the force by its direct expression
                       F = grad S - (1/2) x^T (dA/dtheta) x + (1/2) phi^T (dA/dtheta) phi,
                       x = A^{-1} y from a Cholesky solve (not the frozen-x rewrite,
                       which the library uses; the two must agree).
  * Sec. 3.2.2       : drift-kick-drift leapfrog, read as
                       theta_half = theta_0 + dt/2 pi_0;  pi_1 = pi_0 - dt F(theta_half);
                       theta_1 = theta_half + dt/2 pi_1
                       (the printed kick updates pi_1 from itself; pi_0 is meant).
  * Algorithm 1      : one update = draw xi, form phi, draw pi, integrate N_int steps,
                       Metropolis test against a uniform X <= acceptance.

Kernel family: ``kern`` = None is the stationary SE kernel of oracle/se_kernel.py;
otherwise a pair (A_fn, dA_fn) of callables (X, theta) -> A and -> [dA/dtheta_p]
(e.g. the Chebyshev-amplitude family of oracle/cheb_kernel.py).

Prior: ``None`` is the paper's flat prior (S = 0).  A dict {"mu", "prec"} gives
the diagonal Gaussian S = sum prec (theta - mu)^2 / 2 used by the tiny-N test.
``free`` marks which components move (the paper fixes sigma or l at times);
fixed components get no kick.

Parity status: pinned (finite differences of U for the force, the Gaussian
identity, reversibility and O(dt^2) energy error of the leapfrog map, and the
tiny-N sampler against quadrature of Eq. P) - see tests/test_oracle_hmc.py.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .se_kernel import A_matrix, dA_dtheta


def _A(X, theta, ard, kern):
    return A_matrix(X, theta, ard) if kern is None else kern[0](X, theta)


def _dA(X, theta, ard, kern):
    return dA_dtheta(X, theta, ard) if kern is None else kern[1](X, theta)


def prior_S(theta, prior):
    if prior is None:
        return 0.0
    t = np.asarray(theta, np.float64)
    return 0.5 * float(np.sum(prior["prec"] * (t - prior["mu"]) ** 2))


def prior_grad(theta, prior):
    t = np.asarray(theta, np.float64)
    if prior is None:
        return np.zeros_like(t)
    return np.asarray(prior["prec"], np.float64) * (t - prior["mu"])


def solve(X, theta, y, ard):
    """x = A(theta)^{-1} y by Cholesky (Eq. xtheta)."""
    A = A_matrix(X, theta, ard)
    return sla.cho_solve(sla.cho_factor(A, lower=True), np.asarray(y, np.float64))


def potential(X, y, phi, theta, ard, prior=None, kern=None):
    """U_phi(theta) of Eq. U."""
    A = _A(X, theta, ard, kern)
    x = sla.cho_solve(sla.cho_factor(A, lower=True), y)
    return prior_S(theta, prior) + 0.5 * float(y @ x) + 0.5 * float(phi @ A @ phi)


def force(X, y, phi, theta, ard, prior=None, kern=None):
    """F_phi(theta) = grad U by the direct expression of Sec. 3.2.1."""
    A = _A(X, theta, ard, kern)
    x = sla.cho_solve(sla.cho_factor(A, lower=True), y)
    mats = _dA(X, theta, ard, kern)
    F = prior_grad(theta, prior)
    for p, M in enumerate(mats):
        F[p] += -0.5 * float(x @ M @ x) + 0.5 * float(phi @ M @ phi)
    return F


def hamiltonian(X, y, phi, theta, pi, ard, prior=None, kern=None):
    pi = np.asarray(pi, np.float64)
    return potential(X, y, phi, theta, ard, prior, kern) + 0.5 * float(pi @ pi)


def leapfrog(X, y, phi, theta, pi, dt, ard, prior=None, free=None, n_steps=1, kern=None):
    """n_steps of the drift-kick-drift map of Sec. 3.2.2, drifts not merged."""
    theta = np.array(theta, np.float64)
    pi = np.array(pi, np.float64)
    mask = np.ones_like(theta) if free is None else np.asarray(free, np.float64)
    for _ in range(n_steps):
        theta_half = theta + 0.5 * dt * pi * mask
        F = force(X, y, phi, theta_half, ard, prior, kern)
        pi = pi - dt * F * mask
        theta = theta_half + 0.5 * dt * pi * mask
    return theta, pi


def accept(H_old, H_new, u):
    """Metropolis test of Algorithm 1: accept iff u <= min(1, exp(H_old - H_new)).

    Evaluated as log(u) <= H_old - H_new, which is the same event for u in (0, 1].
    """
    return bool(np.log(u) <= H_old - H_new)


def log_posterior(X, y, theta, ard, prior=None):
    """log P(theta) of Eq. P, up to an additive constant, with an exact determinant."""
    A = A_matrix(X, theta, ard)
    c, low = sla.cho_factor(A, lower=True)
    x = sla.cho_solve((c, low), y)
    logdet = 2.0 * float(np.sum(np.log(np.diag(c))))
    return -0.5 * logdet - 0.5 * float(y @ x) - prior_S(theta, prior)


def inv_sqrt_apply(A, xi):
    """A^{-1/2} xi for symmetric positive definite A (the Gibbs draw of Sec. 3.1)."""
    w, Q = np.linalg.eigh(A)
    scale = 1.0 / np.sqrt(w)
    coeff = Q.T @ xi
    return Q @ (coeff * (scale if coeff.ndim == 1 else scale[:, None]))


def phi_exact(X, theta, xi, ard):
    return inv_sqrt_apply(A_matrix(X, theta, ard), np.asarray(xi, np.float64))


def hmc_update(X, y, theta, ard, dt, n_int, xi, pi0, u, prior=None, free=None):
    """One iteration of Algorithm 1 with the exact Gibbs draw.

    xi, pi0, u are the caller's random numbers (xi ~ N(0, I_N), pi0 ~ N(0, I_n),
    u ~ U[0, 1]).  Returns (theta_next, accepted, H_old, H_new).
    """
    theta = np.asarray(theta, np.float64)
    mask = np.ones_like(theta) if free is None else np.asarray(free, np.float64)
    phi = phi_exact(X, theta, xi, ard)
    pi = np.asarray(pi0, np.float64) * mask
    H0 = hamiltonian(X, y, phi, theta, pi, ard, prior)
    th1, pi1 = leapfrog(X, y, phi, theta, pi, dt, ard, prior, free, n_int)
    H1 = hamiltonian(X, y, phi, th1, pi1, ard, prior)
    ok = accept(H0, H1, u)
    return (th1 if ok else theta), ok, H0, H1


# ---------------------------------------------------------------------------
# Batched (many chains, tiny N) forms of the same definitions, used by the
# quadrature test.  Each function is the single-chain definition above
# evaluated on a stack of chains; no formula differs.
# ---------------------------------------------------------------------------

def _A_and_dA_batch(X, thetas, ard):
    """Stacks A (B, N, N) and dA/dtheta (B, n, N, N) for chains' thetas (B, n)."""
    X = np.asarray(X, np.float64)
    n, d = X.shape
    thetas = np.asarray(thetas, np.float64)
    k = d if ard else 1
    alpha = np.exp(thetas[:, 0])
    ell = np.exp(thetas[:, 1:1 + k])
    if not ard:
        ell = np.repeat(ell, d, axis=1)
    sigma2 = np.exp(thetas[:, 1 + k])
    diff2 = (X[:, None, :] - X[None, :, :]) ** 2                    # (N, N, d)
    scaled = diff2[None, :, :, :] / (ell[:, None, None, :] ** 2)   # (B, N, N, d)
    K = alpha[:, None, None] * np.exp(-0.5 * scaled.sum(axis=-1))
    eye = np.eye(n)
    A = K + sigma2[:, None, None] * eye
    dA = [K]
    if ard:
        dA.extend(K * scaled[..., kk] for kk in range(d))
    else:
        dA.append(K * scaled.sum(axis=-1))
    dA.append(sigma2[:, None, None] * eye[None])
    return A, np.stack(dA, axis=1)


def potential_batch(X, y, phis, thetas, ard, prior=None):
    A, _ = _A_and_dA_batch(X, thetas, ard)
    x = np.linalg.solve(A, np.broadcast_to(y, phis.shape)[..., None])[..., 0]
    S = 0.0 if prior is None else 0.5 * np.sum(prior["prec"] * (thetas - prior["mu"]) ** 2, axis=1)
    return S + 0.5 * np.einsum("n,bn->b", y, x) + 0.5 * np.einsum("bi,bij,bj->b", phis, A, phis)


def force_batch(X, y, phis, thetas, ard, prior=None):
    A, dA = _A_and_dA_batch(X, thetas, ard)
    x = np.linalg.solve(A, np.broadcast_to(y, phis.shape)[..., None])[..., 0]
    F = -0.5 * np.einsum("bi,bpij,bj->bp", x, dA, x) + 0.5 * np.einsum("bi,bpij,bj->bp", phis, dA, phis)
    if prior is not None:
        F = F + prior["prec"] * (thetas - prior["mu"])
    return F


def phi_exact_batch(X, thetas, xis, ard):
    A, _ = _A_and_dA_batch(X, thetas, ard)
    w, Q = np.linalg.eigh(A)
    return np.einsum("bij,bj->bi", Q, np.einsum("bji,bj->bi", Q, xis) / np.sqrt(w))


def hmc_update_batch(X, y, thetas, ard, dt, n_int, xis, pis, us, prior=None, free=None):
    """Algorithm 1 for B independent chains at once (tiny N).  Returns (thetas, accepted)."""
    thetas = np.asarray(thetas, np.float64)
    mask = np.ones(thetas.shape[1]) if free is None else np.asarray(free, np.float64)
    phis = phi_exact_batch(X, thetas, xis, ard)
    pi = pis * mask
    H0 = potential_batch(X, y, phis, thetas, ard, prior) + 0.5 * np.sum(pi * pi, axis=1)
    th = thetas.copy()
    for _ in range(n_int):
        th_half = th + 0.5 * dt * pi * mask
        pi = pi - dt * force_batch(X, y, phis, th_half, ard, prior) * mask
        th = th_half + 0.5 * dt * pi * mask
    H1 = potential_batch(X, y, phis, th, ard, prior) + 0.5 * np.sum(pi * pi, axis=1)
    with np.errstate(over="ignore", invalid="ignore"):
        ok = np.log(us) <= (H0 - H1)
    ok &= np.isfinite(H1)
    return np.where(ok[:, None], th, thetas), ok

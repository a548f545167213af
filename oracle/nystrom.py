"""FP64 randomized Nystrom preconditioner (test infrastructure only).

Definitions followed: the randomized Nystrom approximation and preconditioner
of Frangella, Tropp and Udell ("Randomized Nystrom preconditioning", SIAM J.
Matrix Anal. Appl. 2023), which the paper uses for its solves (Sec. 3.1, end;
Sec. 3.2.3; Sec. 4.2 setup), with the Woodbury identity applied to the
diagonal part of A:
  * Omega = Q R (thin QR of the N x r Gaussian test matrix), Y = K Q,
    nu = sqrt(N) eps ||Y||_2, Y_nu = Y + nu Q, Q^T Y_nu = L L^T (Cholesky),
    B = Y_nu L^{-T} = U S W^T (thin SVD), Lambda = max(S^2 - nu, 0):
    K_hat = U Lambda U^T approximates K (it depends on Omega only through its
    range, and on nu at the level nu).
  * for A = K + mu I:  P^{-1} = (lambda_r + mu) U (Lambda + mu)^{-1} U^T + (I - U U^T),
    lambda_r the smallest of Lambda; mu = sigma^2 (+ a shift lambda_p of Eq. pex).
  * preconditioned CG: the textbook recurrences with z = P^{-1} r.
``eps`` is the FP64 unit roundoff by default, as in Frangella et al.

Parity status: pinned (exactness on kernels of rank <= r, K - K_hat PSD, the
closed-form spectrum of P^{-1} A when K_hat = K, P^{-1} = I without a range,
PCG against a dense solve) - see tests/test_oracle_nystrom.py.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def nystrom(K, Omega, eps: float = 2.0 ** -52):
    """(U, Lambda) of the randomized Nystrom approximation of PSD K with test matrix Omega."""
    K = np.asarray(K, np.float64)
    Q, _ = np.linalg.qr(np.asarray(Omega, np.float64))
    n = K.shape[0]
    Y = K @ Q
    nu = np.sqrt(n) * eps * np.linalg.norm(Y, 2)
    Y_nu = Y + nu * Q
    W = Q.T @ Y_nu
    L = np.linalg.cholesky(0.5 * (W + W.T))
    B = sla.solve_triangular(L, Y_nu.T, lower=True).T        # Y_nu L^{-T}
    U, S, _ = np.linalg.svd(B, full_matrices=False)
    lam = np.maximum(S * S - nu, 0.0)
    return U, lam


def precond_apply(U, lam, mu, r):
    """P^{-1} r for A = K + mu I."""
    r = np.asarray(r, np.float64)
    c = U.T @ r
    lam_r = lam[-1]
    return U @ ((lam_r + mu) / (lam + mu) * c) + (r - U @ c)


def pcg(A, b, apply_pinv, tol: float, maxiter: int):
    """Preconditioned CG on A x = b from x = 0; stops when |r| <= tol |b|.  Returns (x, iterations)."""
    b = np.asarray(b, np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    z = apply_pinv(r)
    p = z.copy()
    rz = r @ z
    bn = np.linalg.norm(b)
    for k in range(maxiter):
        if np.linalg.norm(r) <= tol * bn:
            return x, k
        q = A @ p
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        z = apply_pinv(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxiter

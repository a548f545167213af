"""FP64 squared-exponential kernel matrix, products and adjoint (test infrastructure only).

Definitions followed:
  * kernel, Sec. 1:   K(x, x') = alpha * exp(-|x - x'|^2 / (2 l^2)); the ARD form
    replaces |x - x'|^2 / l^2 by sum_k (x_k - x'_k)^2 / l_k^2.
  * Eq. kerdef:       A_ij = sigma^2 delta_ij + K(x_i, x_j)  (constant noise).
  * Sec. 3.2.1, primitive (3): gradients of quadratic forms in A(theta).

Hyperparameters: theta = [log alpha, log l_1..log l_k, log sigma^2], k = 1 or d.

Parity status: pinned (closed forms, limits, invariances, central differences
of ``kmv`` itself for the adjoint) - see tests/test_oracle_kernel.py.
"""
from __future__ import annotations

import numpy as np


def unpack_theta(theta, d: int, ard: bool):
    """Return (alpha, ell[d], sigma2) from a log-parameter vector."""
    theta = np.asarray(theta, dtype=np.float64)
    k = d if ard else 1
    if theta.shape != (k + 2,):
        raise ValueError(f"theta must have {k + 2} entries, got {theta.shape}")
    alpha = float(np.exp(theta[0]))
    ell = np.exp(theta[1:1 + k])
    if not ard:
        ell = np.full(d, ell[0])
    sigma2 = float(np.exp(theta[1 + k]))
    return alpha, ell, sigma2


def scaled_sq_dist(Xa, Xb, ell):
    """r2[a, b] = sum_k (Xa[a,k] - Xb[b,k])^2 / ell_k^2, from direct differences."""
    Xa = np.asarray(Xa, np.float64)
    Xb = np.asarray(Xb, np.float64)
    r2 = np.zeros((Xa.shape[0], Xb.shape[0]))
    for k in range(Xa.shape[1]):
        diff = (Xa[:, k, None] - Xb[None, :, k]) / ell[k]
        r2 += diff * diff
    return r2


def kernel_matrix(Xa, Xb, theta, ard: bool):
    """K[a, b] = alpha exp(-r2/2) (Sec. 1)."""
    alpha, ell, _ = unpack_theta(theta, np.shape(Xa)[1], ard)
    return alpha * np.exp(-0.5 * scaled_sq_dist(Xa, Xb, ell))


def A_matrix(X, theta, ard: bool):
    """Dense A = K + sigma^2 I (Eq. kerdef)."""
    _, _, sigma2 = unpack_theta(theta, np.shape(X)[1], ard)
    K = kernel_matrix(X, X, theta, ard)
    return K + sigma2 * np.eye(K.shape[0])


def kmv(X, theta, V, ard: bool, rows=None, col_shift=None, block: int = 256):
    """Rows of A(theta) V, computed block of rows by block of rows.

    rows      : optional row indices; returns A[rows, :] @ V.
    col_shift : optional per-column shift s_c; column c becomes (A + s_c I) V[:, c]
                (the shifted systems of Eq. pex).
    """
    X = np.asarray(X, np.float64)
    V = np.asarray(V, np.float64)
    squeeze = V.ndim == 1
    if squeeze:
        V = V[:, None]
    n = X.shape[0]
    rows = np.arange(n) if rows is None else np.asarray(rows)
    _, _, sigma2 = unpack_theta(theta, X.shape[1], ard)
    out = np.zeros((len(rows), V.shape[1]))
    for s in range(0, len(rows), block):
        r = rows[s:s + block]
        Kb = kernel_matrix(X[r], X, theta, ard)
        out[s:s + block] = Kb @ V + sigma2 * V[r]
    if col_shift is not None:
        out += np.asarray(col_shift, np.float64)[None, :] * V[rows]
    return out[:, 0] if squeeze else out


def dA_dtheta(X, theta, ard: bool):
    """Dense partial derivatives dA/dtheta_p, one N x N matrix per hyperparameter.

    d/dlog alpha   : K
    d/dlog l_k     : K o (x_ik - x_jk)^2 / l_k^2 (ARD); the sum over k (isotropic)
    d/dlog sigma^2 : sigma^2 I
    """
    X = np.asarray(X, np.float64)
    d = X.shape[1]
    alpha, ell, sigma2 = unpack_theta(theta, d, ard)
    K = kernel_matrix(X, X, theta, ard)
    mats = [K]
    per_dim = [K * ((X[:, k, None] - X[None, :, k]) / ell[k]) ** 2 for k in range(d)]
    if ard:
        mats.extend(per_dim)
    else:
        mats.append(sum(per_dim))
    mats.append(sigma2 * np.eye(X.shape[0]))
    return mats


def kmv_adjoint(X, theta, V, G, ard: bool, rows=None, block: int = 256):
    """Adjoint of L = sum_{i,c} G_ic (A V)_ic.

    Returns (grad_theta, grad_V) with
      dL/dV          = A^T G = A G
      dL/dlog alpha  = sum_ij W_ij K_ij,                     W = G V^T
      dL/dlog l_k    = sum_ij W_ij K_ij (x_ik - x_jk)^2/l_k^2 (isotropic: summed over k)
      dL/dlog sigma2 = sigma^2 sum G o V
    ``rows`` declares that G vanishes outside those rows (the sampled-row form);
    the result is then exact for the whole of dL/dV and dL/dtheta.
    """
    X = np.asarray(X, np.float64)
    V = np.asarray(V, np.float64)
    G = np.asarray(G, np.float64)
    if V.ndim == 1:
        V = V[:, None]
        G = G[:, None]
    n, d = X.shape
    alpha, ell, sigma2 = unpack_theta(theta, d, ard)
    rows = np.arange(n) if rows is None else np.asarray(rows)
    k = d if ard else 1
    g = np.zeros(k + 2)
    gV = np.zeros_like(V)
    for s in range(0, len(rows), block):
        r = rows[s:s + block]
        Kb = kernel_matrix(X[r], X, theta, ard)           # (|r|, N)
        W = G[r] @ V.T                                     # (|r|, N)
        WK = W * Kb
        g[0] += WK.sum()
        for kk in range(d):
            dk = ((X[r, kk, None] - X[None, :, kk]) / ell[kk]) ** 2
            contrib = (WK * dk).sum()
            if ard:
                g[1 + kk] += contrib
            else:
                g[1] += contrib
        gV += Kb.T @ G[r]
    g[k + 1] = sigma2 * float((G[rows] * V[rows]).sum())
    gV[rows] += sigma2 * G[rows]
    return g, gV


def quad_form_grad(X, theta, z, ard: bool):
    """grad_theta [z^T A(theta) z] from the dense dA/dtheta (primitive (3), Sec. 3.2.1)."""
    z = np.asarray(z, np.float64)
    return np.array([z @ M @ z for M in dA_dtheta(X, theta, ard)])

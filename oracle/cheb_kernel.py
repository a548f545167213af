"""FP64 non-stationary squared-exponential kernel with a Chebyshev log-amplitude
(test infrastructure only).

Definitions followed (Sec. 4, the kernel family of the numerical experiments):
  * T_n is the Chebyshev polynomial of the first kind; points lie in [-1, 1]^d.
  * C_theta(x) = sum over multi-indices (i_1..i_d) in [0, N_cheb)^d of
        Theta[i_1, .., i_d] T_{i_1}(x^1) ... T_{i_d}(x^d).
  * K(x, x') = exp(C(x)) exp(C(x')) exp(-|x - x'|^2 / (2 l^2)); the ARD form
    replaces |x - x'|^2 / l^2 by sum_k (x_k - x'_k)^2 / l_k^2 (the paper uses one l).
  * A = K + sigma^2 I with constant noise (Eq. kerdef).

Hyperparameters: theta = [Theta flattened row-major (i_1 slowest), log l_1..log l_k,
log sigma^2], k = 1 (isotropic) or d (ARD); N_cheb^d + k + 1 entries.

Derivatives (from the definition, entry by entry):
  dK_ij/dTheta_t   = (T_t(x_i) + T_t(x_j)) K_ij,  T_t(x) = prod_k T_{t_k}(x^k)
  dK_ij/dlog l_k   = K_ij (x_ik - x_jk)^2 / l_k^2  (isotropic: summed over k)
  dA/dlog sigma^2  = sigma^2 I

Parity status: pinned (the cosine form of T_n, a hand-evaluated amplitude, the
N_cheb = 1 reduction to the stationary kernel, the amplitude/correlation split,
positive definiteness, and central differences of u^T A v for the derivatives) -
see tests/test_oracle_cheb.py.
"""
from __future__ import annotations

import itertools

import numpy as np

from .se_kernel import scaled_sq_dist


def cheb_T(n: int, x):
    """T_n(x) by the three-term recurrence T_0 = 1, T_1 = x, T_{k+1} = 2 x T_k - T_{k-1}."""
    x = np.asarray(x, np.float64)
    t_prev, t = np.ones_like(x), x.copy()
    if n == 0:
        return t_prev
    for _ in range(n - 1):
        t_prev, t = t, 2.0 * x * t - t_prev
    return t


def n_coeffs(n_cheb: int, d: int) -> int:
    return n_cheb ** d


def unpack_theta(theta, d: int, n_cheb: int, ard: bool):
    """Return (Theta[N_cheb]*d, ell[d], sigma2)."""
    theta = np.asarray(theta, np.float64)
    nc = n_coeffs(n_cheb, d)
    k = d if ard else 1
    if theta.shape != (nc + k + 1,):
        raise ValueError(f"theta must have {nc + k + 1} entries, got {theta.shape}")
    Theta = theta[:nc].reshape((n_cheb,) * d)
    ell = np.exp(theta[nc:nc + k])
    if not ard:
        ell = np.full(d, ell[0])
    sigma2 = float(np.exp(theta[nc + k]))
    return Theta, ell, sigma2


def basis(X, n_cheb: int):
    """B[i, t] = T_t(x_i) for every multi-index t in row-major order (i_1 slowest)."""
    X = np.asarray(X, np.float64)
    n, d = X.shape
    out = np.zeros((n, n_coeffs(n_cheb, d)))
    for col, idx in enumerate(itertools.product(range(n_cheb), repeat=d)):
        v = np.ones(n)
        for k in range(d):
            v = v * cheb_T(idx[k], X[:, k])
        out[:, col] = v
    return out


def log_amplitude(X, theta, n_cheb: int, ard: bool):
    """C_theta(x_i) for every point (Sec. 4)."""
    X = np.asarray(X, np.float64)
    Theta, _, _ = unpack_theta(theta, X.shape[1], n_cheb, ard)
    return basis(X, n_cheb) @ Theta.reshape(-1)


def kernel_matrix(X, theta, n_cheb: int, ard: bool):
    """K[i, j] = e^{C_i} e^{C_j} exp(-r2_ij / 2)."""
    X = np.asarray(X, np.float64)
    _, ell, _ = unpack_theta(theta, X.shape[1], n_cheb, ard)
    a = np.exp(log_amplitude(X, theta, n_cheb, ard))
    return a[:, None] * a[None, :] * np.exp(-0.5 * scaled_sq_dist(X, X, ell))


def A_matrix(X, theta, n_cheb: int, ard: bool):
    """Dense A = K + sigma^2 I."""
    _, _, sigma2 = unpack_theta(theta, np.shape(X)[1], n_cheb, ard)
    K = kernel_matrix(X, theta, n_cheb, ard)
    return K + sigma2 * np.eye(K.shape[0])


def dA_dtheta(X, theta, n_cheb: int, ard: bool):
    """dA/dtheta_p as dense N x N matrices, in the order of theta."""
    X = np.asarray(X, np.float64)
    n, d = X.shape
    _, ell, sigma2 = unpack_theta(theta, d, n_cheb, ard)
    K = kernel_matrix(X, theta, n_cheb, ard)
    B = basis(X, n_cheb)
    mats = [(B[:, t, None] + B[None, :, t]) * K for t in range(B.shape[1])]
    per_dim = [K * ((X[:, k, None] - X[None, :, k]) / ell[k]) ** 2 for k in range(d)]
    if ard:
        mats.extend(per_dim)
    else:
        mats.append(sum(per_dim))
    mats.append(sigma2 * np.eye(n))
    return mats


def kmv(X, theta, V, n_cheb: int, ard: bool, col_shift=None):
    """A V (columns shifted by col_shift when given)."""
    V = np.asarray(V, np.float64)
    out = A_matrix(X, theta, n_cheb, ard) @ V
    if col_shift is not None:
        out = out + np.asarray(col_shift, np.float64)[None, :] * V
    return out


def kmv_adjoint(X, theta, V, G, n_cheb: int, ard: bool):
    """(grad_theta, grad_V) of L = sum G o (A V): grad_p = sum_c G_c^T (dA/dtheta_p) V_c, grad_V = A G."""
    V = np.asarray(V, np.float64)
    G = np.asarray(G, np.float64)
    if V.ndim == 1:
        V, G = V[:, None], G[:, None]
    g = np.array([float(np.sum(G * (M @ V))) for M in dA_dtheta(X, theta, n_cheb, ard)])
    return g, A_matrix(X, theta, n_cheb, ard) @ G

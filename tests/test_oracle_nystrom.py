"""Pins for oracle/nystrom.py (the randomized Nystrom preconditioner the paper
uses for its solves): exactness on kernels of rank <= r, K - K_hat PSD, the
closed-form spectrum of P^{-1} A when K_hat = K, P^{-1} = I without a range,
and PCG against a dense solve."""
import math

import numpy as np

from oracle import nystrom as ny
from oracle import se_kernel as sk


def _low_rank_kernel(rng, n, k):
    F = rng.standard_normal((n, k))
    return F @ F.T


def test_exact_on_kernels_of_rank_at_most_r():
    rng = np.random.default_rng(1)
    K = _low_rank_kernel(rng, 80, 6)
    U, lam = ny.nystrom(K, rng.standard_normal((80, 10)), eps=2.0 ** -52)
    K_hat = U @ np.diag(lam) @ U.T
    assert np.linalg.norm(K_hat - K) <= 1e-9 * np.linalg.norm(K)
    # the top eigenvalues are those of K, the rest vanish
    ev = np.sort(np.linalg.eigvalsh(K))[::-1]
    np.testing.assert_allclose(lam[:6], ev[:6], rtol=1e-9)
    assert np.all(lam[6:] <= 1e-9 * ev[0])


def test_approximation_is_below_the_kernel():
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, size=(120, 2))
    K = sk.kernel_matrix(X, X, np.array([0.0, math.log(0.4), math.log(0.01)]), ard=False)
    U, lam = ny.nystrom(K, rng.standard_normal((120, 15)), eps=2.0 ** -52)
    K_hat = U @ np.diag(lam) @ U.T
    gap = np.linalg.eigvalsh(K - K_hat)
    assert gap.min() >= -1e-8 * np.linalg.norm(K, 2)
    assert np.all(lam >= 0) and np.all(np.diff(lam) <= 0)
    np.testing.assert_allclose(U.T @ U, np.eye(15), atol=1e-10)


def test_preconditioned_spectrum_when_the_approximation_is_exact():
    # K_hat = K of rank 5: P^{-1} A = (lambda_5 + mu) on range(U) and mu on its complement
    rng = np.random.default_rng(3)
    K = _low_rank_kernel(rng, 60, 5)
    mu = 0.3
    U, lam = ny.nystrom(K, rng.standard_normal((60, 5)), eps=2.0 ** -52)
    A = K + mu * np.eye(60)
    PA = np.column_stack([ny.precond_apply(U, lam, mu, A[:, j]) for j in range(60)])
    ev = np.sort(np.linalg.eigvals(PA).real)
    np.testing.assert_allclose(ev[:55], mu, rtol=1e-9)
    np.testing.assert_allclose(ev[55:], lam[-1] + mu, rtol=1e-9)


def test_no_range_is_the_identity():
    r = np.random.default_rng(4).standard_normal(30)
    U = np.zeros((30, 3))
    lam = np.zeros(3)
    np.testing.assert_allclose(ny.precond_apply(U, lam, 0.1, r), r, rtol=0, atol=0)


def test_pcg_matches_dense_solve_and_needs_fewer_iterations():
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, size=(300, 2))
    th = np.array([0.0, math.log(0.5), math.log(1e-3)])
    A = sk.A_matrix(X, th, ard=False)
    K = A - 1e-3 * np.eye(300)
    b = rng.standard_normal(300)
    U, lam = ny.nystrom(K, rng.standard_normal((300, 40)))
    x_p, it_p = ny.pcg(A, b, lambda r: ny.precond_apply(U, lam, 1e-3, r), 1e-10, 2000)
    x_c, it_c = ny.pcg(A, b, lambda r: r, 1e-10, 5000)
    x_ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x_p - x_ref) <= 1e-6 * np.linalg.norm(x_ref)
    assert it_p * 3 < it_c, (it_p, it_c)

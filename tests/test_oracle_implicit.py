"""Pins for oracle/implicit.py (the implicit midpoint step of Sec. 3.2.3 solved by
Anderson acceleration, App. B): the Walker-Ni equivalence with GMRES on a linear
map, the fixed point against the implicit equations with Cholesky solves and the
direct force, reversibility, second order against the leapfrog map, fixed
components."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import hmc
from oracle import implicit as im
from oracle import se_kernel as sk


def _gmres_iterate(A, b, n):
    """argmin over y in span{b, Ab, .., A^{n-1} b} of |b - A y| (y_0 = 0)."""
    if n == 0:
        return np.zeros_like(b)
    Kr = np.column_stack([np.linalg.matrix_power(A, j) @ b for j in range(n)])
    Q, _ = np.linalg.qr(Kr)
    c = np.linalg.lstsq(A @ Q, b, rcond=None)[0]
    return Q @ c


def test_anderson_full_history_is_gmres_on_a_linear_map():
    rng = np.random.default_rng(1)
    B = rng.standard_normal((12, 12))
    A = np.eye(12) + 0.3 * (B + B.T) / np.sqrt(12)          # eigenvalues in (0, 2): g contracts
    b = rng.standard_normal(12)
    g_lin = lambda x: (np.eye(12) - A) @ x + b
    seen = []

    def g(x):
        seen.append(x.copy())
        return g_lin(x)

    im.anderson(g, np.zeros(12), k=50, tol=0.0, maxiter=6)
    # x_{n+1} = g(y_n), y_n the n-th GMRES iterate
    for n in range(5):
        np.testing.assert_allclose(seen[n + 1], g_lin(_gmres_iterate(A, b, n)), rtol=1e-8, atol=1e-10)


def _setup(seed=3, n=40):
    w = wl.ragged([n], d=2, chains=1, m=1, ard=True, seed=seed, sigma2=0.1)
    X, y = w.X, w.y
    th0 = w.theta[0]
    rng = np.random.default_rng(seed + 1)
    phi = rng.standard_normal(n)
    pi0 = 0.5 * rng.standard_normal(th0.size)
    A0 = sk.A_matrix(X, th0, True)
    R = np.eye(n) / np.linalg.eigvalsh(A0)[-1]
    return X, y, phi, th0, pi0, R


def test_fixed_point_solves_the_implicit_equations():
    X, y, phi, th0, pi0, R = _setup()
    dt = 0.05
    th1, pi1, x, it = im.implicit_midpoint(X, y, phi, th0, pi0, dt, True, R, k=10, tol=1e-13, maxiter=2000)
    assert it < 2000
    tbar = 0.5 * (th0 + th1)
    A = sk.A_matrix(X, tbar, True)
    assert np.linalg.norm(A @ x - y) <= 1e-10 * np.linalg.norm(y)
    np.testing.assert_allclose(th1, th0 + dt * 0.5 * (pi0 + pi1), rtol=0, atol=1e-12)
    # the direct force (Cholesky solve inside) at the midpoint
    np.testing.assert_allclose(pi1, pi0 - dt * hmc.force(X, y, phi, tbar, True), rtol=0, atol=1e-8)


def test_midpoint_map_is_reversible():
    X, y, phi, th0, pi0, R = _setup(seed=5)
    dt = 0.05
    th1, pi1, x, _ = im.implicit_midpoint(X, y, phi, th0, pi0, dt, True, R, tol=1e-13, maxiter=2000)
    th2, pi2, _, _ = im.implicit_midpoint(X, y, phi, th1, -pi1, dt, True, R, tol=1e-13, maxiter=2000, x0=x)
    np.testing.assert_allclose(th2, th0, rtol=0, atol=1e-9)
    np.testing.assert_allclose(-pi2, pi0, rtol=0, atol=1e-8)


def test_second_order_agreement_with_leapfrog():
    X, y, phi, th0, pi0, R = _setup(seed=7)
    diffs = []
    for dt in (0.04, 0.02):
        th_m, pi_m, _, _ = im.implicit_midpoint(X, y, phi, th0, pi0, dt, True, R, tol=1e-13, maxiter=2000)
        th_l, pi_l = hmc.leapfrog(X, y, phi, th0, pi0, dt, True)
        diffs.append(np.linalg.norm(th_m - th_l) + np.linalg.norm(pi_m - pi_l))
    # two second-order one-step maps differ by O(dt^3)
    assert 5.0 < diffs[0] / diffs[1] < 12.0, diffs


def test_fixed_components_stay():
    X, y, phi, th0, pi0, R = _setup(seed=9)
    free = np.array([1, 1, 0, 1], np.float64)
    th1, pi1, _, _ = im.implicit_midpoint(X, y, phi, th0, pi0, 0.05, True, R, tol=1e-12, maxiter=2000, free=free)
    assert th1[2] == th0[2] and pi1[2] == pi0[2]

"""Pins for oracle/cheb_kernel.py (the Chebyshev log-amplitude kernel of Sec. 4):
the cosine form of T_n, hand-evaluated amplitudes (including the index order of
Theta), the N_cheb = 1 reduction to the stationary kernel, the split of K into
amplitudes and a stationary correlation, positive definiteness, and central
differences of u^T A v for every derivative."""
import math

import numpy as np
import pytest

from oracle import cheb_kernel as ck
from oracle import hmc
from oracle import se_kernel as sk


def test_chebyshev_polynomials_match_cosine_form():
    # T_n(cos t) = cos(n t): a formula independent of the recurrence
    t = np.linspace(0.0, math.pi, 37)
    for n in range(9):
        np.testing.assert_allclose(ck.cheb_T(n, np.cos(t)), np.cos(n * t), atol=1e-13)


def test_amplitude_hand_evaluated_and_index_order():
    # d = 2, N_cheb = 3, only Theta[1, 2] = 0.3 at x = (0.5, -0.25):
    # T_1(0.5) = 0.5, T_2(-0.25) = 2 * 0.0625 - 1 = -0.875 -> C = 0.3 * 0.5 * -0.875
    X = np.array([[0.5, -0.25]])
    theta = np.zeros(9 + 2)
    theta[1 * 3 + 2] = 0.3
    assert ck.log_amplitude(X, theta, 3, ard=False)[0] == pytest.approx(-0.13125, rel=1e-15)
    # the transposed index multiplies T_2(0.5) T_1(-0.25) = (-0.5) (-0.25) instead
    theta2 = np.zeros(9 + 2)
    theta2[2 * 3 + 1] = 0.3
    assert ck.log_amplitude(X, theta2, 3, ard=False)[0] == pytest.approx(0.0375, rel=1e-15)
    # K_ii = exp(2 C(x_i)) (the stationary factor is 1 on the diagonal)
    K = ck.kernel_matrix(X, theta, 3, ard=False)
    assert K[0, 0] == pytest.approx(math.exp(-0.2625), rel=1e-15)


def test_order_one_is_the_stationary_kernel():
    # N_cheb = 1: C = Theta_0 everywhere, K = e^{2 Theta_0} SE, i.e. log alpha = 2 Theta_0
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, size=(40, 3))
    th = np.array([0.35, math.log(0.7), math.log(0.05)])
    th_se = np.array([0.7, math.log(0.7), math.log(0.05)])
    np.testing.assert_allclose(ck.A_matrix(X, th, 1, ard=False), sk.A_matrix(X, th_se, ard=False), rtol=1e-14)


def test_amplitude_times_stationary_correlation():
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, size=(30, 2))
    theta = np.concatenate([0.3 * rng.standard_normal(16), [math.log(0.5), math.log(0.3), math.log(0.01)]])
    K = ck.kernel_matrix(X, theta, 4, ard=True)
    d = np.sqrt(np.diag(K))
    corr = K / d[:, None] / d[None, :]
    ell = np.array([0.5, 0.3])
    r2 = (((X[:, None, :] - X[None, :, :]) / ell) ** 2).sum(-1)
    np.testing.assert_allclose(corr, np.exp(-0.5 * r2), rtol=1e-13)
    np.testing.assert_allclose(np.log(d), ck.log_amplitude(X, theta, 4, ard=True), rtol=1e-13, atol=1e-14)


def test_positive_definite():
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, size=(60, 2))
    theta = np.concatenate([0.5 * rng.standard_normal(9), [math.log(0.4), math.log(0.02)]])
    A = ck.A_matrix(X, theta, 3, ard=False)
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() >= 0.02 * (1 - 1e-9)


@pytest.mark.parametrize("ard", [False, True])
def test_derivatives_by_central_differences(ard):
    rng = np.random.default_rng(4)
    d, nc = 2, 3
    X = rng.uniform(-1, 1, size=(25, d))
    k = d if ard else 1
    theta = np.concatenate([0.3 * rng.standard_normal(nc ** d), np.log(rng.uniform(0.3, 1.0, k)),
                            [math.log(0.05)]])
    u, v = rng.standard_normal(25), rng.standard_normal(25)
    g, gV = ck.kmv_adjoint(X, theta, v, u, nc, ard)
    h = 1e-6
    for p in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        fd = (u @ ck.A_matrix(X, tp, nc, ard) @ v - u @ ck.A_matrix(X, tm, nc, ard) @ v) / (2 * h)
        assert g[p] == pytest.approx(fd, rel=1e-6, abs=1e-8), p
    np.testing.assert_allclose(gV[:, 0], ck.A_matrix(X, theta, nc, ard) @ u, rtol=1e-14)


def test_force_of_the_family_is_the_gradient_of_the_potential():
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, size=(30, 2))
    theta = np.concatenate([0.2 * rng.standard_normal(4), [math.log(0.5), math.log(0.05)]])
    y, phi = rng.standard_normal(30), rng.standard_normal(30)
    kern = (lambda X_, t: ck.A_matrix(X_, t, 2, False), lambda X_, t: ck.dA_dtheta(X_, t, 2, False))
    F = hmc.force(X, y, phi, theta, False, kern=kern)
    h = 1e-6
    for p in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        fd = (hmc.potential(X, y, phi, tp, False, kern=kern) - hmc.potential(X, y, phi, tm, False, kern=kern)) / (2 * h)
        assert F[p] == pytest.approx(fd, rel=1e-6, abs=1e-7), p

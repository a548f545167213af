"""Pins for oracle/se_kernel.py: values fixed by the kernel's definition (Sec. 1,
Eq. kerdef), its limits and invariances, and finite differences for the adjoint."""
import math

import numpy as np
import pytest

from oracle import se_kernel as sk
import workloads as wl


def test_two_point_closed_form_isotropic():
    # x = (0, 1), alpha = 2, l = 1, sigma^2 = 0.5:
    # A = [[alpha + s2, alpha e^{-1/2}], [alpha e^{-1/2}, alpha + s2]]
    X = np.array([[0.0], [1.0]])
    th = np.array([math.log(2.0), 0.0, math.log(0.5)])
    A = sk.A_matrix(X, th, ard=False)
    off = 2.0 * 0.6065306597126334          # e^{-1/2}
    np.testing.assert_allclose(A, [[2.5, off], [off, 2.5]], rtol=1e-15)


def test_two_point_closed_form_ard():
    # x0 = (0, 0), x1 = (1, 2), l = (1, 2): scaled distance 1 + 1 = 2 -> e^{-1}
    X = np.array([[0.0, 0.0], [1.0, 2.0]])
    th = np.array([0.0, 0.0, math.log(2.0), math.log(0.1)])
    K = sk.kernel_matrix(X, X, th, ard=True)
    assert K[0, 1] == pytest.approx(0.36787944117144233, rel=1e-15)
    assert K[0, 0] == 1.0


def test_symmetric_positive_definite():
    w = wl.ragged([150], d=3, chains=1, m=1, seed=3)
    A = sk.A_matrix(w.X, w.theta[0], ard=True)
    assert np.array_equal(A, A.T)
    s2 = math.exp(w.theta[0, -1])
    assert np.linalg.eigvalsh(A).min() >= s2 * (1 - 1e-9)


def test_matvec_of_unit_vector_is_column():
    w = wl.ragged([70], d=2, chains=1, m=1, seed=4)
    A = sk.A_matrix(w.X, w.theta[0], ard=True)
    E = np.eye(70)[:, [0, 17, 69]]
    Y = sk.kmv(w.X, w.theta[0], E, ard=True, block=16)
    np.testing.assert_array_equal(Y, A[:, [0, 17, 69]])


def test_lengthscale_limits():
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, (40, 2))
    V = rng.standard_normal((40, 3))
    alpha, s2 = 1.7, 0.3
    # l -> infinity: K -> alpha 1 1^T
    th = np.array([math.log(alpha), 30.0, math.log(s2)])
    Y = sk.kmv(X, th, V, ard=False)
    np.testing.assert_allclose(Y, alpha * np.ones((40, 1)) * V.sum(0) + s2 * V, rtol=1e-12)
    # l -> 0 with distinct points: K -> alpha I
    th = np.array([math.log(alpha), -30.0, math.log(s2)])
    np.testing.assert_allclose(sk.kmv(X, th, V, ard=False), (alpha + s2) * V, rtol=1e-15)


def test_ard_with_equal_lengthscales_is_isotropic():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((50, 4))
    iso = np.array([0.3, math.log(0.7), math.log(0.05)])
    ard = np.array([0.3] + [math.log(0.7)] * 4 + [math.log(0.05)])
    np.testing.assert_allclose(sk.A_matrix(X, iso, False), sk.A_matrix(X, ard, True), rtol=1e-14)


def test_permutation_and_translation_invariance():
    w = wl.ragged([60], d=3, chains=1, m=2, seed=5)
    th = w.theta[0]
    V = w.V[0]
    perm = np.random.default_rng(0).permutation(60)
    Y = sk.kmv(w.X, th, V, True)
    Yp = sk.kmv(w.X[perm] + np.array([3.0, -1.0, 0.5]), th, V[perm], True)
    np.testing.assert_allclose(Yp, Y[perm], rtol=1e-12, atol=1e-13)


def test_linear_in_alpha():
    w = wl.ragged([30], d=2, chains=1, m=1, seed=6)
    th = w.theta[0].copy()
    K1 = sk.kernel_matrix(w.X, w.X, th, True)
    th[0] += math.log(3.0)
    np.testing.assert_allclose(sk.kernel_matrix(w.X, w.X, th, True), 3.0 * K1, rtol=1e-14)


def test_col_shift_is_shifted_operator():
    w = wl.ragged([45], d=2, chains=1, m=3, seed=7)
    th = w.theta[0]
    A = sk.A_matrix(w.X, th, True)
    s = np.array([0.0, 0.5, 3.0])
    Y = sk.kmv(w.X, th, w.V[0], True, col_shift=s)
    for c in range(3):
        np.testing.assert_allclose(Y[:, c], (A + s[c] * np.eye(45)) @ w.V[0][:, c], rtol=1e-12)


@pytest.mark.parametrize("ard", [False, True])
def test_adjoint_theta_matches_central_differences(ard):
    w = wl.ragged([55], d=3, chains=1, m=2, ard=ard, seed=8)
    th, V, G = w.theta[0], w.V[0], w.G[0]

    def L(t):
        return float(np.sum(G * sk.kmv(w.X, t, V, ard)))

    g, _ = sk.kmv_adjoint(w.X, th, V, G, ard)
    h = 1e-5
    fd = np.array([(L(th + h * e) - L(th - h * e)) / (2 * h) for e in np.eye(len(th))])
    np.testing.assert_allclose(g, fd, rtol=1e-7, atol=1e-7 * np.abs(fd).max())


def test_adjoint_V_matches_directional_derivative():
    w = wl.ragged([40], d=2, chains=1, m=3, seed=9)
    th, V, G = w.theta[0], w.V[0], w.G[0]
    _, gV = sk.kmv_adjoint(w.X, th, V, G, True)
    D = np.random.default_rng(3).standard_normal(V.shape)
    # L is linear in V, so the directional derivative is exact
    dL = float(np.sum(G * sk.kmv(w.X, th, D, True)))
    assert float(np.sum(gV * D)) == pytest.approx(dL, rel=1e-12)


def test_adjoint_alpha_and_noise_identities():
    w = wl.ragged([35], d=2, chains=1, m=2, seed=10)
    th, V, G = w.theta[0], w.V[0], w.G[0]
    g, _ = sk.kmv_adjoint(w.X, th, V, G, True)
    s2 = math.exp(th[-1])
    L = float(np.sum(G * sk.kmv(w.X, th, V, True)))
    noise = s2 * float(np.sum(G * V))
    assert g[-1] == pytest.approx(noise, rel=1e-13)
    # L is alpha * (K0 part) + noise part, so dL/dlog alpha is the K part of L
    assert g[0] == pytest.approx(L - noise, rel=1e-12)


def test_isotropic_lengthscale_gradient_is_sum_of_ard():
    w = wl.ragged([30], d=3, chains=1, m=1, seed=11)
    V, G = w.V[0], w.G[0]
    iso = np.array([0.2, math.log(0.6), math.log(0.05)])
    ard = np.array([0.2] + [math.log(0.6)] * 3 + [math.log(0.05)])
    gi, _ = sk.kmv_adjoint(w.X, iso, V, G, False)
    ga, _ = sk.kmv_adjoint(w.X, ard, V, G, True)
    assert gi[1] == pytest.approx(ga[1:4].sum(), rel=1e-12)


def test_sampled_row_adjoint_is_exact():
    w = wl.ragged([80], d=2, chains=1, m=2, seed=12)
    th, V = w.theta[0], w.V[0]
    rows = np.array([3, 40, 79])
    G = np.zeros_like(V)
    G[rows] = w.G[0][rows]
    g_full, gV_full = sk.kmv_adjoint(w.X, th, V, G, True)
    g_rows, gV_rows = sk.kmv_adjoint(w.X, th, V, G, True, rows=rows)
    np.testing.assert_allclose(g_rows, g_full, rtol=1e-12)
    np.testing.assert_allclose(gV_rows, gV_full, rtol=1e-12, atol=1e-15)


def test_quad_form_grad_matches_adjoint():
    w = wl.ragged([25], d=2, chains=1, m=1, seed=13)
    z = w.V[0][:, 0]
    g1 = sk.quad_form_grad(w.X, w.theta[0], z, True)
    g2, _ = sk.kmv_adjoint(w.X, w.theta[0], z, z, True)
    np.testing.assert_allclose(g1, g2, rtol=1e-12)

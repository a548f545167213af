"""Pins for oracle/poles.py (App. A) and oracle/diagnostics.py (Sec. 4.1, App. C)."""
import math

import numpy as np
import pytest
from scipy.special import ellipk
from scipy.stats import norm

from oracle import poles, diagnostics as dg, se_kernel as sk
import workloads as wl


@pytest.mark.parametrize("kappa,tol", [(5e2, 1e-12), (1e5, 1e-7), (1e7, 5e-6)])
def test_pole_expansion_scalar_error(kappa, tol):
    # sum_j w_j / (lam + lambda_j) must reproduce lam^{-1/2} on the whole interval [m, M]
    m_lo, M_hi = 0.05, 0.05 * kappa
    w, s = poles.pole_weights_shifts(m_lo, M_hi, 15)
    assert np.all(s >= 0) and np.all(w > 0)
    lam = np.geomspace(m_lo, M_hi, 2001)
    rel = np.abs(poles.inv_sqrt_scalar(lam, w, s) * np.sqrt(lam) - 1.0)
    assert rel.max() < tol


def test_pole_expansion_convergence_rate():
    # App. A: error O(exp(-2 pi K N_p / K')), K = K(k^2), K' = K(1 - k^2)
    m_lo, M_hi = 1.0, 1e6
    lam = np.geomspace(m_lo, M_hi, 3001)
    errs = []
    for npl in (4, 8):
        w, s = poles.pole_weights_shifts(m_lo, M_hi, npl)
        errs.append(np.abs(poles.inv_sqrt_scalar(lam, w, s) * np.sqrt(lam) - 1).max())
    k2 = m_lo / M_hi
    rate = 2 * math.pi * ellipk(k2) / ellipk(1 - k2)
    observed = math.log(errs[0] / errs[1]) / 4
    assert observed == pytest.approx(rate, rel=0.25)


def test_pole_expansion_matrix_matches_eigendecomposition():
    w = wl.ragged([300], d=2, chains=1, m=1, seed=31)
    A = sk.A_matrix(w.X, w.theta[0], True)
    ev = np.linalg.eigvalsh(A)
    s2 = math.exp(w.theta[0, -1])
    M_hi = float(np.abs(A).sum(1).max())       # ||A||_inf >= lambda_max for this entrywise-nonnegative A
    assert M_hi >= ev.max()
    xi = np.random.default_rng(4).standard_normal(300)
    got = poles.inv_sqrt_apply(A, xi, s2, M_hi)
    evals, Q = np.linalg.eigh(A)
    exact = Q @ ((Q.T @ xi) / np.sqrt(evals))
    wts, sh = poles.pole_weights_shifts(s2, M_hi, 15)
    scal = np.abs(poles.inv_sqrt_scalar(ev, wts, sh) - ev ** -0.5).max()
    # truncation bound of the scalar expansion plus the rounding of the dense solves
    rounding = 50 * np.finfo(float).eps * (ev.max() / ev.min()) * np.linalg.norm(exact)
    assert np.linalg.norm(got - exact) <= 1.01 * scal * np.linalg.norm(xi) + rounding
    assert np.linalg.norm(got - exact) < 1e-8 * np.linalg.norm(exact)


def test_iat_of_ar1_process():
    rho, n = 0.8, 200000
    rng = np.random.default_rng(5)
    e = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = e[0] / math.sqrt(1 - rho * rho)
    for i in range(1, n):
        x[i] = rho * x[i - 1] + e[i]
    assert dg.iat(x) == pytest.approx((1 + rho) / (1 - rho), rel=0.1)


def test_iat_of_independent_samples_is_one():
    x = np.random.default_rng(6).standard_normal(50000)
    assert dg.iat(x) == pytest.approx(1.0, abs=0.1)


def test_moving_window_mean_of_consecutive_integers():
    # mean of floor(i/2) .. i for the sequence X_k = k is (floor(i/2) + i) / 2
    xs = np.arange(101, dtype=float)
    T = dg.moving_window_mean(xs)
    np.testing.assert_allclose(T, [(i // 2 + i) / 2 for i in range(101)])


def test_marginal_cdf_of_gaussian_grid():
    g = np.linspace(-9, 9, 601)
    a, b = np.meshgrid(g, g, indexing="ij")
    logp = -0.5 * ((a - 0.5) ** 2 / 0.64 + (b + 1.0) ** 2 / 2.25)
    c0 = dg.marginal_cdf_grid(logp, g, 0)
    c1 = dg.marginal_cdf_grid(logp, g, 1)
    np.testing.assert_allclose(c0, norm.cdf(g, 0.5, 0.8), atol=2e-4)
    np.testing.assert_allclose(c1, norm.cdf(g, -1.0, 1.5), atol=2e-4)


@pytest.mark.parametrize("ard", [False, True])
def test_spectral_interval_contains_the_spectrum(ard):
    # App. A needs [m, M] to contain every eigenvalue of A: m = sigma^2 <= lambda_min,
    # M = max row sum >= lambda_max (K0 >= 0 entrywise), with M - lambda_max small
    # for a smooth kernel on clustered points
    w = wl.ragged([240], d=3, chains=1, m=1, ard=ard, seed=41)
    A = sk.A_matrix(w.X, w.theta[0], ard)
    lam = np.linalg.eigvalsh(A)
    m_lo, M_hi = poles.spectral_interval(w.X, w.theta[0], ard)
    assert m_lo == pytest.approx(math.exp(w.theta[0][-1]), rel=1e-15)
    assert m_lo <= lam[0] * (1 + 1e-12)
    assert lam[-1] <= M_hi * (1 + 1e-12)
    # for the all-equal-points limit (rank-one K0) the row sum is the top eigenvalue exactly
    X1 = np.zeros((16, 2))
    th = np.array([math.log(2.0), math.log(0.5), math.log(0.1)])
    m1, M1 = poles.spectral_interval(X1, th, False)
    assert M1 == pytest.approx(2.0 * 16 + 0.1, rel=1e-14)
    assert np.linalg.eigvalsh(sk.A_matrix(X1, th, False))[-1] == pytest.approx(M1, rel=1e-12)


def test_phi_pole_matches_inverse_square_root():
    # the pole-expansion draw equals A^{-1/2} xi within the scalar error of the
    # expansion on [m, M] (App. A) times |xi|
    w = wl.ragged([200], d=2, chains=1, m=1, ard=True, seed=43)
    xi = np.random.default_rng(7).standard_normal(200)
    m_lo, M_hi = poles.spectral_interval(w.X, w.theta[0], True)
    for npl in (8, 15):
        phi = poles.phi_pole(w.X, w.theta[0], xi, True, npl)
        exact = sk_hmc_phi(w, xi)
        wts, sh = poles.pole_weights_shifts(m_lo, M_hi, npl)
        lam = np.geomspace(m_lo, M_hi, 4001)
        scal = np.abs(poles.inv_sqrt_scalar(lam, wts, sh) - lam ** -0.5).max()
        assert np.linalg.norm(phi - exact) <= 1.01 * scal * np.linalg.norm(xi) + 1e-10


def sk_hmc_phi(w, xi):
    from oracle import hmc
    return hmc.phi_exact(w.X, w.theta[0], xi, True)

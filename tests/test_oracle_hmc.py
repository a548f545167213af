"""Pins for oracle/hmc.py: finite differences of U for the force (Sec. 3.2.1), the
Gaussian identity behind the augmentation (Sec. 3), reversibility / volume
preservation / O(dt^2) energy error of the leapfrog map (Sec. 3.2.2), and the
tiny-N sampler of Algorithm 1 against quadrature of Eq. P (the design of Sec. 4.1)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import hmc, se_kernel as sk, diagnostics as dg
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "verification_sec41.json")


def _problem(n=24, d=2, seed=21):
    w = wl.ragged([n], d=d, chains=1, m=1, seed=seed)
    rng = np.random.default_rng(seed)
    phi = rng.standard_normal(n)
    return w.X, w.y, phi, w.theta[0]


@pytest.mark.parametrize("prior", [None, {"mu": np.zeros(4), "prec": np.array([1.0, 2.0, 0.5, 1.0])}])
def test_force_is_gradient_of_potential(prior):
    X, y, phi, th = _problem()
    F = hmc.force(X, y, phi, th, True, prior)
    h = 1e-5
    fd = np.array([(hmc.potential(X, y, phi, th + h * e, True, prior)
                    - hmc.potential(X, y, phi, th - h * e, True, prior)) / (2 * h) for e in np.eye(len(th))])
    np.testing.assert_allclose(F, fd, rtol=1e-6, atol=1e-7 * np.abs(fd).max())


def test_force_equals_frozen_x_quadratic_form_gradient():
    # Sec. 3.2.1: F = grad_theta u(theta, x) at x = A^{-1} y, u = S - x^T A x / 2 + phi^T A phi / 2
    X, y, phi, th = _problem()
    x = hmc.solve(X, th, y, True)
    V = np.stack([x, phi], axis=1)
    G = np.stack([-0.5 * x, 0.5 * phi], axis=1)
    g, _ = sk.kmv_adjoint(X, th, V, G, True)
    np.testing.assert_allclose(hmc.force(X, y, phi, th, True), g, rtol=1e-9, atol=1e-12)


def test_gaussian_identity_monte_carlo():
    # int exp(-z^T A z / 2) dz = (2 pi)^{N/2} det(A)^{-1/2}; log_posterior with y = 0 and
    # a flat prior is -log det(A) / 2, so it must reproduce the integral.
    X = np.array([[0.0], [0.4], [1.1]])
    th = np.array([0.0, math.log(0.5), math.log(0.2)])
    A = sk.A_matrix(X, th, False)
    n = 3
    lam_min = np.linalg.eigvalsh(A).min()
    s2 = 1.0 / lam_min
    rng = np.random.default_rng(0)
    z = math.sqrt(s2) * rng.standard_normal((400000, n))
    log_q = -0.5 * np.sum(z * z, 1) / s2 - 0.5 * n * math.log(2 * math.pi * s2)
    wts = np.exp(-0.5 * np.einsum("si,ij,sj->s", z, A, z) - log_q)
    est, se = wts.mean(), wts.std() / math.sqrt(len(wts))
    exact = math.exp(0.5 * n * math.log(2 * math.pi) + hmc.log_posterior(X, np.zeros(n), th, False))
    assert abs(est - exact) < 4 * se
    assert se / exact < 0.01


def test_gibbs_draw_has_covariance_inverse_A():
    X = np.array([[0.0], [0.3], [0.9], [1.4]])
    th = np.array([0.2, math.log(0.6), math.log(0.3)])
    A = sk.A_matrix(X, th, False)
    rng = np.random.default_rng(1)
    xi = rng.standard_normal((4, 200000))
    phi = hmc.inv_sqrt_apply(A, xi)
    C = phi @ phi.T / xi.shape[1]
    Ainv = np.linalg.inv(A)
    np.testing.assert_allclose(C, Ainv, atol=0.02 * np.abs(Ainv).max())


def test_leapfrog_is_reversible():
    X, y, phi, th = _problem()
    pi = np.random.default_rng(2).standard_normal(len(th))
    t1, p1 = hmc.leapfrog(X, y, phi, th, pi, 0.05, True, n_steps=3)
    t2, p2 = hmc.leapfrog(X, y, phi, t1, -p1, 0.05, True, n_steps=3)
    np.testing.assert_allclose(t2, th, atol=1e-10)
    np.testing.assert_allclose(-p2, pi, atol=1e-10)


def test_leapfrog_preserves_volume():
    X, y, phi, th = _problem(n=12, d=1)
    pi = np.array([0.3, -0.2, 0.1])
    z0 = np.concatenate([th, pi])
    n = len(th)

    def step(z):
        t, p = hmc.leapfrog(X, y, phi, z[:n], z[n:], 0.1, False)
        return np.concatenate([t, p])

    h = 1e-6
    J = np.stack([(step(z0 + h * e) - step(z0 - h * e)) / (2 * h) for e in np.eye(2 * n)], axis=1)
    assert np.linalg.det(J) == pytest.approx(1.0, abs=1e-6)


def test_leapfrog_energy_error_is_second_order():
    X, y, phi, th = _problem(n=20, d=1, seed=30)
    pi = np.array([0.5, -0.4, 0.3])
    H0 = hmc.hamiltonian(X, y, phi, th, pi, False)
    errs = []
    for k, dt in enumerate([0.04, 0.02, 0.01]):
        t1, p1 = hmc.leapfrog(X, y, phi, th, pi, dt, False, n_steps=10 * 2 ** k)
        errs.append(abs(hmc.hamiltonian(X, y, phi, t1, p1, False) - H0))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.2 < r1 < 4.8 and 3.2 < r2 < 4.8


def test_accept_rule_boundary():
    assert hmc.accept(1.0, 2.0, math.exp(-1.0))          # X == acceptance probability accepts
    assert not hmc.accept(1.0, 2.0, math.exp(-1.0) * (1 + 1e-12))
    assert hmc.accept(2.0, 1.0, 0.999999)                 # downhill always accepts


def test_free_mask_keeps_fixed_components():
    X, y, phi, th = _problem()
    free = np.array([1.0, 1.0, 1.0, 0.0])
    t1, p1 = hmc.leapfrog(X, y, phi, th, np.array([0.1, 0.2, -0.1, 0.0]), 0.1, True, free=free, n_steps=2)
    assert t1[3] == th[3] and p1[3] == 0.0


def test_log_posterior_determinant_matches_slogdet():
    X, y, _, th = _problem(n=30)
    A = sk.A_matrix(X, th, True)
    sign, logdet = np.linalg.slogdet(A)
    lp = hmc.log_posterior(X, y, th, True)
    assert lp == pytest.approx(-0.5 * logdet - 0.5 * y @ np.linalg.solve(A, y), rel=1e-12)


def test_sampler_matches_quadrature_tiny_n():
    """Algorithm 1 with leapfrog HMC on the Sec. 4.1 data (N = 10 equispaced points
    on [-1, 1), y = 1, sigma^2 = 0.1 fixed, dt = 0.4, N_int = 3) with the squared-
    exponential kernel, theta = (log alpha, log l), a proper N(0, 1) prior (the
    flat prior of the paper is improper on log parameters), against trapezoid
    quadrature of Eq. P."""
    cfg = json.load(open(GOLDEN))
    w = wl.tiny_verification(cfg["n_points"])
    X, y = w.X, w.y
    assert np.all(y == cfg["y"])
    base = w.theta[0].copy()
    assert math.exp(base[-1]) == pytest.approx(cfg["sigma2_fixed"])
    prior = {"mu": np.zeros(3), "prec": np.array([1.0, 1.0, 0.0])}
    free = np.array([1.0, 1.0, 0.0])

    # quadrature of P(theta) over (log alpha, log l)
    g = np.linspace(-5.0, 5.0, 161)
    logp = np.empty((len(g), len(g)))
    for i, a in enumerate(g):
        for j, l in enumerate(g):
            logp[i, j] = hmc.log_posterior(X, y, np.array([a, l, base[-1]]), False, prior)
    cdfs = [dg.marginal_cdf_grid(logp, g, ax) for ax in (0, 1)]

    B, updates, burn = 192, 700, 150
    rng = wl.rng_for(0)
    th = np.tile(np.array([0.01, 0.01, base[-1]]), (B, 1))   # Sec. 4 initialises theta at 0.01
    trace, acc = [], []
    for _t in range(updates):
        xi = rng.standard_normal((B, len(y)))
        pi = rng.standard_normal((B, 3))
        u = rng.uniform(size=B)
        th, ok = hmc.hmc_update_batch(X, y, th, False, cfg["leapfrog_dt"], cfg["leapfrog_n_int"],
                                      xi, pi, u, prior, free)
        trace.append(th[:, :2].copy())
        acc.append(ok.mean())
    trace = np.array(trace[burn:])                          # (L, B, 2)
    assert np.mean(acc) > 0.4
    pts = np.linspace(-3.0, 3.0, cfg["cdf_points"])
    L = trace.shape[0]
    for ax in range(2):
        tau = np.mean([dg.iat(trace[:, b, ax]) for b in range(0, B, 8)])
        n_eff = B * L / tau
        radius = math.sqrt(math.log(2 / 0.01) / (2 * n_eff))
        emp = np.array([(trace[:, :, ax] <= p).mean() for p in pts])
        ref = np.interp(pts, g, cdfs[ax])
        assert np.abs(emp - ref).max() < radius, (ax, np.abs(emp - ref).max(), radius)


def test_c1_step_005_is_beyond_the_unit_mass_leapfrog_stability_limit():
    # The N = 2048 workload (d = 1, alpha = 1, l = 0.2, sigma^2 = 0.01) with the
    # paper's M = I (Sec. 3.2) and the exact FP64 force: at dt = 0.01 the energy
    # error stays small along the trajectory, at dt = 0.05 it grows
    # geometrically step after step (the stiffest mode of U has
    # dt * omega > 2), so no update can be accepted at that step whatever the
    # precision of the products.
    w = wl.c1()
    X, y = w.X.astype(np.float64), w.y.astype(np.float64)
    th0 = np.array(w.theta[0], np.float64)
    rng = np.random.default_rng(11)
    xi, pi0 = rng.standard_normal(w.n_total), rng.standard_normal(th0.shape)
    phi = hmc.phi_exact(X, th0, xi, False)
    H0 = hmc.hamiltonian(X, y, phi, th0, pi0, False)

    def energy_errors(dt, n):
        th, pi, out = th0.copy(), pi0.copy(), []
        for _ in range(n):
            th, pi = hmc.leapfrog(X, y, phi, th, pi, dt, False)
            out.append(hmc.hamiltonian(X, y, phi, th, pi, False) - H0)
        return np.array(out)

    small = energy_errors(0.01, 4)
    assert np.abs(small).max() < 0.05, small
    big = np.abs(energy_errors(0.05, 4))
    assert big[-1] > 20.0, big
    assert np.all(big[2:] / big[1:-1] > 5.0), big

"""GPU parity of kmv_cg_solve, leapfrog_step and kmv_energy against the FP64 oracle.

The solve stops at a relative residual of cg_tol; single leapfrog steps from
identical inputs are compared with a tolerance derived from it (the force error
is bounded by ||dA|| ||x|| ||x - x*||), energies to 1e-6 relative."""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import se_kernel as sk, hmc as ohmc
from helpers import to_dev, f32

pytestmark = pytest.mark.gpu


def _phi(w, seed):
    return np.random.default_rng(seed).standard_normal((w.chains, w.n_total)).astype(np.float32)


@pytest.mark.parametrize("prec", ["fp32", "bf16_hilo"])
def test_cg_solve_residual(kmv_handle, prec):
    w = wl.ragged([300, 0, 180], d=2, chains=2, m=1, seed=51, sigma2=0.1)
    pts, theta, _, _ = to_dev(w)
    y = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    x, st, it = kmv_handle.kmv_cg_solve(pts, theta, y, tol=1e-6, maxiter=500, prec=prec)
    assert torch.all(st == 0)
    x = x.cpu().numpy()
    X, yh = f32(w.X), f32(w.y)
    for b in (0, 2):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        for c in range(2):
            s = b * 2 + c
            xs = f32(x[c, r0:r1])
            res = yh[r0:r1] - sk.kmv(X[r0:r1], w.theta[s], xs, True)
            A_norm = np.abs(sk.A_matrix(X[r0:r1], w.theta[s], True)).sum(1).max()
            floor = 20 * 2.0 ** -24 * A_norm * np.linalg.norm(xs)
            rel = np.linalg.norm(res) / np.linalg.norm(yh[r0:r1])
            # the BF16 solve is refined against the FP32 operator: same criterion
            assert rel <= 1e-6 + floor / np.linalg.norm(yh[r0:r1]), (b, c, rel)


def test_cg_reports_non_convergence_and_warm_start(kmv_handle):
    w = wl.ragged([400], d=1, chains=1, m=1, seed=52, sigma2=0.01)
    pts, theta, _, _ = to_dev(w)
    y = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    _, st, it = kmv_handle.kmv_cg_solve(pts, theta, y, tol=1e-6, maxiter=2)
    assert int(st[0]) == 4 and int(it[0]) == 2          # KMV_ENOTCONV
    x, st, it = kmv_handle.kmv_cg_solve(pts, theta, y, tol=1e-5, maxiter=2000)
    assert int(st[0]) == 0
    n_cold = int(it[0])
    _, st2, it2 = kmv_handle.kmv_cg_solve(pts, theta, y, x=x.clone(), tol=1e-5, maxiter=2000, warm_start=True)
    assert int(st2[0]) == 0 and int(it2[0]) < n_cold


def _lf_inputs(w, seed):
    rng = np.random.default_rng(seed)
    pi0 = 0.3 * rng.standard_normal(w.theta.shape)
    return _phi(w, seed), pi0


@pytest.mark.parametrize("prec", ["fp32", "bf16_hilo"])
@pytest.mark.parametrize("ard", [False, True])
def test_leapfrog_step_matches_oracle(kmv_handle, ard, prec):
    w = wl.ragged([260, 140], d=2, chains=2, m=1, ard=ard, seed=53, sigma2=0.1)
    pts, theta, _, _ = to_dev(w)
    phi, pi0 = _lf_inputs(w, 54)
    prior = (np.zeros(w.n_theta), np.full(w.n_theta, 0.5))
    y = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    th = theta.clone()
    pi = torch.tensor(pi0, dtype=torch.float64, device="cuda")
    pr = tuple(torch.tensor(a, dtype=torch.float64, device="cuda") for a in prior)
    st, it, _ = kmv_handle.leapfrog_step(pts, y, torch.tensor(phi, device="cuda"), th, pi, 0.05,
                                         prior=pr, cg_tol=1e-7, cg_maxiter=2000, prec=prec)
    assert torch.all(st == 0)
    th, pi = th.cpu().numpy(), pi.cpu().numpy()
    X, yh = f32(w.X), f32(w.y)
    for b in range(2):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        for c in range(2):
            s = b * 2 + c
            t_o, p_o = ohmc.leapfrog(X[r0:r1], yh[r0:r1], f32(phi[c, r0:r1]), w.theta[s], pi0[s], 0.05,
                                     ard, {"mu": prior[0], "prec": prior[1]})
            F_scale = np.abs(ohmc.force(X[r0:r1], yh[r0:r1], f32(phi[c, r0:r1]), w.theta[s], ard)).max()
            # force error budget: the adjoint (1e-4 relative gradients) + solve at cg_tol
            tol_F = 1e-3 * max(F_scale, 1.0)
            np.testing.assert_allclose(pi[s], p_o, atol=0.05 * tol_F, rtol=0)
            np.testing.assert_allclose(th[s], t_o, atol=0.5 * 0.05 ** 2 * tol_F + 1e-12, rtol=0)


@pytest.mark.parametrize("prec", ["fp32", "bf16_hilo"])
def test_leapfrog_free_mask_and_reversibility(kmv_handle, prec):
    w = wl.ragged([300], d=1, chains=3, m=1, ard=False, seed=55, sigma2=0.1)
    pts, theta, _, _ = to_dev(w)
    phi, pi0 = _lf_inputs(w, 56)
    pi0[:, 2] = 0.0
    y = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    ph = torch.tensor(phi, device="cuda")
    mask = torch.tensor([1, 1, 0], dtype=torch.uint8, device="cuda")
    th = theta.clone()
    pi = torch.tensor(pi0, dtype=torch.float64, device="cuda")
    for _ in range(3):
        kmv_handle.leapfrog_step(pts, y, ph, th, pi, 0.05, free_mask=mask, cg_tol=1e-7, cg_maxiter=2000,
                                 prec=prec)
    assert torch.equal(th[:, 2], theta[:, 2])
    pi.neg_()
    for _ in range(3):
        kmv_handle.leapfrog_step(pts, y, ph, th, pi, 0.05, free_mask=mask, cg_tol=1e-7, cg_maxiter=2000,
                                 prec=prec)
    pi.neg_()
    np.testing.assert_allclose(th.cpu().numpy(), w.theta, atol=2e-5)
    np.testing.assert_allclose(pi.cpu().numpy(), pi0, atol=2e-4)


def test_energy_matches_oracle(kmv_handle):
    w = wl.ragged([350, 90], d=3, chains=2, m=1, seed=57, sigma2=0.1)
    pts, theta, _, _ = to_dev(w)
    phi, pi0 = _lf_inputs(w, 58)
    y = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    prior = (np.full(w.n_theta, 0.1), np.full(w.n_theta, 2.0))
    pr = tuple(torch.tensor(a, dtype=torch.float64, device="cuda") for a in prior)
    H, terms, st, _ = kmv_handle.kmv_energy(pts, y, torch.tensor(phi, device="cuda"), theta,
                                            torch.tensor(pi0, dtype=torch.float64, device="cuda"),
                                            prior=pr, cg_tol=1e-8, cg_maxiter=3000)
    assert torch.all(st == 0)
    H, terms = H.cpu().numpy(), terms.cpu().numpy()
    X, yh = f32(w.X), f32(w.y)
    for b in range(2):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        for c in range(2):
            s = b * 2 + c
            ref = ohmc.hamiltonian(X[r0:r1], yh[r0:r1], f32(phi[c, r0:r1]), w.theta[s], pi0[s], True,
                                   {"mu": prior[0], "prec": prior[1]})
            assert abs(H[s] - ref) <= 1e-5 * abs(ref), (s, H[s], ref)
            A = sk.A_matrix(X[r0:r1], w.theta[s], True)
            pap = 0.5 * f32(phi[c, r0:r1]) @ A @ f32(phi[c, r0:r1])
            # FP32 kernel entries, FP64 accumulation: ~1e-6 relative
            assert abs(terms[s, 2] - pap) <= 1e-6 * abs(pap) + 1e-9


def test_energy_error_is_second_order_in_dt(kmv_handle):
    """H along a trajectory of fixed length conserves to O(dt^2) (Sec. 3.2.2), and the
    energy error matches the oracle's leapfrog on the same inputs."""
    w = wl.ragged([256], d=1, chains=1, m=1, ard=False, seed=59, sigma2=0.1)
    pts, theta, _, _ = to_dev(w)
    phi, _ = _lf_inputs(w, 60)
    y = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    ph = torch.tensor(phi, device="cuda")
    pi0 = torch.tensor([[0.4, -0.3, 0.2]], dtype=torch.float64, device="cuda")
    H0 = kmv_handle.kmv_energy(pts, y, ph, theta, pi0, cg_tol=1e-8, cg_maxiter=3000)[0].item()
    X, yh = f32(w.X), f32(w.y)
    H0_ref = ohmc.hamiltonian(X, yh, f32(phi[0]), w.theta[0], pi0.cpu().numpy()[0], False)
    assert abs(H0 - H0_ref) <= 1e-5 * abs(H0_ref)
    errs = []
    for k, dt in enumerate([0.02, 0.01]):
        th, pi = theta.clone(), pi0.clone()
        for _ in range(16 * 2 ** k):
            kmv_handle.leapfrog_step(pts, y, ph, th, pi, dt, cg_tol=1e-8, cg_maxiter=3000)
        H1 = kmv_handle.kmv_energy(pts, y, ph, th, pi, cg_tol=1e-8, cg_maxiter=3000)[0].item()
        t_o, p_o = ohmc.leapfrog(X, yh, f32(phi[0]), w.theta[0], pi0.cpu().numpy()[0], dt, False,
                                 n_steps=16 * 2 ** k)
        dH_ref = ohmc.hamiltonian(X, yh, f32(phi[0]), t_o, p_o, False) - H0_ref
        assert abs((H1 - H0) - dH_ref) <= 1e-2 * abs(dH_ref) + 1e-3 * abs(H0_ref) * 1e-3
        errs.append(abs(H1 - H0))
    assert 3.2 < errs[0] / errs[1] < 5.0, errs


@pytest.mark.parametrize("prec", ["fp32", "bf16_hilo"])
def test_leapfrog_force_with_cancelling_quadratic_forms(kmv_handle, prec):
    """On c1 (N = 2048, sigma^2 = 0.01) x = A^-1 y oscillates and the two
    quadratic forms of the force are sums of N^2 terms that cancel to ~1e-7 of
    their size.  Both forms must still give the oracle's step: the force is the
    adjoint of the call's precision (in the BF16 form the tensor-core adjoint,
    whose split operands keep each pair's term near FP32 accuracy; the solve is
    refined against the FP32 operator)."""
    w = wl.c1()
    pts, theta, _, _ = to_dev(w)
    X, yh = f32(w.X), f32(w.y)
    xi = np.random.default_rng(5).standard_normal(w.n_total)
    phi = f32(ohmc.phi_exact(X, w.theta[0], xi, w.ard))
    pi0 = np.array([[0.1, -0.2, 0.05]])
    dt = 0.01
    th = theta.clone()
    pi = torch.tensor(pi0, dtype=torch.float64, device="cuda")
    y = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    st, _, _ = kmv_handle.leapfrog_step(pts, y, torch.tensor(phi[None].astype(np.float32), device="cuda"), th, pi, dt,
                                        cg_tol=1e-7, cg_maxiter=5000, prec=prec)
    assert torch.all(st == 0)
    t_o, p_o = ohmc.leapfrog(X, yh, phi, w.theta[0], pi0[0], dt, w.ard)
    F_scale = np.abs(ohmc.force(X, yh, phi, w.theta[0], w.ard)).max()
    # FP32 rounding of sums that cancel this strongly leaves ~1e-3 of the force
    tol_F = 2e-3 * max(F_scale, 1.0)
    np.testing.assert_allclose(pi.cpu().numpy()[0], p_o, atol=dt * tol_F, rtol=0)
    np.testing.assert_allclose(th.cpu().numpy()[0], t_o, atol=0.5 * dt ** 2 * tol_F + 1e-12, rtol=0)

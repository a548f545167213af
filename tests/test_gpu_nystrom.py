"""GPU parity of the randomized Nystrom preconditioner (kmv_nystrom_build,
kmv_set_preconditioner) against the FP64 oracle (oracle/nystrom.py), through
the C ABI: the factorisation (eigenvalues, the reconstructed K_hat, orthonormal
columns), preconditioned CG in both forms (same solution, fewer iterations),
the leapfrog step with and without it, and the argument checks."""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import cheb_kernel as ck
from oracle import nystrom as ny
from oracle import se_kernel as sk
from helpers import to_dev, f32

pytestmark = pytest.mark.gpu


def _omega(w, rank, seed):
    return np.random.default_rng(seed).standard_normal((w.chains, w.n_total, rank)).astype(np.float32)


def _check_factor(w, U, lam, st, Om, rank, kmat):
    X = f32(w.X)
    for b in range(w.n_inst):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        for c in range(w.chains):
            s = b * w.chains + c
            if r1 - r0 < rank:
                assert st[s] == 4 and np.all(lam[s] == 0.0)   # KMV_ENOTCONV: the identity
                continue
            assert st[s] == 0
            K = kmat(X[r0:r1], s)
            U_o, lam_o = ny.nystrom(K, Om[c, r0:r1].astype(np.float64))
            # the device's Y carries the FP32 product's rounding and its shift is
            # raised to match (up to ~1e-6 of lambda_1 here); the oracle's is FP64's
            np.testing.assert_allclose(lam[s], lam_o, rtol=0, atol=5e-4 * lam_o[0])
            Us = U[c, :, r0:r1].astype(np.float64).T
            Kh = Us @ np.diag(lam[s]) @ Us.T
            Kh_o = U_o @ np.diag(lam_o) @ U_o.T
            assert np.linalg.norm(Kh - Kh_o) <= 2e-3 * np.linalg.norm(Kh_o)
            # the leading columns are orthonormal; further down the FP32 product's
            # rounding (1e-7 of the largest entries) is amplified by lam_0 / lam_k
            top = lam[s] > 1e-2 * lam[s][0]
            np.testing.assert_allclose(Us[:, top].T @ Us[:, top], np.eye(top.sum()), atol=1e-3)
            # and the preconditioner built from them is positive definite
            mu = math.exp(w.theta[s, -1])
            d = (lam[s][-1] + mu) / (lam[s] + mu) - 1.0
            Pinv = np.eye(r1 - r0) + Us @ np.diag(d) @ Us.T
            assert np.linalg.eigvalsh(0.5 * (Pinv + Pinv.T)).min() > 0.0


@pytest.mark.parametrize("prec", ["fp32", "bf16_hilo"])
def test_factorisation_matches_oracle(kmv_handle, prec):
    w = wl.ragged([400, 0, 250, 12], d=2, chains=2, m=1, ard=True, seed=81)
    pts, theta, _, _ = to_dev(w)
    rank = 24
    Om = _omega(w, rank, 82)
    U, lam, st = kmv_handle.nystrom_build(pts, theta, torch.tensor(Om, device="cuda"), prec=prec)
    if prec == "fp32":
        _check_factor(w, U.cpu().numpy(), lam.cpu().numpy(), st.cpu().numpy(), Om, rank,
                      lambda X, s: sk.kernel_matrix(X, X, w.theta[s], True))
    else:
        # the BF16 product's 2e-3 error bounds how well the factorisation can agree
        lam, st = lam.cpu().numpy(), st.cpu().numpy()
        X = f32(w.X)
        for b, (r0, r1) in enumerate(zip(w.offsets[:-1], w.offsets[1:])):
            if r1 - r0 < rank:
                continue
            for c in range(w.chains):
                s = b * w.chains + c
                K = sk.kernel_matrix(X[r0:r1], X[r0:r1], w.theta[s], True)
                _, lam_o = ny.nystrom(K, Om[c, r0:r1].astype(np.float64))
                np.testing.assert_allclose(lam[s][:4], lam_o[:4], rtol=1e-2)


def test_factorisation_of_the_chebyshev_family(kmv_handle):
    from paper_2412_20884_gb300 import Points
    w = wl.cheb([300], d=2, n_cheb=3, chains=2, m=1, seed=83)
    pts = Points(torch.tensor(w.X, dtype=torch.float32, device="cuda"), w.offsets, ard=False, cheb=3)
    theta = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
    rank = 16
    Om = _omega(w, rank, 84)
    U, lam, st = kmv_handle.nystrom_build(pts, theta, torch.tensor(Om, device="cuda"))
    _check_factor(w, U.cpu().numpy(), lam.cpu().numpy(), st.cpu().numpy(), Om, rank,
                  lambda X, s: ck.kernel_matrix(X, w.theta[s], 3, False))


@pytest.mark.parametrize("prec", ["fp32", "bf16_hilo"])
def test_preconditioned_cg(kmv_handle, prec):
    w = wl.ragged([600, 300], d=2, chains=2, m=1, ard=False, seed=85, ell_range=(0.3, 0.6), sigma2=1e-3)
    pts, theta, _, _ = to_dev(w)
    rhs = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    x0, st0, it0 = kmv_handle.kmv_cg_solve(pts, theta, rhs, tol=1e-6, maxiter=5000, prec=prec)
    U, lam, st = kmv_handle.nystrom_build(pts, theta, torch.tensor(_omega(w, 64, 86), device="cuda"))
    assert torch.all(st == 0)
    kmv_handle.set_preconditioner(pts, U, lam)
    try:
        x1, st1, it1 = kmv_handle.kmv_cg_solve(pts, theta, rhs, tol=1e-6, maxiter=5000, prec=prec)
    finally:
        kmv_handle.set_preconditioner(pts)
    assert torch.all(st0 == 0) and torch.all(st1 == 0)
    x0, x1 = x0.cpu().numpy(), x1.cpu().numpy()
    X, yh = f32(w.X), f32(w.y)
    for b in range(w.n_inst):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        for c in range(w.chains):
            s = b * w.chains + c
            A = sk.A_matrix(X[r0:r1], w.theta[s], False)
            bn = np.linalg.norm(yh[r0:r1])
            x_ref = np.linalg.solve(A, yh[r0:r1])
            # cg_tol plus the floor of an FP32 solution: rounding x alone leaves
            # a residual of up to 2^-24 |A| |x| (kappa ~ 1e5 here)
            floor = 20 * 2.0 ** -24 * np.linalg.eigvalsh(A)[-1] * np.linalg.norm(x_ref) / bn
            res1 = np.linalg.norm(yh[r0:r1] - A @ x1[c, r0:r1]) / bn
            res0 = np.linalg.norm(yh[r0:r1] - A @ x0[c, r0:r1]) / bn
            assert res1 <= 1e-5 + floor, (s, res1, res0, floor)
    it0, it1 = it0.cpu().numpy(), it1.cpu().numpy()
    assert np.all(it1 * 2 < it0), (it0, it1)


def test_leapfrog_with_and_without_preconditioner(kmv_handle):
    w = wl.ragged([300, 200], d=2, chains=2, m=1, ard=True, seed=87, sigma2=0.01)
    pts, theta, _, _ = to_dev(w)
    rng = np.random.default_rng(88)
    phi = torch.tensor(rng.standard_normal((w.chains, w.n_total)).astype(np.float32), device="cuda")
    pi0 = torch.tensor(0.3 * rng.standard_normal(w.theta.shape), dtype=torch.float64, device="cuda")
    y = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    th_a, pi_a = theta.clone(), pi0.clone()
    kmv_handle.leapfrog_step(pts, y, phi, th_a, pi_a, 0.02, cg_tol=1e-8, cg_maxiter=4000)
    U, lam, _ = kmv_handle.nystrom_build(pts, theta, torch.tensor(_omega(w, 32, 89), device="cuda"))
    kmv_handle.set_preconditioner(pts, U, lam)
    try:
        th_b, pi_b = theta.clone(), pi0.clone()
        st, it, _ = kmv_handle.leapfrog_step(pts, y, phi, th_b, pi_b, 0.02, cg_tol=1e-8, cg_maxiter=4000)
    finally:
        kmv_handle.set_preconditioner(pts)
    assert torch.all(st == 0)
    # both solves to 1e-8: the forces agree to 1e-3 of their size (the FP32 force budget)
    kick = np.abs(pi_a.cpu().numpy() - pi0.cpu().numpy()).max()
    tol_pi = 1e-3 * kick + 1e-9
    np.testing.assert_allclose(pi_b.cpu().numpy(), pi_a.cpu().numpy(), rtol=0, atol=tol_pi)
    np.testing.assert_allclose(th_b.cpu().numpy(), th_a.cpu().numpy(), rtol=0, atol=0.5 * 0.02 * tol_pi + 1e-12)


@pytest.mark.parametrize("prec", ["fp32", "bf16_hilo"])
def test_preconditioned_phi_refresh(kmv_handle, prec):
    from oracle import poles
    w = wl.ragged([500, 260], d=2, chains=2, m=1, ard=True, seed=93, ell_range=(0.3, 0.8), sigma2=0.01)
    pts, theta, _, _ = to_dev(w)
    xi = np.random.default_rng(94).standard_normal((w.chains, w.n_total)).astype(np.float32)
    xd = torch.tensor(xi, device="cuda")
    phi0, st0, it0 = kmv_handle.phi_refresh(pts, theta, xd, n_poles=15, cg_tol=1e-6, cg_maxiter=3000, prec=prec)
    # the preconditioned draw runs on FP32 products in both forms: its accuracy
    # is compared with the unpreconditioned draw on FP32 products
    phi32, _, _ = kmv_handle.phi_refresh(pts, theta, xd, n_poles=15, cg_tol=1e-6, cg_maxiter=3000, prec="fp32")
    phi32 = phi32.cpu().numpy()
    U, lam, _ = kmv_handle.nystrom_build(pts, theta, torch.tensor(_omega(w, 48, 95), device="cuda"))
    kmv_handle.set_preconditioner(pts, U, lam)
    try:
        phi, st, it, pl = kmv_handle.phi_refresh(pts, theta, xd, n_poles=15, cg_tol=1e-6, cg_maxiter=3000,
                                                 want_poles=True, prec=prec)
    finally:
        kmv_handle.set_preconditioner(pts)
    assert torch.all(st0 == 0) and torch.all(st == 0)
    phi, pl = phi.cpu().numpy(), pl.cpu().numpy()
    X = f32(w.X)
    for b in range(w.n_inst):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        for c in range(w.chains):
            s = b * w.chains + c
            A = sk.A_matrix(X[r0:r1], w.theta[s], True)
            ref = poles.inv_sqrt_apply(A, xi[c, r0:r1].astype(np.float64), pl[s, 0], pl[s, 1], 15)
            xn = np.linalg.norm(xi[c, r0:r1])
            bound = 20 * 1e-6 * xn / math.sqrt(pl[s, 0]) + 1e-5 * np.linalg.norm(ref)
            # sigma^2 = 0.01 puts the FP32 floor of the shifted solves near this bound:
            # the preconditioned draw is held to it or to twice the FP32 multi-shift draw's error
            err0 = np.linalg.norm(phi32[c, r0:r1] - ref)
            assert np.linalg.norm(phi[c, r0:r1] - ref) <= max(bound, 2.0 * err0), (s, bound, err0)
    # fewer iterations than the unpreconditioned multi-shift solve
    assert it.cpu().numpy().max() < it0.cpu().numpy().max(), (it, it0)


def test_preconditioner_arguments(kmv_handle):
    from paper_2412_20884_gb300 import KmvError
    w = wl.ragged([200], d=2, chains=1, m=1, seed=90)
    pts, theta, _, _ = to_dev(w)
    with pytest.raises(KmvError):   # rank above 128
        kmv_handle.nystrom_build(pts, theta, torch.zeros((1, 200, 129), dtype=torch.float32, device="cuda"))
    U, lam, _ = kmv_handle.nystrom_build(pts, theta, torch.tensor(_omega(w, 8, 91), device="cuda"))
    w2 = wl.ragged([150], d=2, chains=1, m=1, seed=92)
    pts2, theta2, _, _ = to_dev(w2)
    kmv_handle.set_preconditioner(pts, U, lam)
    try:
        with pytest.raises(KmvError):   # built for another layout
            kmv_handle.kmv_cg_solve(pts2, theta2, torch.ones(150, dtype=torch.float32, device="cuda"))
    finally:
        kmv_handle.set_preconditioner(pts)

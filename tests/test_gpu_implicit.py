"""GPU parity of kmv_implicit_step (the implicit midpoint step of Sec. 3.2.3
solved by Anderson acceleration, App. B) against the FP64 oracle
(oracle/implicit.py), through the C ABI.  The fixed point does not depend on
the preconditioner R or on the iteration path, so the oracle solves to 1e-12
with its own R and the device result is held to the FP32 force budget of the
leapfrog test.  The stopping test measures the true residual y - A x, whose
FP32 floor (~2^-24 |A| |x|) lies near 1e-6 here, so the device runs to 1e-5."""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import hmc as ohmc
from oracle import implicit as oim
from oracle import se_kernel as sk
from helpers import to_dev, f32

pytestmark = pytest.mark.gpu


def _inputs(w, seed):
    rng = np.random.default_rng(seed)
    phi = rng.standard_normal((w.chains, w.n_total)).astype(np.float32)
    pi0 = 0.5 * rng.standard_normal(w.theta.shape)
    return phi, pi0


def _run(h, w, phi, pi0, dt, prec="fp32", prior=None, free=None, precond_rank=0, tol=1e-5):
    pts, theta, _, _ = to_dev(w)
    y = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    th = theta.clone()
    pi = torch.tensor(pi0, dtype=torch.float64, device="cuda")
    pr = None if prior is None else tuple(torch.tensor(a, dtype=torch.float64, device="cuda") for a in prior)
    fm = None if free is None else torch.tensor(free, dtype=torch.uint8, device="cuda")
    if precond_rank:
        om = torch.tensor(np.random.default_rng(7).standard_normal((w.chains, w.n_total, precond_rank)),
                          dtype=torch.float32, device="cuda")
        U, lam, _ = h.nystrom_build(pts, theta, om)
        h.set_preconditioner(pts, U, lam)
    try:
        st, it, x = h.implicit_step(pts, y, torch.tensor(phi, device="cuda"), th, pi, dt, prior=pr, free_mask=fm,
                                    tol=tol, maxiter=1500, prec=prec)
    finally:
        if precond_rank:
            h.set_preconditioner(pts)
    return st.cpu().numpy(), it.cpu().numpy(), th.cpu().numpy(), pi.cpu().numpy(), x


@pytest.mark.parametrize("prec,rank", [("fp32", 0), ("fp32", 24), ("bf16_hilo", 0)])
def test_implicit_step_solves_the_implicit_equations(kmv_handle, prec, rank):
    """The device's (theta_1, pi_1, x) satisfy Eq. implicitsystem to the stopping
    tolerance, checked with dense FP64 products and the oracle's frozen-x force;
    and lie near the oracle's fixed point (solved to 1e-12), within what the
    tolerance allows at this conditioning."""
    w = wl.ragged([260, 140], d=2, chains=2, m=1, ard=True, seed=101, sigma2=0.1)
    phi, pi0 = _inputs(w, 102)
    prior = (np.zeros(w.n_theta), np.full(w.n_theta, 0.5))
    dt, tol = 0.05, 1e-5
    st, it, th, pi, x = _run(kmv_handle, w, phi, pi0, dt, prec=prec, prior=prior, precond_rank=rank, tol=tol)
    assert np.all(st == 0), (st, it)
    x = x.cpu().numpy()
    X, yh = f32(w.X), f32(w.y)
    pr = {"mu": prior[0], "prec": prior[1]}
    for b in range(w.n_inst):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        for c in range(w.chains):
            s = b * w.chains + c
            tb = 0.5 * (w.theta[s] + th[s])
            xs = x[c, r0:r1].astype(np.float64)
            A = sk.A_matrix(X[r0:r1], tb, True)
            assert np.linalg.norm(A @ xs - yh[r0:r1]) <= 5 * tol * np.linalg.norm(yh[r0:r1])
            scale = 1.0 + max(np.abs(th[s]).max(), np.abs(pi[s]).max())
            np.testing.assert_allclose(th[s], w.theta[s] + 0.5 * dt * (pi0[s] + pi[s]), rtol=0,
                                       atol=2 * dt * tol * scale)
            F = oim.force_frozen(X[r0:r1], f32(phi[c, r0:r1]), tb, xs, True, pr)
            np.testing.assert_allclose(pi[s], pi0[s] - dt * F, rtol=0, atol=dt * 1e-3 * max(np.abs(F).max(), 1.0))
            # the exact fixed point: x is within kappa * tol of it, which bounds the force's error
            A0 = sk.A_matrix(X[r0:r1], w.theta[s], True)
            R = np.eye(r1 - r0) / (1.05 * np.linalg.eigvalsh(A0)[-1])
            t_o, p_o, _, _ = oim.implicit_midpoint(X[r0:r1], yh[r0:r1], f32(phi[c, r0:r1]), w.theta[s], pi0[s], dt,
                                                  True, R, k=10, tol=1e-12, maxiter=3000, prior=pr)
            ev = np.linalg.eigvalsh(A)
            loose = dt * (1e-3 + 10 * tol * ev[-1] / ev[0]) * max(np.abs(F).max(), 1.0)
            np.testing.assert_allclose(pi[s], p_o, atol=loose, rtol=0)


def test_implicit_step_is_reversible_and_keeps_fixed_components(kmv_handle):
    w = wl.ragged([300], d=1, chains=3, m=1, ard=False, seed=103, sigma2=0.1)
    phi, pi0 = _inputs(w, 104)
    free = np.array([1, 1, 0], np.uint8)
    pi0[:, 2] = 0.0
    pts, theta, _, _ = to_dev(w)
    y = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    ph = torch.tensor(phi, device="cuda")
    fm = torch.tensor(free, device="cuda")
    th = theta.clone()
    pi = torch.tensor(pi0, dtype=torch.float64, device="cuda")
    st, _, x = kmv_handle.implicit_step(pts, y, ph, th, pi, 0.05, free_mask=fm, tol=1e-5, maxiter=1500)
    assert torch.all(st == 0)
    assert torch.equal(th[:, 2], theta[:, 2])
    pi.neg_()
    st, _, _ = kmv_handle.implicit_step(pts, y, ph, th, pi, 0.05, free_mask=fm, tol=1e-5, maxiter=1500, x_work=x)
    assert torch.all(st == 0)
    pi.neg_()
    np.testing.assert_allclose(th.cpu().numpy(), w.theta, atol=2e-5)
    np.testing.assert_allclose(pi.cpu().numpy(), pi0, atol=2e-4)


def test_implicit_step_reports_non_convergence(kmv_handle):
    from paper_2412_20884_gb300 import KmvError
    w = wl.ragged([200], d=2, chains=1, m=1, seed=105, sigma2=0.1)
    phi, pi0 = _inputs(w, 106)
    pts, theta, _, _ = to_dev(w)
    y = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    pi = torch.tensor(pi0, dtype=torch.float64, device="cuda")
    st, it, _ = kmv_handle.implicit_step(pts, y, torch.tensor(phi, device="cuda"), theta.clone(), pi, 0.05,
                                         tol=1e-9, maxiter=2)
    assert st.item() == 4 and it.item() == 2    # KMV_ENOTCONV after maxiter iterations
    with pytest.raises(KmvError):
        kmv_handle.implicit_step(pts, y, torch.tensor(phi, device="cuda"), theta.clone(), pi, 0.05, aa_depth=17)

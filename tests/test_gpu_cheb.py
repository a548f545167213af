"""GPU parity of the Chebyshev log-amplitude kernel family of Sec. 4 against the
FP64 oracle (oracle/cheb_kernel.py), through the C ABI: forward, adjoint (Theta,
lengthscale and noise gradients, dL/dV), CG solve, leapfrog step and phi draw.

Tolerances as for the SE kernel: fp32 outputs 1e-5 componentwise (scale
sum_j |A_ij| |V_j|), gradients 1e-4; bf16_hilo 2e-3 and 2e-2.
"""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import cheb_kernel as ck
from oracle import hmc as ohmc
from oracle import poles
from helpers import f32, componentwise_err, grad_err

pytestmark = pytest.mark.gpu

TOL = {"fp32": (1e-5, 1e-4), "bf16_hilo": (2e-3, 2e-2)}
PRECS = ["fp32", "bf16_hilo"]

CASES = [
    # sizes, d, n_cheb, chains, m, ard
    ([300, 0, 170], 2, 3, 2, 3, False),
    ([257], 3, 2, 1, 1, True),          # one column: the few-column product forms
    ([200, 90], 1, 6, 2, 16, False),
    ([140], 2, 1, 1, 2, True),          # order one: a constant amplitude
]


def _dev(w):
    from paper_2412_20884_gb300 import Points
    pts = Points(torch.tensor(w.X, dtype=torch.float32, device="cuda"), w.offsets, ard=w.ard, cheb=w.meta["cheb"])
    theta = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
    V = torch.tensor(w.V, dtype=torch.float32, device="cuda")
    G = torch.tensor(w.G, dtype=torch.float32, device="cuda")
    return pts, theta, V, G


def _A(w, X, s):
    return ck.A_matrix(X, w.theta[s], w.meta["cheb"], w.ard)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{sum(c[0])}d{c[1]}n{c[2]}c{c[3]}m{c[4]}")
def test_forward_and_backward_parity(kmv_handle, prec, case):
    sizes, d, nc, chains, m, ard = case
    w = wl.cheb(sizes, d=d, n_cheb=nc, chains=chains, m=m, ard=ard, seed=sum(sizes) + nc)
    pts, theta, V, G = _dev(w)
    assert pts.n_theta == w.n_theta
    Y = kmv_handle.kmv_forward(pts, theta, V, prec=prec).cpu().numpy()
    gth, gV = kmv_handle.kmv_backward(pts, theta, V, G, prec=prec)
    gth, gV = gth.cpu().numpy(), gV.cpu().numpy()
    X, Vh, Gh = f32(w.X), f32(w.V), f32(w.G)
    ef = eb = eg = 0.0
    for b in range(w.n_inst):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        for c in range(chains):
            s = b * chains + c
            if r1 == r0:
                assert np.all(gth[s] == 0.0)
                continue
            A = _A(w, X[r0:r1], s)
            absA = np.abs(A)
            ef = max(ef, componentwise_err(Y[c, r0:r1], A @ Vh[c, r0:r1], absA @ np.abs(Vh[c, r0:r1])))
            g_ref, gV_ref = ck.kmv_adjoint(X[r0:r1], w.theta[s], Vh[c, r0:r1], Gh[c, r0:r1], nc, ard)
            eg = max(eg, grad_err(gth[s], g_ref))
            eb = max(eb, componentwise_err(gV[c, r0:r1], gV_ref, absA @ np.abs(Gh[c, r0:r1])))
    assert ef <= TOL[prec][0], ef
    assert eb <= TOL[prec][0], eb
    assert eg <= TOL[prec][1], eg


@pytest.mark.parametrize("prec", PRECS)
def test_cg_solve(kmv_handle, prec):
    w = wl.cheb([400, 150], d=2, n_cheb=3, chains=2, m=1, seed=61, sigma2=0.1)
    pts, theta, _, _ = _dev(w)
    rhs = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    x, st, it = kmv_handle.kmv_cg_solve(pts, theta, rhs, tol=1e-7, maxiter=3000, prec=prec)
    assert torch.all(st == 0)
    x = x.cpu().numpy()
    X, yh = f32(w.X), f32(w.y)
    for b in range(w.n_inst):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        for c in range(w.chains):
            s = b * w.chains + c
            A = _A(w, X[r0:r1], s)
            res = np.linalg.norm(yh[r0:r1] - A @ x[c, r0:r1]) / np.linalg.norm(yh[r0:r1])
            assert res <= 1e-5, (s, res)


def test_leapfrog_step_matches_oracle(kmv_handle):
    w = wl.cheb([260, 140], d=2, n_cheb=2, chains=2, m=1, seed=63, sigma2=0.1)
    pts, theta, _, _ = _dev(w)
    rng = np.random.default_rng(64)
    phi = rng.standard_normal((w.chains, w.n_total)).astype(np.float32)
    pi0 = 0.3 * rng.standard_normal(w.theta.shape)
    y = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    th = theta.clone()
    pi = torch.tensor(pi0, dtype=torch.float64, device="cuda")
    st, it, _ = kmv_handle.leapfrog_step(pts, y, torch.tensor(phi, device="cuda"), th, pi, 0.05, cg_tol=1e-7,
                                         cg_maxiter=3000)
    assert torch.all(st == 0)
    th, pi = th.cpu().numpy(), pi.cpu().numpy()
    X, yh = f32(w.X), f32(w.y)
    nc = w.meta["cheb"]
    kern = (lambda X_, t: ck.A_matrix(X_, t, nc, False), lambda X_, t: ck.dA_dtheta(X_, t, nc, False))
    for b in range(w.n_inst):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        for c in range(w.chains):
            s = b * w.chains + c
            t_o, p_o = ohmc.leapfrog(X[r0:r1], yh[r0:r1], f32(phi[c, r0:r1]), w.theta[s], pi0[s], 0.05, False,
                                     kern=kern)
            F_scale = np.abs(ohmc.force(X[r0:r1], yh[r0:r1], f32(phi[c, r0:r1]), w.theta[s], False,
                                        kern=kern)).max()
            tol_F = 1e-3 * max(F_scale, 1.0)
            np.testing.assert_allclose(pi[s], p_o, atol=0.05 * tol_F, rtol=0)
            np.testing.assert_allclose(th[s], t_o, atol=0.5 * 0.05 ** 2 * tol_F + 1e-12, rtol=0)


@pytest.mark.parametrize("prec", PRECS)
def test_phi_refresh(kmv_handle, prec):
    w = wl.cheb([300, 120], d=2, n_cheb=3, chains=2, m=1, seed=65, sigma2=0.1)
    pts, theta, _, _ = _dev(w)
    xi = np.random.default_rng(66).standard_normal((w.chains, w.n_total)).astype(np.float32)
    phi, st, it, pl = kmv_handle.phi_refresh(pts, theta, torch.tensor(xi, device="cuda"), n_poles=15, cg_tol=1e-6,
                                             cg_maxiter=3000, want_poles=True, prec=prec)
    assert torch.all(st == 0)
    phi, pl = phi.cpu().numpy(), pl.cpu().numpy()
    X = f32(w.X)
    for b in range(w.n_inst):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        for c in range(w.chains):
            s = b * w.chains + c
            A = _A(w, X[r0:r1], s)
            # the device's interval: sigma^2 and 1.01 x the largest row sum of A
            assert pl[s, 0] == pytest.approx(math.exp(w.theta[s, -1]), rel=1e-12)
            M = A.sum(axis=1).max()
            assert M * 1.005 <= pl[s, 1] <= M * 1.015
            ref = poles.inv_sqrt_apply(A, xi[c, r0:r1].astype(np.float64), pl[s, 0], pl[s, 1], 15)
            xn = np.linalg.norm(xi[c, r0:r1])
            bound = 20 * 1e-6 * xn / math.sqrt(pl[s, 0]) + 1e-5 * np.linalg.norm(ref)
            assert np.linalg.norm(phi[c, r0:r1] - ref) <= bound


def test_invalid_family_arguments(kmv_handle):
    from paper_2412_20884_gb300 import KmvError, Points
    from paper_2412_20884_gb300 import binding
    x = torch.zeros((64, 3), dtype=torch.float32, device="cuda")
    V = torch.zeros((1, 64, 1), dtype=torch.float32, device="cuda")
    for cheb in (33, 11):        # order above 32; 11^3 > 1024 coefficients
        pts = Points(x, None, ard=False, cheb=cheb)
        theta = torch.zeros((1, pts.n_theta), dtype=torch.float64, device="cuda")
        with pytest.raises(KmvError):
            kmv_handle.kmv_forward(pts, theta, V)
    pts = Points(x, None, ard=False, cheb=2)
    theta = torch.zeros((1, pts.n_theta), dtype=torch.float64, device="cuda")
    with pytest.raises(KmvError) as e:
        binding.kmv_backward_noalloc(pts, theta, V, V)
    assert e.value.status == 7   # KMV_EUNSUPPORTED

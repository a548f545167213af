"""GPU parity of kmv_phi_refresh (the Gibbs draw of Sec. 3.1 by the pole
expansion of App. A) against the FP64 oracle, through the C ABI.

The device reports its spectral interval and pole table; the weights and
shifts must equal the oracle's (scipy elliptic functions) on that interval,
and phi must equal the exact A^{-1/2} xi (eigendecomposition) within the
expansion's error on the interval plus the CG tolerance's effect.
"""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import hmc, poles, se_kernel as sk
from helpers import to_dev, f32

pytestmark = pytest.mark.gpu

PRECS = ["fp32", "bf16_hilo"]


def _draw(h, w, prec, n_poles=15, tol=1e-6):
    pts, theta, _, _ = to_dev(w)
    xi_h = np.random.default_rng(11).standard_normal((w.chains, w.n_total)).astype(np.float32)
    xi = torch.tensor(xi_h, device="cuda")
    phi, st, it, pl = h.phi_refresh(pts, theta, xi, n_poles=n_poles, cg_tol=tol, cg_maxiter=2000,
                                    want_poles=True, prec=prec)
    return xi_h, phi.cpu().numpy(), st.cpu().numpy(), it.cpu().numpy(), pl.cpu().numpy()


@pytest.mark.parametrize("prec", PRECS)
def test_pole_table_matches_oracle(kmv_handle, prec):
    w = wl.ragged([200, 77], d=2, chains=2, m=1, ard=True, seed=51)
    _, _, st, _, pl = _draw(kmv_handle, w, prec, n_poles=15)
    assert np.all(st == 0)
    X = f32(w.X)
    for b in range(w.n_inst):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        for c in range(w.chains):
            s = b * w.chains + c
            m_ref, M_ref = poles.spectral_interval(X[r0:r1], w.theta[s], True)
            m_dev, M_dev = pl[s, 0], pl[s, 1]
            assert m_dev == pytest.approx(m_ref, rel=1e-15)
            # 1% slack over the largest row sum (rounding of the product)
            assert M_ref * 1.005 <= M_dev <= M_ref * 1.015
            wts, sh = poles.pole_weights_shifts(m_dev, M_dev, 15)
            np.testing.assert_allclose(pl[s, 2:17], wts, rtol=1e-10)
            np.testing.assert_allclose(pl[s, 17:32], sh, rtol=1e-10, atol=1e-300)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n_poles", [8, 15])
def test_phi_matches_inverse_square_root(kmv_handle, prec, n_poles):
    w = wl.ragged([200, 0, 77], d=2, chains=2, m=1, ard=True, seed=53)
    tol = 1e-6
    xi, phi, st, it, pl = _draw(kmv_handle, w, prec, n_poles=n_poles, tol=tol)
    assert np.all(st == 0)
    X = f32(w.X)
    for b in range(w.n_inst):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        if r1 == r0:
            continue
        for c in range(w.chains):
            s = b * w.chains + c
            exact = hmc.phi_exact(X[r0:r1], w.theta[s], xi[c, r0:r1].astype(np.float64), True)
            m_dev, M_dev = pl[s, 0], pl[s, 1]
            wts, sh = poles.pole_weights_shifts(m_dev, M_dev, n_poles)
            lam = np.geomspace(m_dev, M_dev, 4001)
            expansion = np.abs(poles.inv_sqrt_scalar(lam, wts, sh) - lam ** -0.5).max()
            xn = np.linalg.norm(xi[c, r0:r1])
            # residual tol of each shifted solve, amplified at most by 1 / sqrt(sigma^2)
            bound = 1.01 * expansion * xn + 20 * tol * xn / math.sqrt(m_dev)
            assert np.linalg.norm(phi[c, r0:r1] - exact) <= bound, (s, np.linalg.norm(phi[c, r0:r1] - exact), bound)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n_poles", [1, 2, 15])
def test_phi_several_tiles_matches_pole_oracle(kmv_handle, prec, n_poles):
    """Several row tiles with ragged tails, an empty instance and three chains:
    phi against the oracle's expansion on the device's interval (dense FP64
    solves of the n_poles shifted systems), within the CG tolerance's effect
    and FP32 rounding.  n_poles 1 and 2 take the few-column product forms."""
    w = wl.ragged([700, 0, 333], d=4, chains=3, m=1, ard=True, seed=57)
    tol = 1e-6
    xi, phi, st, it, pl = _draw(kmv_handle, w, prec, n_poles=n_poles, tol=tol)
    assert np.all(st == 0)
    X = f32(w.X)
    for b in range(w.n_inst):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        for c in range(w.chains):
            s = b * w.chains + c
            if r1 == r0:
                assert it[s] == 0
                continue
            assert it[s] > 0
            A = sk.A_matrix(X[r0:r1], w.theta[s], True)
            ref = poles.inv_sqrt_apply(A, xi[c, r0:r1].astype(np.float64), pl[s, 0], pl[s, 1], n_poles)
            xn = np.linalg.norm(xi[c, r0:r1])
            bound = 20 * tol * xn / math.sqrt(pl[s, 0]) + 1e-5 * np.linalg.norm(ref)
            err = np.linalg.norm(phi[c, r0:r1] - ref)
            assert err <= bound, (s, err, bound)


def test_phi_invalid_arguments(kmv_handle):
    from paper_2412_20884_gb300 import KmvError
    w = wl.ragged([64], d=2, chains=1, m=1, ard=True, seed=55)
    pts, theta, _, _ = to_dev(w)
    xi = torch.zeros((1, 64), dtype=torch.float32, device="cuda")
    for bad in (0, 33):
        with pytest.raises(KmvError):
            kmv_handle.phi_refresh(pts, theta, xi, n_poles=bad)

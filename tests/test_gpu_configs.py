"""GPU parity at the full sizes of the precision and batching workloads, through
the C ABI, against the FP64 oracle on sampled rows.

* precision workload: N = 262,144, d = 32, x ~ U[-1, 1]^32, ARD, m = 64 -
  the forward on 1024 sampled rows, and the whole adjoint with G restricted to
  those rows (then dL/dtheta and dL/dV = A G are exact sums the oracle forms
  in O(|rows| N d)).  This runs the adjoint's column-block launches.
* batching workload: 256 instances, N_b log-uniform in [1e3, 2e4], d = 4,
  4 chains - the whole batch on the GPU, 8 random instances (all their
  chains) checked on 128 sampled rows each: the m = 1 product of the CG
  iterations and the m = 2 adjoint of the force; every other system has G = 0
  and must get an exactly zero gradient.

Tolerances as in test_gpu_kmv: outputs 1e-5 (FP32) / 2e-3 (BF16 hi/lo)
componentwise, gradients 1e-4 relative in both forms."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import se_kernel as sk
from helpers import to_dev, f32, componentwise_err, grad_err

pytestmark = pytest.mark.gpu

TOL = {"fp32": (1e-5, 1e-4), "bf16_hilo": (2e-3, 1e-4)}
PRECS = ["fp32", "bf16_hilo"]


@pytest.fixture(scope="module")
def c3_case():
    """The workload, its sampled-row seed and the oracle's answers (computed once)."""
    w = wl.c3()
    X, Vh = f32(w.X), f32(w.V[0])
    rows = w.rows
    Gs = np.zeros_like(w.G)
    Gs[0, rows] = w.G[0, rows]
    th = w.theta[0]
    Y_ref = sk.kmv(X, th, Vh, True, rows=rows, block=128)
    Y_scale = sk.kmv(X, th, np.abs(Vh), True, rows=rows, block=128)
    g_ref, gV_ref = sk.kmv_adjoint(X, th, Vh, f32(Gs[0]), True, rows=rows, block=128)
    probe = np.sort(np.random.default_rng(1).choice(w.n_total, 512, replace=False))
    gV_scale = np.abs(sk.kernel_matrix(X[probe], X[rows], th, True)) @ np.abs(f32(Gs[0, rows]))
    inr = np.isin(probe, rows)
    gV_scale[inr] += np.exp(th[-1]) * np.abs(f32(Gs[0]))[probe[inr]]
    return dict(w=w, Gs=Gs, Y_ref=Y_ref, Y_scale=Y_scale, g_ref=g_ref, gV_ref=gV_ref[probe], probe=probe,
                gV_scale=np.maximum(gV_scale, 1e-30))


@pytest.mark.parametrize("prec", PRECS)
def test_c3_full_size_sampled_rows(kmv_handle, c3_case, prec):
    w = c3_case["w"]
    pts, theta, V, _ = to_dev(w)
    Y = kmv_handle.kmv_forward(pts, theta, V, prec=prec).cpu().numpy()[0]
    ey = componentwise_err(Y[w.rows], c3_case["Y_ref"], c3_case["Y_scale"])
    Gd = torch.tensor(c3_case["Gs"], dtype=torch.float32, device="cuda")
    gth, gV = kmv_handle.kmv_backward(pts, theta, V, Gd, prec=prec)
    eg = grad_err(gth.cpu().numpy()[0], c3_case["g_ref"])
    ev = componentwise_err(gV.cpu().numpy()[0][c3_case["probe"]], c3_case["gV_ref"], c3_case["gV_scale"])
    print(f"c3 {prec}: forward {ey:.2e}, gradient {eg:.2e}, dL/dV {ev:.2e}")
    assert ey <= TOL[prec][0], ey
    assert eg <= TOL[prec][1], eg
    assert ev <= TOL[prec][0], ev


@pytest.fixture(scope="module")
def c4_case():
    w = wl.c4(m=2)
    rng = np.random.default_rng(7)
    chosen = np.sort(rng.choice(w.n_inst, 8, replace=False))
    rows = {}
    Gs = np.zeros_like(w.G)
    for b in chosen:
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        rows[b] = np.sort(rng.choice(r1 - r0, 128, replace=False))
        Gs[:, r0 + rows[b]] = w.G[:, r0 + rows[b]]
    return dict(w=w, chosen=chosen, rows=rows, Gs=Gs)


@pytest.mark.parametrize("prec", PRECS)
def test_c4_instances_sampled_rows(kmv_handle, c4_case, prec):
    w, chosen, rows, Gs = c4_case["w"], c4_case["chosen"], c4_case["rows"], c4_case["Gs"]
    pts, theta, V, _ = to_dev(w)
    V1 = V[:, :, :1].contiguous()
    Y = kmv_handle.kmv_forward(pts, theta, V1, prec=prec).cpu().numpy()
    Gd = torch.tensor(Gs, dtype=torch.float32, device="cuda")
    gth, gV = kmv_handle.kmv_backward(pts, theta, V, Gd, prec=prec)
    gth, gV = gth.cpu().numpy(), gV.cpu().numpy()
    X = f32(w.X)
    worst = [0.0, 0.0, 0.0]
    for b in chosen:
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        Xb, rb = X[r0:r1], rows[b]
        for c in range(w.chains):
            s = b * w.chains + c
            Vb = f32(w.V[c, r0:r1])
            ref = sk.kmv(Xb, w.theta[s], Vb[:, :1], True, rows=rb)
            scale = sk.kmv(Xb, w.theta[s], np.abs(Vb[:, :1]), True, rows=rb)
            worst[0] = max(worst[0], componentwise_err(Y[c, r0 + rb], ref, scale))
            Gb = f32(Gs[c, r0:r1])
            g_ref, gV_ref = sk.kmv_adjoint(Xb, w.theta[s], Vb, Gb, True, rows=rb)
            worst[1] = max(worst[1], grad_err(gth[s], g_ref))
            sc = sk.kmv(Xb, w.theta[s], np.abs(Gb), True, rows=rb)
            worst[2] = max(worst[2], componentwise_err(gV[c, r0 + rb], gV_ref[rb], np.maximum(sc, 1e-30)))
    others = np.setdiff1d(np.arange(w.n_inst), chosen)
    zero_rows = (others[:, None] * w.chains + np.arange(w.chains)[None, :]).ravel()
    print(f"c4 {prec}: forward {worst[0]:.2e}, gradient {worst[1]:.2e}, dL/dV {worst[2]:.2e}")
    assert np.all(gth[zero_rows] == 0.0)
    assert worst[0] <= TOL[prec][0], worst
    assert worst[1] <= TOL[prec][1], worst
    assert worst[2] <= TOL[prec][0], worst

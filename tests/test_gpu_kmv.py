"""GPU parity of kmv_forward / kmv_backward against the FP64 oracle, through the C ABI.

Tolerances (the stated targets of the method's GPU form):
  fp32       outputs 1e-5 componentwise, gradients 1e-4
  bf16_hilo  outputs 2e-3 componentwise, gradients 1e-4
Componentwise error of Y is |Y - Y*| / (sum_j |A_ij| |V_j|); gradient error is
|g - g*| / max(|g*|, 1e-3 ||g*||_inf).  The oracle sees the FP32-rounded inputs.
"""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import se_kernel as sk
from helpers import to_dev, f32, abs_row_products, componentwise_err, grad_err

pytestmark = pytest.mark.gpu

TOL = {"fp32": (1e-5, 1e-4), "bf16_hilo": (2e-3, 1e-4)}
PRECS = ["fp32", "bf16_hilo"]


def _check_forward(h, w, prec, col_shift=None, want64=False):
    pts, theta, V, _ = to_dev(w)
    cs = None if col_shift is None else torch.tensor(col_shift, dtype=torch.float32, device="cuda")
    out = h.kmv_forward(pts, theta, V, col_shift=cs, Y64=want64, prec=prec)
    Y, Y64 = (out if want64 else (out, None))
    Y = Y.cpu().numpy()
    X, Vh = f32(w.X), f32(w.V)
    cs64 = None if col_shift is None else f32(col_shift)
    worst = 0.0
    for b in range(w.n_inst):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        if r1 == r0:
            continue
        for c in range(w.chains):
            s = b * w.chains + c
            ref = sk.kmv(X[r0:r1], w.theta[s], Vh[c, r0:r1], w.ard, col_shift=cs64)
            scale = abs_row_products(X[r0:r1], w.theta[s], Vh[c, r0:r1], w.ard, None)
            if cs64 is not None:
                scale = scale + np.abs(cs64)[None, :] * np.abs(Vh[c, r0:r1])
            worst = max(worst, componentwise_err(Y[c, r0:r1], ref, scale))
            if want64:
                e64 = componentwise_err(Y64[c, r0:r1].cpu().numpy(), ref, scale)
                assert e64 <= TOL[prec][0]
    assert worst <= TOL[prec][0], worst
    return worst


def _check_backward(h, w, prec):
    pts, theta, V, G = to_dev(w)
    gth, gV = h.kmv_backward(pts, theta, V, G, prec=prec)
    gth, gV = gth.cpu().numpy(), gV.cpu().numpy()
    X, Vh, Gh = f32(w.X), f32(w.V), f32(w.G)
    we, wg = 0.0, 0.0
    for b in range(w.n_inst):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        for c in range(w.chains):
            s = b * w.chains + c
            if r1 == r0:
                assert np.all(gth[s] == 0.0)
                continue
            g_ref, gV_ref = sk.kmv_adjoint(X[r0:r1], w.theta[s], Vh[c, r0:r1], Gh[c, r0:r1], w.ard)
            wg = max(wg, grad_err(gth[s], g_ref))
            scale = abs_row_products(X[r0:r1], w.theta[s], Gh[c, r0:r1], w.ard, None)
            we = max(we, componentwise_err(gV[c, r0:r1], gV_ref, scale))
    assert we <= TOL[prec][0], we
    assert wg <= TOL[prec][1], wg
    return we, wg


# Block widths of the tensor-core adjoint's fold: one group of 8 dimensions or
# several, the wide and the K-split accumulator layouts, XA in tensor or in
# shared memory, one or two dimension blocks (d = 17..31).
FOLD_DIMS = [6, 7, 9, 10, 11, 12, 15, 16, 17, 20, 24, 31]


@pytest.mark.parametrize("d", FOLD_DIMS)
def test_backward_parity_across_fold_widths(kmv_handle, d):
    w = wl.ragged([230, 161], d=d, chains=1, m=5, ard=True, seed=900 + d)
    _check_backward(kmv_handle, w, "bf16_hilo")


CASES = [
    # sizes, d, chains, m, ard
    ([300], 1, 1, 1, False),
    ([257, 0, 129, 1], 3, 2, 2, True),
    ([640], 8, 1, 16, True),
    ([333], 5, 1, 3, True),           # d outside the specialised set
    ([200, 150], 4, 3, 1, True),
    ([190], 32, 1, 17, True),
    ([130], 2, 1, 70, False),         # more columns than one pass holds
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{sum(c[0])}d{c[1]}c{c[2]}m{c[3]}{'ard' if c[4] else 'iso'}")
def test_forward_parity(kmv_handle, prec, case):
    sizes, d, chains, m, ard = case
    w = wl.ragged(sizes, d=d, chains=chains, m=m, ard=ard, seed=sum(sizes) + d)
    _check_forward(kmv_handle, w, prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{sum(c[0])}d{c[1]}c{c[2]}m{c[3]}{'ard' if c[4] else 'iso'}")
def test_backward_parity(kmv_handle, prec, case):
    sizes, d, chains, m, ard = case
    w = wl.ragged(sizes, d=d, chains=chains, m=m, ard=ard, seed=sum(sizes) + 7 * d)
    _check_backward(kmv_handle, w, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_forward_col_shift_and_fp64_rows(kmv_handle, prec):
    w = wl.ragged([270], d=2, chains=2, m=3, seed=41)
    _check_forward(kmv_handle, w, prec, col_shift=np.array([0.0, 0.25, 4.0]), want64=True)


@pytest.mark.parametrize("prec", PRECS)
def test_unit_vector_gives_column(kmv_handle, prec):
    w = wl.ragged([260], d=3, chains=1, m=1, seed=42)
    E = np.zeros((1, 260, 3))
    for k, j in enumerate([0, 131, 259]):
        E[0, j, k] = 1.0
    w.V = E
    _check_forward(kmv_handle, w, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_degenerate_sizes(kmv_handle, prec):
    # single point, one full tile exactly, tile + 1, empty instances around them
    w = wl.ragged([0, 1, 128, 129, 0], d=2, chains=2, m=2, seed=43)
    _check_forward(kmv_handle, w, prec)
    _check_backward(kmv_handle, w, prec)


def test_batched_equals_single_instance_bitwise(kmv_handle):
    w = wl.ragged([150, 300], d=3, chains=2, m=2, seed=44)
    pts, theta, V, G = to_dev(w)
    Y = kmv_handle.kmv_forward(pts, theta, V)
    g, _ = kmv_handle.kmv_backward(pts, theta, V, G)
    from paper_2412_20884_gb300 import Points
    r0, r1 = w.offsets[1], w.offsets[2]
    pts1 = Points(pts.x[r0:r1].contiguous(), None, ard=True)
    Y1 = kmv_handle.kmv_forward(pts1, theta[2:4].contiguous(), V[:, r0:r1].contiguous())
    g1, _ = kmv_handle.kmv_backward(pts1, theta[2:4].contiguous(), V[:, r0:r1].contiguous(),
                                    G[:, r0:r1].contiguous())
    assert torch.equal(Y[:, r0:r1], Y1)
    assert torch.equal(g[2:4], g1)
    # repeated calls are bitwise reproducible
    assert torch.equal(kmv_handle.kmv_backward(pts, theta, V, G)[0], g)


@pytest.mark.parametrize("prec", PRECS)
def test_c2_full_size_sampled_rows(kmv_handle, prec):
    """N = 65,536, d = 8, ARD, m = 16: forward on 256 sampled rows, and the whole
    backward output with G restricted to those rows (exact via the sampled-row form)."""
    w = wl.c2()
    pts, theta, V, G = to_dev(w)
    Y = kmv_handle.kmv_forward(pts, theta, V, prec=prec).cpu().numpy()[0]
    X, Vh = f32(w.X), f32(w.V[0])
    rows = w.rows
    ref = sk.kmv(X, w.theta[0], Vh, True, rows=rows)
    scale = sk.kmv(X, w.theta[0], np.abs(Vh), True, rows=rows)
    assert componentwise_err(Y[rows], ref, scale) <= TOL[prec][0]
    Gs = np.zeros_like(w.G)
    Gs[0, rows] = w.G[0, rows]
    Gd = torch.tensor(Gs, dtype=torch.float32, device="cuda")
    gth, gV = kmv_handle.kmv_backward(pts, theta, V, Gd, prec=prec)
    g_ref, gV_ref = sk.kmv_adjoint(X, w.theta[0], Vh, f32(Gs[0]), True, rows=rows)
    assert grad_err(gth.cpu().numpy()[0], g_ref) <= TOL[prec][1]
    probe = np.sort(np.random.default_rng(0).choice(w.n_total, 512, replace=False))
    gV = gV.cpu().numpy()[0]
    sc = np.abs(sk.kernel_matrix(X[probe], X[rows], w.theta[0], True)) @ np.abs(f32(Gs[0, rows]))
    sc[np.isin(probe, rows)] += math.exp(w.theta[0, -1]) * np.abs(f32(Gs[0]))[probe[np.isin(probe, rows)]]
    assert componentwise_err(gV[probe], gV_ref[probe], np.maximum(sc, 1e-30)) <= TOL[prec][0]


def test_autograd_function(kmv_handle):
    from paper_2412_20884_gb300.autograd import kmv
    w = wl.ragged([210], d=2, chains=1, m=2, seed=45)
    pts, theta, V, G = to_dev(w)
    theta.requires_grad_(True)
    V.requires_grad_(True)
    Y = kmv(theta, V, pts, "fp32", kmv_handle)
    (Y * G).sum().backward()
    g_ref, gV_ref = sk.kmv_adjoint(f32(w.X), w.theta[0], f32(w.V[0]), f32(w.G[0]), True)
    assert grad_err(theta.grad.cpu().numpy()[0], g_ref) <= 1e-4
    assert np.max(np.abs(V.grad.cpu().numpy()[0] - gV_ref)) <= 1e-5 * np.abs(gV_ref).max()


def test_invalid_arguments(kmv_handle):
    from paper_2412_20884_gb300 import KmvError, Points
    w = wl.ragged([50], d=2, chains=1, m=1, seed=46)
    pts, theta, V, G = to_dev(w)
    with pytest.raises(ValueError):
        kmv_handle.kmv_forward(pts, theta[:, :3].contiguous(), V)
    with pytest.raises(KmvError) as e:
        kmv_handle.kmv_forward(pts, theta, V, Y=V)       # aliasing output
    assert e.value.status == 1
    with pytest.raises(KmvError):
        kmv_handle.kmv_cg_solve(pts, theta, torch.ones(50, device="cuda"), tol=-1.0)
    big = Points(torch.zeros((3, 65), device="cuda"), None, ard=False)
    with pytest.raises(KmvError):
        kmv_handle.kmv_forward(big, torch.zeros((1, 3), dtype=torch.float64, device="cuda"),
                               torch.zeros((1, 3, 1), device="cuda"))


@pytest.mark.parametrize("prec", PRECS)
def test_kernel_timing(kmv_handle, prec):
    """kmv_profile_enable / kmv_profile_read count the main-kernel launches of
    each kind and return positive device time; reading clears the records."""
    from paper_2412_20884_gb300.binding import KMV_KERNEL_FORWARD, KMV_KERNEL_ADJOINT
    h = kmv_handle
    w = wl.ragged([300, 77], d=3, chains=2, m=2, ard=True, seed=5)
    pts, theta, V, G = to_dev(w)
    h.profile_enable(True)
    try:
        h.kmv_forward(pts, theta, V, prec=prec)
        h.kmv_backward(pts, theta, V, G, prec=prec)
        fms, fn = h.profile_read(KMV_KERNEL_FORWARD)
        ams, an = h.profile_read(KMV_KERNEL_ADJOINT)
        # the BF16 backward forms dL/dV with a second forward pass
        assert fn == (2 if prec == "bf16_hilo" else 1) and an == 1
        assert fms > 0.0 and ams > 0.0
        assert h.profile_read(KMV_KERNEL_FORWARD) == (0.0, 0)
    finally:
        h.profile_enable(False)
    h.kmv_forward(pts, theta, V, prec=prec)
    assert h.profile_read(KMV_KERNEL_FORWARD) == (0.0, 0)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("m", [1, 16])
def test_many_tiles_per_cta(kmv_handle, prec, m):
    """Enough tiles that every persistent CTA runs several work items of
    several J tiles each (the small cases give one tile per CTA), so the
    phase bookkeeping of the pipelines is exercised over many rounds."""
    w = wl.ragged([6000, 2192], d=4, chains=1, m=m, ard=True, seed=61)
    _check_forward(kmv_handle, w, prec)
    _check_backward(kmv_handle, w, prec)


@pytest.mark.parametrize("case", [c for c in CASES if c[3] <= 2 and c[1] <= 17],
                         ids=lambda c: f"N{sum(c[0])}d{c[1]}c{c[2]}m{c[3]}")
def test_bf16_cg_product_has_fp32_accuracy(kmv_handle, case):
    """The BF16 form's product for one or two columns (the CG iterations and the
    energy's solves): three-way split exponent and FP32 P.v on the FMA pipe.  It
    meets the FP32 form's 1e-5, which is why the BF16 form solves with it directly."""
    sizes, d, chains, m, ard = case
    w = wl.ragged(sizes, d=d, chains=chains, m=m, ard=ard, seed=sum(sizes) + d)
    pts, theta, V, _ = to_dev(w)
    Y = kmv_handle.kmv_forward(pts, theta, V, prec="bf16_hilo").cpu().numpy()
    X, Vh = f32(w.X), f32(w.V)
    for b in range(w.n_inst):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        if r1 == r0:
            continue
        for c in range(w.chains):
            s = b * w.chains + c
            ref = sk.kmv(X[r0:r1], w.theta[s], Vh[c, r0:r1], w.ard)
            scale = abs_row_products(X[r0:r1], w.theta[s], Vh[c, r0:r1], w.ard, None)
            assert componentwise_err(Y[c, r0:r1], ref, scale) <= 1e-5

"""Tile choices and the autotuner of the tensor-core kernels, through the C ABI:
every exp split (MUFU only, one element in 8 or in 4 by the FMA-pipe
polynomial), stage limit and plan density keeps parity with the FP64 oracle;
kmv_autotune records choices, writes its cache file and leaves results at
the stated accuracy."""
import numpy as np
import pytest
import torch

import workloads as wl
from helpers import componentwise_err, f32, to_dev
from test_gpu_kmv import _check_backward, _check_forward

pytestmark = pytest.mark.gpu


def _kinds():
    from paper_2412_20884_gb300.binding import KMV_TILES_ADJOINT, KMV_TILES_FORWARD, KMV_TILES_FORWARD_FMA
    return KMV_TILES_FORWARD, KMV_TILES_FORWARD_FMA, KMV_TILES_ADJOINT


def test_set_get_tiles_and_bad_values(kmv_handle):
    from paper_2412_20884_gb300 import KmvError
    h = kmv_handle
    fwd, fma, adj = _kinds()
    before = [h.get_tiles(k) for k in (fwd, fma, adj)]
    try:
        h.set_tiles(fwd, stages=3, items_per_sm=9, exp_split=8)
        assert h.get_tiles(fwd) == {"stages": 3, "items_per_sm": 9, "exp_split": 8}
        h.set_tiles(fma, stages=0, items_per_sm=6, exp_split=3)   # rounds to the built split 4
        assert h.get_tiles(fma)["exp_split"] == 4
        for bad in ({"stages": 1}, {"stages": 9}, {"items_per_sm": 0}, {"items_per_sm": 65}, {"exp_split": -1}):
            with pytest.raises(KmvError):
                h.set_tiles(fwd, **{**{"stages": 0, "items_per_sm": 6, "exp_split": 0}, **bad})
        with pytest.raises(KmvError):
            h.set_tiles(7)
    finally:
        for k, t in zip((fwd, fma, adj), before):
            h.set_tiles(k, **t)


@pytest.mark.parametrize("split", [0, 8, 4])
@pytest.mark.parametrize("stages,ipsm", [(0, 6), (2, 1), (3, 13)])
def test_tile_choices_keep_parity(kmv_handle, split, stages, ipsm):
    h = kmv_handle
    fwd, fma, adj = _kinds()
    before = [h.get_tiles(k) for k in (fwd, fma, adj)]
    try:
        for k in (fwd, fma, adj):
            h.set_tiles(k, stages=stages, items_per_sm=ipsm, exp_split=split)
        for m in (1, 2, 16):
            w = wl.ragged([700, 0, 129], d=3, chains=2, m=m, ard=True, seed=300 + m)
            _check_forward(h, w, "bf16_hilo")
        w = wl.ragged([900, 257], d=5, chains=1, m=4, ard=True, seed=310)
        _check_backward(h, w, "bf16_hilo")
    finally:
        for k, t in zip((fwd, fma, adj), before):
            h.set_tiles(k, **t)


def test_autotune_records_and_cache(kmv_handle, tmp_path):
    from paper_2412_20884_gb300 import Kmv
    h = kmv_handle
    w = wl.ragged([3000, 1000], d=4, chains=2, m=16, ard=True, seed=320)
    pts, theta, V, G = to_dev(w)
    path = tmp_path / "tiles.txt"
    h.autotune(pts, theta, 16, cache_path=str(path))
    h.autotune(pts, theta, 1, cache_path=str(path))
    lines = [l.split() for l in path.read_text().splitlines() if not l.startswith("#")]
    kinds = sorted({int(l[0]) for l in lines})
    assert kinds == [0, 1, 2], lines
    for l in lines:
        assert int(l[1]) == 4 and int(l[3]) == 11            # d, floor(log2 3000)
        assert float(l[7]) > 0.0
    # the recorded choices are used: results stay at the stated accuracy
    _check_forward(h, w, "bf16_hilo")
    _check_backward(h, w, "bf16_hilo")
    w1 = wl.ragged([3000, 1000], d=4, chains=2, m=1, ard=True, seed=321)
    _check_forward(h, w1, "bf16_hilo")
    # a second handle reads the cache instead of timing again, and writes it back unchanged
    h2 = Kmv(0)
    try:
        before = path.read_text()
        h2.autotune(pts, theta, 16, cache_path=str(path))
        assert path.read_text() == before
    finally:
        h2.close()
    with pytest.raises(Exception):
        h.autotune(pts, theta, 0)


@pytest.mark.parametrize("m", [1, 2])
def test_fma_product_with_many_items_per_cta(kmv_handle, m):
    """The one- and two-column product (the CG iterations' kernel) with a
    dense plan, about 30 work items per CTA: each I tile's two column-half
    warpgroups then hand their row sums over through both parity buffers
    many times.  Sampled rows against the FP64 oracle at the FP32 form's
    1e-5 (componentwise, relative to the row sums of |K||V|)."""
    from oracle import se_kernel as sk
    h = kmv_handle
    _, fma, _ = _kinds()
    before = h.get_tiles(fma)
    w = wl.ragged([12000, 5000], d=3, chains=2, m=m, ard=True, seed=330 + m)
    pts, theta, V, _ = to_dev(w)
    try:
        h.set_tiles(fma, stages=0, items_per_sm=32, exp_split=0)
        Y = h.kmv_forward(pts, theta, V, prec="bf16_hilo").cpu().numpy()
    finally:
        h.set_tiles(fma, **before)
    X, Vh = f32(w.X), f32(w.V)
    rng = np.random.default_rng(331)
    for b in range(w.n_inst):
        r0, r1 = w.offsets[b], w.offsets[b + 1]
        rows = np.sort(rng.choice(r1 - r0, size=64, replace=False))
        for c in range(w.chains):
            s = b * w.chains + c
            ref = sk.kmv(X[r0:r1], w.theta[s], Vh[c, r0:r1], True, rows=rows)
            scale = sk.kmv(X[r0:r1], w.theta[s], np.abs(Vh[c, r0:r1]), True, rows=rows)
            assert componentwise_err(Y[c, r0:r1][rows], ref, scale) <= 1e-5, (b, c)

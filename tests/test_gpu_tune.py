"""Tile choices and the autotuner of the tensor-core kernels, through the C ABI:
every exp split (MUFU only, one element in 8 or in 4 by the FMA-pipe
polynomial), stage limit and plan density keeps parity with the FP64 oracle;
kmv_autotune records choices, writes its cache file and leaves results at
the stated accuracy."""
import numpy as np
import pytest
import torch

import workloads as wl
from helpers import to_dev
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

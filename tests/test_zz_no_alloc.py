"""kmv_backward_noalloc against kmv_backward (KMV_FP32), through the C ABI.

The allocation-free adjoint serves callers that cannot allocate device memory
(graph capture, caller-owned memory pools, allocation-free loops); it keeps its
scratch in a fixed array inside the library.  It must reproduce the handle-based
FP32 adjoint within the FP32 tolerances (gradients 1e-4, dL/dV 1e-5), on two
calls in a row (the second call finds the array holding the first call's data).
This file is collected last so that a failure here stops a run only after every
other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as wl
from helpers import to_dev, grad_err

pytestmark = pytest.mark.gpu


def test_backward_noalloc_matches_backward(kmv_handle):
    from paper_2412_20884_gb300 import binding
    w = wl.ragged([300, 0, 129, 64], d=3, chains=2, m=2, seed=70)
    pts, theta, V, G = to_dev(w)
    g_ref, gV_ref = kmv_handle.kmv_backward(pts, theta, V, G, prec="fp32")
    g_ref, gV_ref = g_ref.cpu().numpy(), gV_ref.cpu().numpy()
    for _call in range(2):
        g, gV = binding.kmv_backward_noalloc(pts, theta, V, G)
        torch.cuda.synchronize()
        g, gV = g.cpu().numpy(), gV.cpu().numpy()
        for s in range(theta.shape[0]):
            if np.all(g_ref[s] == 0):
                assert np.all(g[s] == 0)
            else:
                assert grad_err(g[s], g_ref[s]) <= 1e-4
        assert np.max(np.abs(gV - gV_ref)) <= 1e-5 * np.abs(gV_ref).max()


def test_backward_noalloc_second_shape_then_first(kmv_handle):
    """A different problem in between must not leave stale scratch behind."""
    from paper_2412_20884_gb300 import binding
    a = wl.ragged([200], d=2, chains=1, m=3, seed=71)
    b = wl.ragged([130, 77], d=4, chains=3, m=1, seed=72)
    pa, ta, Va, Ga = to_dev(a)
    pb, tb, Vb, Gb = to_dev(b)
    ref_a = kmv_handle.kmv_backward(pa, ta, Va, Ga)[0].cpu().numpy()
    ref_b = kmv_handle.kmv_backward(pb, tb, Vb, Gb)[0].cpu().numpy()
    got_a1 = binding.kmv_backward_noalloc(pa, ta, Va, Ga, want_grad_V=False)[0].cpu().numpy()
    got_b = binding.kmv_backward_noalloc(pb, tb, Vb, Gb, want_grad_V=False)[0].cpu().numpy()
    got_a2 = binding.kmv_backward_noalloc(pa, ta, Va, Ga, want_grad_V=False)[0].cpu().numpy()
    assert grad_err(got_a1[0], ref_a[0]) <= 1e-4 and grad_err(got_a2[0], ref_a[0]) <= 1e-4
    for s in range(tb.shape[0]):
        assert grad_err(got_b[s], ref_b[s]) <= 1e-4


def test_backward_noalloc_rejects_oversized_problem(kmv_handle):
    """A problem whose tables and partials exceed the fixed scratch is refused
    before any device work (the points are never read)."""
    from paper_2412_20884_gb300 import binding
    L = binding.lib()
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    offsets = np.array([0, 1 << 26], dtype=np.int64)
    pts = binding._Points(1, offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 1, 0,
                          ctypes.c_void_p(dummy.data_ptr()))
    st = L.kmv_backward_noalloc(ctypes.byref(pts), 1, ctypes.c_void_p(dummy.data_ptr()),
                                ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()), 1,
                                ctypes.c_void_p(dummy.data_ptr()), None, None)
    assert st == binding.KMV_EINVAL

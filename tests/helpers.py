"""Shared helpers of the GPU parity tests: device copies of a workload and the
error measures used against the FP64 oracle."""
import numpy as np
import torch

from oracle import se_kernel as sk


def f32(a):
    """The values the GPU sees: inputs rounded to FP32, then exact in FP64."""
    return np.asarray(a, np.float32).astype(np.float64)


def to_dev(w, dev="cuda:0"):
    from paper_2412_20884_gb300 import Points
    pts = Points(torch.tensor(w.X, dtype=torch.float32, device=dev), w.offsets, ard=w.ard)
    theta = torch.tensor(w.theta, dtype=torch.float64, device=dev)
    V = None if w.V is None else torch.tensor(w.V, dtype=torch.float32, device=dev)
    G = None if w.G is None else torch.tensor(w.G, dtype=torch.float32, device=dev)
    return pts, theta, V, G


def abs_row_products(X, theta, V, ard, rows):
    """sum_j |A_ij| |V_jc| for the given rows (the scale of componentwise errors)."""
    return sk.kmv(X, theta, np.abs(V), ard, rows=rows)


def componentwise_err(Y, Y_ref, scale):
    return float(np.max(np.abs(Y - Y_ref) / np.maximum(scale, 1e-300)))


def grad_err(g, g_ref):
    """max_p |g_p - g*_p| / max(|g*_p|, 1e-3 ||g*||_inf)."""
    g, g_ref = np.asarray(g), np.asarray(g_ref)
    floor = 1e-3 * np.abs(g_ref).max()
    return float(np.max(np.abs(g - g_ref) / np.maximum(np.abs(g_ref), floor)))

"""Algorithm 1 on the GPU (paper_2412_20884_gb300.sampler.hmc_update: phi draw,
energies, leapfrog steps and the Metropolis test, all through the C ABI) on the
Sec. 4.1 verification data, against trapezoid quadrature of Eq. P computed by
the FP64 oracle; the same settings as the oracle's own sampler test, in both
precision forms (the BF16 form draws phi, solves and forms the force with the
tensor-core products; the energies are FP32 in both)."""
import json
import math
import os

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import diagnostics as dg
from oracle import hmc

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "verification_sec41.json")


@pytest.mark.parametrize("prec", ["fp32", "bf16_hilo"])
def test_algorithm1_matches_quadrature(kmv_handle, prec):
    from paper_2412_20884_gb300 import Points
    from paper_2412_20884_gb300.sampler import hmc_update
    cfg = json.load(open(GOLDEN))
    w = wl.tiny_verification(cfg["n_points"])
    X, y = w.X, w.y
    base = w.theta[0].copy()
    prior_np = {"mu": np.zeros(3), "prec": np.array([1.0, 1.0, 0.0])}
    g = np.linspace(-5.0, 5.0, 161)
    logp = np.empty((len(g), len(g)))
    for i, a in enumerate(g):
        for j, l in enumerate(g):
            logp[i, j] = hmc.log_posterior(X, y, np.array([a, l, base[-1]]), False, prior_np)
    cdfs = [dg.marginal_cdf_grid(logp, g, ax) for ax in (0, 1)]

    B, updates, burn = 192, 700, 150
    dev = "cuda"
    pts = Points(torch.tensor(X, dtype=torch.float32, device=dev), None, ard=False)
    yd = torch.tensor(y, dtype=torch.float32, device=dev)
    prior = (torch.zeros(3, dtype=torch.float64, device=dev), torch.tensor([1.0, 1.0, 0.0], dtype=torch.float64,
                                                                           device=dev))
    free = torch.tensor([1, 1, 0], dtype=torch.uint8, device=dev)
    th = torch.tensor(np.tile(np.array([0.01, 0.01, base[-1]]), (B, 1)), dtype=torch.float64, device=dev)
    rng = wl.rng_for(0)
    trace, acc = [], []
    for _t in range(updates):
        xi = torch.tensor(rng.standard_normal((B, len(y))), dtype=torch.float32, device=dev)
        pi = torch.tensor(rng.standard_normal((B, 3)), dtype=torch.float64, device=dev)
        u = torch.tensor(1.0 - rng.uniform(size=B), dtype=torch.float64, device=dev)   # (0, 1]
        ok, fail = hmc_update(kmv_handle, pts, yd, th, cfg["leapfrog_dt"], cfg["leapfrog_n_int"], xi, pi, u,
                              prior=prior, free_mask=free, prec=prec)
        trace.append(th[:, :2].cpu().numpy().copy())
        acc.append(float(ok.float().mean()))
        assert int((fail != 0).sum()) == 0
    trace = np.array(trace[burn:])
    assert np.mean(acc) > 0.4
    pts_c = np.linspace(-3.0, 3.0, cfg["cdf_points"])
    L = trace.shape[0]
    for ax in range(2):
        tau = np.mean([dg.iat(trace[:, b, ax]) for b in range(0, B, 8)])
        n_eff = B * L / tau
        radius = math.sqrt(math.log(2 / 0.01) / (2 * n_eff))
        emp = np.array([(trace[:, :, ax] <= p).mean() for p in pts_c])
        ref = np.interp(pts_c, g, cdfs[ax])
        assert np.abs(emp - ref).max() < radius, (ax, np.abs(emp - ref).max(), radius)

"""Seeded synthetic inputs shared by the tests, the benchmark and the FP64 oracle.

This module only draws random numbers and builds data sets.  It holds none of
the method's arithmetic (no kernel, no product, no gradient, no sampler), so
the CUDA path and the oracle can both consume it without sharing any
computation.

Every generator uses ``numpy.random.Generator(PCG64(seed))``.  Hyperparameters
are returned in the log parameterisation used throughout the library:

    theta = [log alpha, log ell_1 .. log ell_k, log sigma^2]

with k = 1 (isotropic) or k = d (ARD, one lengthscale per input dimension).

The shapes follow the paper's workloads (Sec. 4.1 and 4.2: points in a box,
smooth targets plus Gaussian noise, a squared-exponential kernel whose
lengthscale narrows as N grows) and the five benchmark configurations:

  * ``c1`` : N=2048, d=1, x ~ U[0,1], y = sin(2 pi x) + N(0, 0.1^2), isotropic
             theta = (log 1, log 0.2, log 0.01), one vector v ~ N(0, I).
  * ``c2`` : N=65536, d=8, x ~ N(0, I), ARD lengthscales log-uniform in
             [0.3, 3], alpha = 1, sigma^2 = 0.05, m = 16 vectors V, G ~ N(0, I).
  * ``c3`` : N=262144, d=32, x ~ U[-1,1]^32, ARD lengthscales log-uniform in
             [0.5, 5], alpha = 1, sigma^2 = 0.05, m = 64.
  * ``c4`` : 256 independent instances, N_b = floor(exp(U[log 1e3, log 2e4])),
             d = 4, x ~ U[0,1]^4, y = sum_k sin(2 pi x_k) + N(0, 0.05^2), ARD
             lengthscales log-uniform in [0.3, 3], 4 chains per instance.
  * ``c5`` : N=1048576, d=3, x ~ U[0,1]^3, y = sum_k sin(2 pi x_k) + N(0, 0.05^2),
             lengthscale from the narrowing rule 2 l^2 = (N/1e4)^(-2/d) of
             Sec. 4.2, sigma^2 = 0.1, 8 chains.

Every generator takes an ``n`` override so the tests can build the same
distribution at sizes the oracle finishes in seconds.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Workload:
    """A batch of GP instances with per-(instance, chain) hyperparameters.

    X        : (N_total, d) float64, instances concatenated along rows.
    offsets  : (n_inst + 1,) int64, rows of instance b are offsets[b]:offsets[b+1].
    y        : (N_total,) float64 observations.
    theta    : (n_inst * chains, n_theta) float64, row b * chains + c.
    V, G     : (chains, N_total, m) float64 right-hand sides / adjoint seeds.
    rows     : optional sampled row indices (global) for large-N checks.
    """

    name: str
    X: np.ndarray
    offsets: np.ndarray
    y: np.ndarray
    theta: np.ndarray
    ard: bool
    chains: int
    V: np.ndarray | None = None
    G: np.ndarray | None = None
    rows: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return self.X.shape[1]

    @property
    def n_inst(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_total(self) -> int:
        return int(self.offsets[-1])

    @property
    def n_theta(self) -> int:
        return self.theta.shape[1]

    @property
    def m(self) -> int:
        return 0 if self.V is None else self.V.shape[2]


def log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))


def theta_vector(alpha: float, ells, sigma2: float) -> np.ndarray:
    ells = np.atleast_1d(np.asarray(ells, dtype=np.float64))
    return np.concatenate([[math.log(alpha)], np.log(ells), [math.log(sigma2)]])


def _vectors(rng, chains, n, m):
    if m == 0:
        return None
    return rng.standard_normal((chains, n, m))


def c1(n: int = 2048, m: int = 1, seed: int = 0) -> Workload:
    rng = rng_for(seed)
    x = rng.uniform(0.0, 1.0, size=(n, 1))
    y = np.sin(2 * np.pi * x[:, 0]) + 0.1 * rng.standard_normal(n)
    theta = theta_vector(1.0, [0.2], 0.01)[None, :]
    V = _vectors(rng, 1, n, m)
    G = _vectors(rng, 1, n, m)
    return Workload("c1", x, np.array([0, n], np.int64), y, theta, False, 1, V, G)


def c2(n: int = 65536, m: int = 16, n_rows: int = 256, seed: int = 0) -> Workload:
    rng = rng_for(seed)
    d = 8
    x = rng.standard_normal((n, d))
    ells = log_uniform(rng, 0.3, 3.0, d)
    theta = theta_vector(1.0, ells, 0.05)[None, :]
    V = _vectors(rng, 1, n, m)
    G = _vectors(rng, 1, n, m)
    y = rng.standard_normal(n)
    rows = np.sort(rng.choice(n, size=min(n_rows, n), replace=False))
    return Workload("c2", x, np.array([0, n], np.int64), y, theta, True, 1, V, G, rows)


def c3(n: int = 262144, m: int = 64, n_rows: int = 1024, seed: int = 0) -> Workload:
    rng = rng_for(seed)
    d = 32
    x = rng.uniform(-1.0, 1.0, size=(n, d))
    ells = log_uniform(rng, 0.5, 5.0, d)
    theta = theta_vector(1.0, ells, 0.05)[None, :]
    V = _vectors(rng, 1, n, m)
    G = _vectors(rng, 1, n, m)
    y = rng.standard_normal(n)
    rows = np.sort(rng.choice(n, size=min(n_rows, n), replace=False))
    return Workload("c3", x, np.array([0, n], np.int64), y, theta, True, 1, V, G, rows)


def c4(n_inst: int = 256, n_lo: float = 1e3, n_hi: float = 2e4, chains: int = 4,
       m: int = 1, seed: int = 0) -> Workload:
    rng = rng_for(seed)
    d = 4
    sizes = np.floor(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=n_inst))).astype(np.int64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offsets[-1])
    x = rng.uniform(0.0, 1.0, size=(n, d))
    y = np.sin(2 * np.pi * x).sum(axis=1) + 0.05 * rng.standard_normal(n)
    thetas = []
    for _b in range(n_inst):
        ells = log_uniform(rng, 0.3, 3.0, d)
        t = theta_vector(1.0, ells, 0.05)
        for _c in range(chains):
            thetas.append(t + 0.05 * rng.standard_normal(t.shape))
    theta = np.stack(thetas)
    V = _vectors(rng, chains, n, m)
    G = _vectors(rng, chains, n, m)
    return Workload("c4", x, offsets, y, theta, True, chains, V, G)


def c5(n: int = 1048576, chains: int = 8, m: int = 1, seed: int = 0, n_rows: int = 1024) -> Workload:
    rng = rng_for(seed)
    d = 3
    x = rng.uniform(0.0, 1.0, size=(n, d))
    y = np.sin(2 * np.pi * x).sum(axis=1) + 0.05 * rng.standard_normal(n)
    ell = math.sqrt(0.5 * (n / 1e4) ** (-2.0 / d))
    t = theta_vector(1.0, [ell] * d, 0.1)
    theta = np.stack([t + 0.02 * rng.standard_normal(t.shape) for _ in range(chains)])
    V = _vectors(rng, chains, n, m)
    G = _vectors(rng, chains, n, m)
    rows = np.sort(rng.choice(n, size=min(n_rows, n), replace=False))
    return Workload("c5", x, np.array([0, n], np.int64), y, theta, True, chains, V, G, rows)


def ragged(sizes, d: int = 3, chains: int = 2, m: int = 2, ard: bool = True,
           seed: int = 0, ell_range=(0.3, 2.0), sigma2: float = 0.05) -> Workload:
    """Several instances of the given sizes (zero sizes allowed), generic shapes for parity tests."""
    rng = rng_for(seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offsets[-1])
    x = rng.uniform(-1.0, 1.0, size=(n, d))
    y = np.cos(x).prod(axis=1) + 0.1 * rng.standard_normal(n)
    thetas = []
    for _b in range(len(sizes)):
        for _c in range(chains):
            k = d if ard else 1
            ells = log_uniform(rng, ell_range[0], ell_range[1], k)
            alpha = math.exp(rng.uniform(-0.5, 0.5))
            thetas.append(theta_vector(alpha, ells, sigma2 * math.exp(rng.uniform(-0.5, 0.5))))
    theta = np.stack(thetas)
    V = _vectors(rng, chains, n, m)
    G = _vectors(rng, chains, n, m)
    return Workload("ragged", x, offsets, y, theta, ard, chains, V, G)


def cheb(sizes, d: int = 2, n_cheb: int = 3, chains: int = 2, m: int = 2, ard: bool = False,
         seed: int = 0, ell_range=(0.3, 1.0), sigma2: float = 0.05, theta_scale: float = 0.3) -> Workload:
    """Instances for the Chebyshev log-amplitude kernel of Sec. 4: points uniform in
    [-1, 1]^d, theta rows [Theta (n_cheb^d, N(0, theta_scale^2) / (1 + |t|_1)), log l, log sigma^2]."""
    rng = rng_for(seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offsets[-1])
    x = rng.uniform(-1.0, 1.0, size=(n, d))
    y = np.cos(2.0 * x).prod(axis=1) + 0.1 * rng.standard_normal(n)
    deg = np.indices((n_cheb,) * d).reshape(d, -1).sum(axis=0)
    thetas = []
    for _b in range(len(sizes)):
        for _c in range(chains):
            k = d if ard else 1
            coef = theta_scale * rng.standard_normal(deg.size) / (1.0 + deg)
            ells = log_uniform(rng, ell_range[0], ell_range[1], k)
            thetas.append(np.concatenate([coef, np.log(ells), [math.log(sigma2)]]))
    theta = np.stack(thetas)
    V = _vectors(rng, chains, n, m)
    G = _vectors(rng, chains, n, m)
    return Workload("cheb", x, offsets, y, theta, ard, chains, V, G, meta={"cheb": n_cheb})


def tiny_verification(n: int = 10) -> Workload:
    """Sec. 4.1's verification data: N equispaced points on [-1, 1), y_i = 1."""
    x = (-1.0 + 2.0 * np.arange(n) / n)[:, None]
    y = np.ones(n)
    theta = theta_vector(1.0, [math.sqrt(0.5)], 0.1)[None, :]
    return Workload("tiny", x, np.array([0, n], np.int64), y, theta, False, 1)


CONFIGS = {"c1": c1, "c2": c2, "c3": c3, "c4": c4, "c5": c5}

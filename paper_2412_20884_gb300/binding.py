"""ctypes binding of libkmv (include/kmv.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  There is no CPU fallback; if ``_build/libkmv.so`` is missing the
binding raises at load time.  Tensors are torch CUDA tensors (torch supplies
device memory and streams); all calls are enqueued on the current torch
stream unless a stream is given.

Python names match the C entry points: ``kmv_forward``, ``kmv_backward``,
``kmv_cg_solve``, ``leapfrog_step``, ``kmv_energy``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

KMV_OK, KMV_EINVAL, KMV_ENOMEM, KMV_ECUDA, KMV_ENOTCONV, KMV_ETIMEOUT, KMV_ENONFINITE, KMV_EUNSUPPORTED = range(8)
PRECISIONS = {"fp32": 0, "bf16_hilo": 1}

_LIB = None


class KmvError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{message} (status {status})")
        self.status = status


class _Nystrom(C.Structure):
    _fields_ = [("rank", C.c_int32), ("n_inst", C.c_int32), ("chains", C.c_int32), ("n_total", C.c_int64),
                ("U", C.c_void_p), ("lam", C.c_void_p)]


class _Tiles(C.Structure):
    _fields_ = [("stages", C.c_int32), ("items_per_sm", C.c_int32), ("exp_split", C.c_int32)]


class _Points(C.Structure):
    _fields_ = [("n_inst", C.c_int32), ("offsets", C.POINTER(C.c_int64)), ("d", C.c_int32),
                ("ard", C.c_int32), ("x", C.c_void_p), ("cheb", C.c_int32)]


_P = C.c_void_p
_SIGS = {
    "kmv_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "kmv_destroy": (C.c_int, [_P]),
    "kmv_status_string": (C.c_char_p, [C.c_int]),
    "kmv_last_error": (C.c_char_p, [_P]),
    "kmv_workspace_bytes": (C.c_int64, [_P]),
    "kmv_forward": (C.c_int, [_P, C.POINTER(_Points), C.c_int32, _P, _P, C.c_int32, _P, _P, _P, C.c_int, _P]),
    "kmv_backward": (C.c_int, [_P, C.POINTER(_Points), C.c_int32, _P, _P, _P, C.c_int32, _P, _P, C.c_int, _P]),
    "kmv_cg_solve": (C.c_int, [_P, C.POINTER(_Points), C.c_int32, _P, _P, C.c_int32, _P, C.c_double,
                               C.c_int32, C.c_int32, _P, _P, C.c_int, _P]),
    "leapfrog_step": (C.c_int, [_P, C.POINTER(_Points), C.c_int32, _P, _P, _P, _P, C.c_double, _P, _P, _P,
                                C.c_double, C.c_int32, _P, _P, _P, C.c_int, _P]),
    "kmv_implicit_step": (C.c_int, [_P, C.POINTER(_Points), C.c_int32, _P, _P, _P, _P, C.c_double, _P, _P, _P,
                                    C.c_int32, C.c_double, C.c_int32, _P, _P, _P, C.c_int, _P]),
    "kmv_energy": (C.c_int, [_P, C.POINTER(_Points), C.c_int32, _P, _P, _P, _P, _P, _P, C.c_double,
                             C.c_int32, _P, _P, _P, _P, _P, C.c_int, _P]),
    "kmv_backward_noalloc": (C.c_int, [C.POINTER(_Points), C.c_int32, _P, _P, _P, C.c_int32, _P, _P, _P]),
    "kmv_phi_refresh": (C.c_int, [_P, C.POINTER(_Points), C.c_int32, _P, _P, _P, C.c_int32, C.c_double,
                                  C.c_int32, _P, _P, _P, C.c_int, _P]),
    "kmv_nystrom_build": (C.c_int, [_P, C.POINTER(_Points), C.c_int32, _P, C.c_int32, _P, _P, _P, _P, C.c_int,
                                    _P]),
    "kmv_set_preconditioner": (C.c_int, [_P, _P]),
    "kmv_accept": (C.c_int, [C.c_int32, C.c_int32, _P, _P, _P, _P, _P, _P, _P, _P]),
    "kmv_status_merge": (C.c_int, [C.c_int32, _P, _P, _P]),
    "kmv_profile_enable": (C.c_int, [_P, C.c_int32]),
    "kmv_set_tiles": (C.c_int, [_P, C.c_int32, C.POINTER(_Tiles)]),
    "kmv_get_tiles": (C.c_int, [_P, C.c_int32, C.POINTER(_Tiles)]),
    "kmv_autotune": (C.c_int, [_P, C.POINTER(_Points), C.c_int32, _P, C.c_int32, C.c_char_p, _P]),
    "kmv_profile_read": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
}

KMV_KERNEL_FORWARD, KMV_KERNEL_ADJOINT = 0, 1
KMV_TILES_FORWARD, KMV_TILES_FORWARD_FMA, KMV_TILES_ADJOINT = 0, 1, 2


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libkmv.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libkmv.so not found at {path}: run __graft_entry__.build() first")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _need(t, dtype, name, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


class Points:
    """A point set: instances concatenated along rows of x (N_total, d).

    cheb = N_cheb >= 1 selects the Chebyshev log-amplitude kernel of Sec. 4, with
    theta rows [Theta (N_cheb^d), log l (1 or d), log sigma^2]; 0 is the SE kernel."""

    def __init__(self, x: torch.Tensor, offsets=None, ard: bool = True, cheb: int = 0):
        _need(x, torch.float32, "x")
        if x.dim() != 2:
            raise ValueError("x must be (N_total, d)")
        self.x = x
        n = x.shape[0]
        off = np.array([0, n] if offsets is None else offsets, dtype=np.int64)
        if off[0] != 0 or off[-1] != n or np.any(np.diff(off) < 0):
            raise ValueError("offsets must start at 0, end at N_total and be non-decreasing")
        self.offsets = np.ascontiguousarray(off)
        self.ard = bool(ard)
        self.d = x.shape[1]
        self.n_inst = len(off) - 1
        self.n_total = n
        self.cheb = int(cheb)
        k = self.d if self.ard else 1
        self.n_theta = (self.cheb ** self.d + k + 1) if self.cheb else 2 + k
        self._c = _Points(self.n_inst, self.offsets.ctypes.data_as(C.POINTER(C.c_int64)), self.d,
                          int(self.ard), C.c_void_p(x.data_ptr()), self.cheb)

    @property
    def c(self):
        return C.byref(self._c)

    def pairs(self, chains: int = 1) -> int:
        nb = np.diff(self.offsets).astype(np.float64)
        return int(np.sum(nb * nb)) * chains


class Kmv:
    """A libkmv handle bound to one CUDA device."""

    def __init__(self, device: int = 0):
        self.L = lib()
        self.device = device
        h = C.c_void_p()
        st = self.L.kmv_create(C.byref(h), device)
        if st != KMV_OK:
            raise KmvError(st, "kmv_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.kmv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != KMV_OK:
            msg = self.L.kmv_last_error(self.h).decode() or self.L.kmv_status_string(st).decode()
            raise KmvError(st, msg)

    def workspace_bytes(self) -> int:
        return int(self.L.kmv_workspace_bytes(self.h))

    def profile_enable(self, on: bool = True):
        """Time every main product-kernel launch with CUDA events (kmv_profile_enable)."""
        self._check(self.L.kmv_profile_enable(self.h, 1 if on else 0))

    def profile_read(self, kind: int):
        """(total_ms, launches) of one kernel kind since the last read (kmv_profile_read)."""
        ms, n = C.c_double(0.0), C.c_int64(0)
        self._check(self.L.kmv_profile_read(self.h, kind, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def set_tiles(self, kernel: int, stages: int = 0, items_per_sm: int = 6, exp_split: int = 0):
        """Default tile choices of one tensor-core kernel kind (kmv_set_tiles)."""
        t = _Tiles(stages, items_per_sm, exp_split)
        self._check(self.L.kmv_set_tiles(self.h, kernel, C.byref(t)))

    def get_tiles(self, kernel: int) -> dict:
        """Default tile choices of one kernel kind (kmv_get_tiles)."""
        t = _Tiles()
        self._check(self.L.kmv_get_tiles(self.h, kernel, C.byref(t)))
        return {"stages": t.stages, "items_per_sm": t.items_per_sm, "exp_split": t.exp_split}

    def autotune(self, pts: "Points", theta, m: int, cache_path=None, stream=None):
        """Time candidate tiles for this call shape and record the fastest (kmv_autotune; synchronous)."""
        chains = self._chains(pts, theta)
        _need(theta, torch.float64, "theta", (pts.n_inst * chains, pts.n_theta))
        path = None if cache_path is None else os.fsencode(cache_path)
        self._check(self.L.kmv_autotune(self.h, pts.c, chains, _ptr(theta), int(m), path, _stream(stream)))

    @staticmethod
    def _prec(prec):
        return PRECISIONS[prec] if isinstance(prec, str) else int(prec)

    def _chains(self, pts, theta):
        n_sys = theta.shape[0]
        if n_sys % pts.n_inst:
            raise ValueError("theta rows must be n_inst * chains")
        return n_sys // pts.n_inst

    # ------------------------------------------------------------------ products
    def kmv_forward(self, pts: Points, theta, V, col_shift=None, Y=None, Y64=False,
                    prec="fp32", stream=None):
        chains = self._chains(pts, theta)
        _need(theta, torch.float64, "theta", (pts.n_inst * chains, pts.n_theta))
        m = V.shape[-1]
        _need(V, torch.float32, "V", (chains, pts.n_total, m))
        if col_shift is not None:
            _need(col_shift, torch.float32, "col_shift", (m,))
        if Y is None:
            Y = torch.empty_like(V)
        _need(Y, torch.float32, "Y", V.shape)
        y64 = None
        if Y64 is True:
            y64 = torch.empty(V.shape, dtype=torch.float64, device=V.device)
        elif isinstance(Y64, torch.Tensor):
            y64 = _need(Y64, torch.float64, "Y64", V.shape)
        self._check(self.L.kmv_forward(self.h, pts.c, chains, _ptr(theta), _ptr(V), m, _ptr(col_shift),
                                       _ptr(Y), _ptr(y64), self._prec(prec), _stream(stream)))
        return (Y, y64) if y64 is not None else Y

    def kmv_backward(self, pts: Points, theta, V, G, want_grad_V=True, grad_theta=None, grad_V=None,
                     prec="fp32", stream=None):
        chains = self._chains(pts, theta)
        _need(theta, torch.float64, "theta", (pts.n_inst * chains, pts.n_theta))
        m = V.shape[-1]
        _need(V, torch.float32, "V", (chains, pts.n_total, m))
        _need(G, torch.float32, "G", V.shape)
        if grad_theta is None:
            grad_theta = torch.empty_like(theta)
        _need(grad_theta, torch.float64, "grad_theta", theta.shape)
        if want_grad_V and grad_V is None:
            grad_V = torch.empty_like(V)
        if grad_V is not None:
            _need(grad_V, torch.float32, "grad_V", V.shape)
        self._check(self.L.kmv_backward(self.h, pts.c, chains, _ptr(theta), _ptr(V), _ptr(G), m,
                                        _ptr(grad_theta), _ptr(grad_V), self._prec(prec), _stream(stream)))
        return grad_theta, grad_V

    # ------------------------------------------------------------------ solves / HMC
    def kmv_cg_solve(self, pts: Points, theta, rhs, x=None, tol=1e-6, maxiter=1000, warm_start=False,
                     prec="fp32", stream=None):
        chains = self._chains(pts, theta)
        _need(theta, torch.float64, "theta", (pts.n_inst * chains, pts.n_theta))
        per_chain = rhs.dim() == 2
        _need(rhs, torch.float32, "rhs", (chains, pts.n_total) if per_chain else (pts.n_total,))
        if x is None:
            x = torch.zeros((chains, pts.n_total), dtype=torch.float32, device=rhs.device)
        _need(x, torch.float32, "x", (chains, pts.n_total))
        status = torch.empty(pts.n_inst * chains, dtype=torch.int32, device=rhs.device)
        iters = torch.empty_like(status)
        self._check(self.L.kmv_cg_solve(self.h, pts.c, chains, _ptr(theta), _ptr(rhs), int(per_chain),
                                        _ptr(x), float(tol), int(maxiter), int(bool(warm_start)),
                                        _ptr(status), _ptr(iters), self._prec(prec), _stream(stream)))
        return x, status, iters

    def nystrom_build(self, pts: Points, theta, omega, prec="fp32", stream=None):
        """Randomized Nystrom factorisation K ~ U diag(lam) U^T per system (kmv_nystrom_build).
        omega: (chains, N_total, rank) N(0, 1) draws.  Returns (U (chains, rank, N_total), lam, status)."""
        chains = self._chains(pts, theta)
        n_sys = pts.n_inst * chains
        _need(theta, torch.float64, "theta", (n_sys, pts.n_theta))
        rank = omega.shape[-1]
        _need(omega, torch.float32, "omega", (chains, pts.n_total, rank))
        U = torch.empty((chains, rank, pts.n_total), dtype=torch.float32, device=omega.device)
        lam = torch.empty((n_sys, rank), dtype=torch.float64, device=omega.device)
        status = torch.empty(n_sys, dtype=torch.int32, device=omega.device)
        self._check(self.L.kmv_nystrom_build(self.h, pts.c, chains, _ptr(theta), int(rank), _ptr(omega), _ptr(U),
                                             _ptr(lam), _ptr(status), self._prec(prec), _stream(stream)))
        return U, lam, status

    def set_preconditioner(self, pts: Points, U=None, lam=None):
        """Precondition every later CG solve on this handle with (U, lam) (kmv_set_preconditioner);
        U = None clears it.  The tensors are kept referenced while set."""
        if U is None:
            self._pc = None
            self._check(self.L.kmv_set_preconditioner(self.h, None))
            return
        chains, rank, n = U.shape
        _need(U, torch.float32, "U", (chains, rank, pts.n_total))
        _need(lam, torch.float64, "lam", (pts.n_inst * chains, rank))
        self._pc = (U, lam, _Nystrom(rank, pts.n_inst, chains, n, C.c_void_p(U.data_ptr()),
                                     C.c_void_p(lam.data_ptr())))
        self._check(self.L.kmv_set_preconditioner(self.h, C.byref(self._pc[2])))

    def phi_refresh(self, pts: Points, theta, xi, n_poles=15, cg_tol=1e-6, cg_maxiter=1000, phi=None,
                    want_poles=False, prec="fp32", stream=None):
        """phi = A^{-1/2} xi per system by the pole expansion (kmv_phi_refresh).
        Returns (phi, status, iters[, poles (n_sys, 2 + 2 n_poles)])."""
        chains = self._chains(pts, theta)
        n_sys = pts.n_inst * chains
        _need(theta, torch.float64, "theta", (n_sys, pts.n_theta))
        _need(xi, torch.float32, "xi", (chains, pts.n_total))
        if phi is None:
            phi = torch.empty_like(xi)
        _need(phi, torch.float32, "phi", (chains, pts.n_total))
        status = torch.empty(n_sys, dtype=torch.int32, device=xi.device)
        iters = torch.empty_like(status)
        poles = torch.empty((n_sys, 2 + 2 * n_poles), dtype=torch.float64, device=xi.device) if want_poles else None
        self._check(self.L.kmv_phi_refresh(self.h, pts.c, chains, _ptr(theta), _ptr(xi), _ptr(phi), int(n_poles),
                                           float(cg_tol), int(cg_maxiter), _ptr(status), _ptr(iters), _ptr(poles),
                                           self._prec(prec), _stream(stream)))
        return (phi, status, iters, poles) if want_poles else (phi, status, iters)

    def leapfrog_step(self, pts: Points, y, phi, theta, pi, dt, prior=None, free_mask=None,
                      cg_tol=1e-6, cg_maxiter=1000, x_work=None, prec="fp32", stream=None):
        chains = self._chains(pts, theta)
        n_sys = pts.n_inst * chains
        _need(y, torch.float32, "y", (pts.n_total,))
        _need(phi, torch.float32, "phi", (chains, pts.n_total))
        _need(theta, torch.float64, "theta", (n_sys, pts.n_theta))
        _need(pi, torch.float64, "pi", (n_sys, pts.n_theta))
        mu = prec_ = None
        if prior is not None:
            mu = _need(prior[0], torch.float64, "prior_mu", (pts.n_theta,))
            prec_ = _need(prior[1], torch.float64, "prior_prec", (pts.n_theta,))
        if free_mask is not None:
            _need(free_mask, torch.uint8, "free_mask", (pts.n_theta,))
        if x_work is None:
            x_work = torch.empty((chains, pts.n_total), dtype=torch.float32, device=y.device)
        status = torch.empty(n_sys, dtype=torch.int32, device=y.device)
        iters = torch.empty_like(status)
        self._check(self.L.leapfrog_step(self.h, pts.c, chains, _ptr(y), _ptr(phi), _ptr(theta), _ptr(pi),
                                         float(dt), _ptr(mu), _ptr(prec_), _ptr(free_mask), float(cg_tol),
                                         int(cg_maxiter), _ptr(x_work), _ptr(status), _ptr(iters),
                                         self._prec(prec), _stream(stream)))
        return status, iters, x_work

    def implicit_step(self, pts: Points, y, phi, theta, pi, dt, prior=None, free_mask=None, aa_depth=10,
                      tol=1e-6, maxiter=200, x_work=None, prec="fp32", stream=None):
        """One implicit midpoint step by Anderson acceleration (kmv_implicit_step); theta, pi
        and x_work (the starting x; zeros when None) are updated in place.  Returns (status, iters, x_work)."""
        chains = self._chains(pts, theta)
        n_sys = pts.n_inst * chains
        _need(y, torch.float32, "y", (pts.n_total,))
        _need(phi, torch.float32, "phi", (chains, pts.n_total))
        _need(theta, torch.float64, "theta", (n_sys, pts.n_theta))
        _need(pi, torch.float64, "pi", (n_sys, pts.n_theta))
        mu = prec_ = None
        if prior is not None:
            mu = _need(prior[0], torch.float64, "prior_mu", (pts.n_theta,))
            prec_ = _need(prior[1], torch.float64, "prior_prec", (pts.n_theta,))
        if free_mask is not None:
            _need(free_mask, torch.uint8, "free_mask", (pts.n_theta,))
        if x_work is None:
            x_work = torch.zeros((chains, pts.n_total), dtype=torch.float32, device=y.device)
        _need(x_work, torch.float32, "x_work", (chains, pts.n_total))
        status = torch.empty(n_sys, dtype=torch.int32, device=y.device)
        iters = torch.empty_like(status)
        self._check(self.L.kmv_implicit_step(self.h, pts.c, chains, _ptr(y), _ptr(phi), _ptr(theta), _ptr(pi),
                                             float(dt), _ptr(mu), _ptr(prec_), _ptr(free_mask), int(aa_depth),
                                             float(tol), int(maxiter), _ptr(x_work), _ptr(status), _ptr(iters),
                                             self._prec(prec), _stream(stream)))
        return status, iters, x_work

    def kmv_energy(self, pts: Points, y, phi, theta, pi=None, prior=None, cg_tol=1e-6, cg_maxiter=1000,
                   x_work=None, prec="fp32", stream=None):
        chains = self._chains(pts, theta)
        n_sys = pts.n_inst * chains
        _need(y, torch.float32, "y", (pts.n_total,))
        _need(phi, torch.float32, "phi", (chains, pts.n_total))
        _need(theta, torch.float64, "theta", (n_sys, pts.n_theta))
        if pi is not None:
            _need(pi, torch.float64, "pi", (n_sys, pts.n_theta))
        mu = prec_ = None
        if prior is not None:
            mu = _need(prior[0], torch.float64, "prior_mu", (pts.n_theta,))
            prec_ = _need(prior[1], torch.float64, "prior_prec", (pts.n_theta,))
        if x_work is None:
            x_work = torch.empty((chains, pts.n_total), dtype=torch.float32, device=y.device)
        H = torch.empty(n_sys, dtype=torch.float64, device=y.device)
        terms = torch.empty((n_sys, 3), dtype=torch.float64, device=y.device)
        status = torch.empty(n_sys, dtype=torch.int32, device=y.device)
        iters = torch.empty_like(status)
        self._check(self.L.kmv_energy(self.h, pts.c, chains, _ptr(y), _ptr(phi), _ptr(theta), _ptr(pi),
                                      _ptr(mu), _ptr(prec_), float(cg_tol), int(cg_maxiter), _ptr(x_work),
                                      _ptr(H), _ptr(terms), _ptr(status), _ptr(iters), self._prec(prec),
                                      _stream(stream)))
        return H, terms, status, iters


def kmv_backward_noalloc(pts: Points, theta, V, G, want_grad_V=True, grad_theta=None, grad_V=None,
                         stream=None):
    """The FP32 adjoint without device allocation or handle (include/kmv.h).

    For callers that cannot allocate device memory (device memory held by
    their own pool or arena, loops that cannot take the synchronisation an
    allocation may imply); its scratch is a fixed 4 MiB array in the library,
    shared by all calls on a device.  Raises KmvError with status KMV_EINVAL
    when the problem does not fit that array.
    """
    L = lib()
    n_sys = theta.shape[0]
    if n_sys % pts.n_inst:
        raise ValueError("theta rows must be n_inst * chains")
    chains = n_sys // pts.n_inst
    _need(theta, torch.float64, "theta", (n_sys, pts.n_theta))
    m = V.shape[-1]
    _need(V, torch.float32, "V", (chains, pts.n_total, m))
    _need(G, torch.float32, "G", V.shape)
    if grad_theta is None:
        grad_theta = torch.empty_like(theta)
    _need(grad_theta, torch.float64, "grad_theta", theta.shape)
    if want_grad_V and grad_V is None:
        grad_V = torch.empty_like(V)
    if grad_V is not None:
        _need(grad_V, torch.float32, "grad_V", V.shape)
    st = L.kmv_backward_noalloc(pts.c, chains, _ptr(theta), _ptr(V), _ptr(G), m, _ptr(grad_theta), _ptr(grad_V),
                                _stream(stream))
    if st != KMV_OK:
        what = "bad argument or scratch limit exceeded" if st == KMV_EINVAL else L.kmv_status_string(st).decode()
        raise KmvError(st, f"kmv_backward_noalloc: {what}")
    return grad_theta, grad_V


_DEFAULT = {}


def accept(H_old, H_new, u, theta_old, theta, status=None, stream=None):
    """The Metropolis test of Algorithm 1 (kmv_accept): theta of rejected systems is
    restored from theta_old in place.  Returns accepted (n_sys int32)."""
    L = lib()
    n_sys, n_theta = theta.shape
    for t, nm in ((H_old, "H_old"), (H_new, "H_new"), (u, "u")):
        _need(t, torch.float64, nm, (n_sys,))
    _need(theta_old, torch.float64, "theta_old", theta.shape)
    _need(theta, torch.float64, "theta", theta.shape)
    if status is not None:
        _need(status, torch.int32, "status", (n_sys,))
    accepted = torch.empty(n_sys, dtype=torch.int32, device=theta.device)
    st = L.kmv_accept(n_sys, n_theta, _ptr(H_old), _ptr(H_new), _ptr(u), _ptr(status), _ptr(theta_old),
                      _ptr(theta), _ptr(accepted), _stream(stream))
    if st != KMV_OK:
        raise KmvError(st, "kmv_accept: " + L.kmv_status_string(st).decode())
    return accepted


def status_merge(src, dst, stream=None):
    """dst = the first failure of src and dst, per system, in place (kmv_status_merge)."""
    L = lib()
    _need(src, torch.int32, "src", dst.shape)
    _need(dst, torch.int32, "dst", src.shape)
    st = L.kmv_status_merge(int(dst.numel()), _ptr(src), _ptr(dst), _stream(stream))
    if st != KMV_OK:
        raise KmvError(st, "kmv_status_merge: " + L.kmv_status_string(st).decode())
    return dst


def default_handle(device: int = 0) -> Kmv:
    if device not in _DEFAULT:
        _DEFAULT[device] = Kmv(device)
    return _DEFAULT[device]

"""torch.autograd.Function around kmv_forward / kmv_backward.

Y = A(theta) V.  Given the upstream gradient G = dLoss/dY, the hand-written
adjoint returns dLoss/dtheta (FP64, one row per system) and dLoss/dV = A G,
recomputing kernel tiles instead of storing them (Sec. 3.2.1 primitive (3)).
"""
from __future__ import annotations

import torch

from .binding import Points, default_handle


class KmvFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, V, pts: Points, prec: str = "fp32", handle=None):
        h = handle if handle is not None else default_handle(V.device.index or 0)
        Y = h.kmv_forward(pts, theta.contiguous(), V.contiguous(), prec=prec)
        ctx.save_for_backward(theta, V)
        ctx.pts, ctx.prec, ctx.h = pts, prec, h
        return Y

    @staticmethod
    def backward(ctx, gY):
        theta, V = ctx.saved_tensors
        want_V = ctx.needs_input_grad[1]
        g_theta, g_V = ctx.h.kmv_backward(ctx.pts, theta.contiguous(), V.contiguous(),
                                          gY.contiguous().to(torch.float32), want_grad_V=want_V,
                                          prec=ctx.prec)
        return (g_theta if ctx.needs_input_grad[0] else None), g_V, None, None, None


def kmv(theta, V, pts: Points, prec: str = "fp32", handle=None):
    """Differentiable Y = A(theta) V."""
    return KmvFunction.apply(theta, V, pts, prec, handle)

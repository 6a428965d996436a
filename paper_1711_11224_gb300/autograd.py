"""Differentiable convolution Y = X (*) H with hand-written backward kernels.

forward:  Y_b = X_b (*) H                           (Property 1, one batched launch)
backward: dX_b = (A_n^h)^T dY_b = M_2p(dY_b (*) H~)  (Property 2, the adjoint kernel)
          dH(j) = sum_b sum_k X_b(k) dY_b(k + j)     (template-gradient kernel)
"""
from __future__ import annotations

import torch

from .plan import Plan

_plans = {}


def _plan(m, p, device):
    key = (tuple(m), tuple(p), device)
    pl = _plans.get(key)
    if pl is None:
        with torch.cuda.device(device):
            pl = Plan(m, p)
        _plans[key] = pl
    return pl


class ConvFn(torch.autograd.Function):
    """Y[B, *(m+2p)] = X[B, *m] (*) H[*(2p+1)], gradients for X and H."""

    @staticmethod
    def forward(ctx, X, H):
        if X.dim() != H.dim() + 1:
            raise ValueError("X must be (B, *m) with the same n as H")
        X = X.contiguous()
        H = H.contiguous()
        p = tuple((q - 1) // 2 for q in H.shape)
        pl = _plan(X.shape[1:], p, X.device)
        pl.set_psf(H)
        Y = pl.forward(X)
        ctx.save_for_backward(X, H)
        ctx.p = p
        return Y

    @staticmethod
    def backward(ctx, dY):
        X, H = ctx.saved_tensors
        dY = dY.contiguous()
        pl = _plan(X.shape[1:], ctx.p, X.device)
        pl.set_psf(H)                      # the template of this graph node, whatever ran since
        dX = pl.adjoint(dY) if ctx.needs_input_grad[0] else None
        dH = pl.grad_psf(X, dY) if ctx.needs_input_grad[1] else None
        return dX, dH


def conv(X, H):
    """Batched full convolution with autograd support (X: (B, *m), H: (2p+1) per axis)."""
    return ConvFn.apply(X, H)

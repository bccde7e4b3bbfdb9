"""Curvature as a differentiable torch function: forward and backward are the
C entry points mecuco_curvature and mecuco_curvature_backward (the neighbour
lists are an input and are treated as constants).  Only X and idx are saved;
the backward recomputes every patch quantity."""
from __future__ import annotations

import torch

from . import api


class MeCuCoCurvature(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X: torch.Tensor, idx: torch.Tensor, k: int, variant: str = "literal",
                precision: str = "fp32"):
        c = api.context(X.device.index or 0)
        kappa = c.mecuco_curvature(X.detach(), k, idx=idx, variant=variant, precision=precision)
        ctx.save_for_backward(X, idx)
        ctx.k, ctx.variant, ctx.precision = k, variant, precision
        return kappa

    @staticmethod
    def backward(ctx, dkappa: torch.Tensor):
        X, idx = ctx.saved_tensors
        c = api.context(X.device.index or 0)
        dX = c.mecuco_curvature_backward(X.detach(), ctx.k, idx, dkappa, variant=ctx.variant)
        return dX.to(X.dtype), None, None, None, None


def curvature(X: torch.Tensor, idx: torch.Tensor, k: int, variant: str = "literal",
              precision: str = "fp32") -> torch.Tensor:
    """Per-point Fast-mode curvature, differentiable with respect to X."""
    return MeCuCoCurvature.apply(X, idx, k, variant, precision)

"""Differentiable F and F* matvecs for PyTorch.

F is linear and real, so for d = F m the vector-Jacobian product is
F^T g = F* g (Section 2.3: F* runs the same five phases with the conjugate
transpose block matvec).  The backward of ``toeplitz_matvec`` is therefore the
library's F* kernel path, and the backward of ``toeplitz_rmatvec`` is F, so
higher-order derivatives work as well.  Both directions use the precisions set
on the operator.
"""
from __future__ import annotations

import torch

from .operator import Operator

__all__ = ["toeplitz_matvec", "toeplitz_rmatvec", "ToeplitzLinear"]


class _Matvec(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m: torch.Tensor, op: Operator) -> torch.Tensor:
        ctx.op = op
        return op.matvec(m.contiguous())

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        return _Rmatvec.apply(g, ctx.op), None


class _Rmatvec(torch.autograd.Function):
    @staticmethod
    def forward(ctx, d: torch.Tensor, op: Operator) -> torch.Tensor:
        ctx.op = op
        return op.rmatvec(d.contiguous())

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        return _Matvec.apply(g, ctx.op), None


def toeplitz_matvec(op: Operator, m: torch.Tensor) -> torch.Tensor:
    """d = F m with autograd support; m is (Nt, Nm) or (K, Nt, Nm)."""
    return _Matvec.apply(m, op)


def toeplitz_rmatvec(op: Operator, d: torch.Tensor) -> torch.Tensor:
    """m = F* d with autograd support; d is (Nt, Nd) or (K, Nt, Nd)."""
    return _Rmatvec.apply(d, op)


class ToeplitzLinear(torch.nn.Module):
    """``torch.nn`` wrapper: forward(m) = F m, gradients through F*."""

    def __init__(self, op: Operator):
        super().__init__()
        self.op = op

    def forward(self, m: torch.Tensor) -> torch.Tensor:
        return toeplitz_matvec(self.op, m)

"""torch.autograd binding of the forward operator with hand-written gradients.

``mpi_forward_autograd(c, beta, model, grid, r, v)`` returns s = A(c; beta)
([n_ch, T]) and differentiates with respect to the concentration image c and
the particle parameter beta = 1/(mu0 H_sat):

    dL/dc    = A^T g                      (mpi_adjoint)
    dL/dbeta = <g, dA(c; beta)/dbeta>     (mpi_dbeta, FP64 reduction)

with g = dL/ds.  Both are library kernels; this module only routes tensors.
"""
from __future__ import annotations

import torch

from . import api


def _model_with_beta(model, beta: float) -> dict:
    m = dict(model) if isinstance(model, dict) else {k: getattr(model, k) for k in ("beta", "G", "p")}
    m["beta"] = float(beta)
    return m


class MPIForward(torch.autograd.Function):
    """s = A(c; beta) with backward through A^T and the beta-derivative kernel."""

    @staticmethod
    def forward(ctx, c, beta, model, grid, r, v):
        m = _model_with_beta(model, beta.item() if isinstance(beta, torch.Tensor) else beta)
        c_ = c.detach().contiguous()
        s = api.mpi_forward(m, grid, r, v, c_)
        ctx.save_for_backward(c_)
        ctx.m, ctx.grid, ctx.r, ctx.v = m, grid, r, v
        ctx.beta_is_tensor = isinstance(beta, torch.Tensor)
        ctx.beta_dtype = beta.dtype if ctx.beta_is_tensor else None
        return s

    @staticmethod
    def backward(ctx, g):
        (c,) = ctx.saved_tensors
        g = g.contiguous().to(c.dtype)
        grad_c = grad_beta = None
        if ctx.needs_input_grad[0]:
            grad_c = api.mpi_adjoint(ctx.m, ctx.grid, ctx.r, ctx.v, g)
        if ctx.beta_is_tensor and ctx.needs_input_grad[1]:
            grad_beta = api.mpi_dbeta(ctx.m, ctx.grid, ctx.r, ctx.v, c, g).to(ctx.beta_dtype)
        return grad_c, grad_beta, None, None, None, None


def mpi_forward_autograd(c: torch.Tensor, beta, model, grid, r: torch.Tensor,
                         v: torch.Tensor) -> torch.Tensor:
    """Differentiable forward operator; ``beta`` may be a float or a 0-d tensor."""
    return MPIForward.apply(c, beta, model, grid, r, v)

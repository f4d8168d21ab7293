"""torch.autograd Functions over the differentiation entry points.

Both compute the gradient in the same library call as the loss (one pass of
the forward with its checkpoints and one reverse sweep) and keep it for the
backward, which only scales it by the incoming gradient.

    loss = SubspaceLoss.apply(P_hat, B, ctx, precision)
    loss = NlssLoss.apply(P_hat, S, ctx, precision)
    loss = UnrolledPCG.apply(P, op, b, T, nu, omega, precision)
"""
from __future__ import annotations

import torch

from . import _lib as L
from . import api


class SubspaceLoss(torch.autograd.Function):
    """||(I - Q Q^T) B||_F^2, Q = qf(P_hat) (Sec. 3); differentiable in P_hat."""

    @staticmethod
    def forward(fctx, P_hat, B, ctx, precision=L.NLSP_FP64):
        loss, grad = api.subspace_loss(ctx, P_hat.detach(), B.detach(), precision, grad=P_hat.requires_grad)
        fctx.save_for_backward(grad if grad is not None else torch.zeros(0))
        return torch.tensor(loss, dtype=torch.float64, device=P_hat.device)

    @staticmethod
    def backward(fctx, g):
        (grad,) = fctx.saved_tensors
        return g * grad, None, None, None


class NlssLoss(torch.autograd.Function):
    """(1/k) sum_l (1 - ||Q_{1:l}^T S||^2 / ||S||^2), Q = qf(P_hat) (Sec. 3,
    nested subspace loss); differentiable in P_hat."""

    @staticmethod
    def forward(fctx, P_hat, S, ctx, precision=L.NLSP_FP64):
        loss, grad = api.nlss_loss(ctx, P_hat.detach(), S.detach(), precision, grad=P_hat.requires_grad)
        fctx.save_for_backward(grad if grad is not None else torch.zeros(0))
        return torch.tensor(loss, dtype=torch.float64, device=P_hat.device)

    @staticmethod
    def backward(fctx, g):
        (grad,) = fctx.saved_tensors
        return g * grad, None, None, None


class UnrolledPCG(torch.autograd.Function):
    """||r_T|| after T PCG steps with the two-level preconditioner from P."""

    @staticmethod
    def forward(fctx, P, op, b, T=10, nu=2, omega=2.0 / 3.0, precision=L.NLSP_FP64):
        loss, grad = api.unrolled_pcg(op, P.detach(), b.detach(), T, nu, omega, precision, grad=P.requires_grad)
        fctx.save_for_backward(grad if grad is not None else torch.zeros(0))
        return torch.tensor(loss, dtype=torch.float64, device=P.device)

    @staticmethod
    def backward(fctx, g):
        (grad,) = fctx.saved_tensors
        return g * grad, None, None, None, None, None, None

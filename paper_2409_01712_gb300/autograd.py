"""torch.autograd.Function over the held-out loss of KRR.

``held_out_loss(log_gamma, log_lambda, G, Y, T, Yt)`` fits KRR on (G, Y) with
gamma = exp(log_gamma), lambda = exp(log_lambda) through libkrr.so (Build,
Factor, Solve), predicts T and returns the held-out mean squared error.  Its
backward pass returns d loss / d log gamma and d loss / d log lambda from
krr_grad_hyper, the hand-written adjoint that reuses the Cholesky factor.
The adjoint runs inside forward, while the factor exists; backward only
scales the stored gradient.  Only argument marshalling happens here.
"""
from __future__ import annotations

import math

import torch

from .krr import KRR


class HeldOutLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_gamma, log_lambda, g, y, t, yt, tile=1024):
        gamma = math.exp(float(log_gamma))
        lam = math.exp(float(log_lambda))
        with KRR(tile=tile, mode="mixed") as model:
            model.build_kernel(g, gamma)
            model.factor(lam)
            a, _ = model.solve(y)
            loss, dlog_gamma, dlog_lambda = model.grad_hyper(t, yt, a)
        ctx.grads = (dlog_gamma, dlog_lambda)
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        dg, dl = ctx.grads
        return (grad_out * dg, grad_out * dl, None, None, None, None, None)


def held_out_loss(log_gamma, log_lambda, g, y, t, yt, tile: int = 1024):
    """Held-out MSE as a differentiable function of (log gamma, log lambda)."""
    return HeldOutLoss.apply(log_gamma, log_lambda, g, y, t, yt, tile)

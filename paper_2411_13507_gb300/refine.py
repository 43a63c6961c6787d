"""Differentiable trajectory refinement: torch.autograd.Function over plan_refine.

loss_s = w_snap * J_snap + mu * sum phi_delta(margin) for each degree-p segment
(reach margins on the hodograph control points, free margins of the interior
control points, relaxed log-barrier, exact snap energy); forward and backward
both run the CUDA kernels behind plan_refine.  All tensors are float32 on the
GPU: P [S][p+1][m], T [S], A [S][rmax][m], b [S][rmax], nrows int32 [S].
"""
from __future__ import annotations

from typing import Sequence

import torch

from . import plan as _plan


class Refiner:
    """A libplan context configured for refinement segments of one model."""

    def __init__(self, m: int = 3, gamma: int = 3, degree: int = 7, bounds: Sequence[float] = (3.0, 6.0, 30.0),
                 w_snap: float = 1.0, mu: float = 1.0, delta: float = 0.1, stream=None):
        self.planner = _plan.Planner(m, gamma, degree, bounds, arith="f32", input="f32", stream=stream)
        self.weights = (float(w_snap), float(mu), float(delta))

    def forward(self, P, T, A, b, nrows):
        loss = torch.empty(P.shape[0], dtype=torch.float32, device=P.device)
        self.planner.refine_async(P, T, A, b, nrows, self.weights, loss=loss)
        return loss

    def backward(self, P, T, A, b, nrows, grad_loss):
        dP = torch.empty_like(P)
        dT = torch.empty_like(T)
        self.planner.refine_async(P, T, A, b, nrows, self.weights, grad_loss=grad_loss.contiguous(),
                                  dP=dP, dT=dT)
        return dP, dT

    def check(self):
        st = self.planner.wait()
        if st != _plan.PLAN_OK:
            raise _plan.PlanError(st, "refine")


class RefineLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, P, T, A, b, nrows, refiner: Refiner):
        P, T, A, b, nrows = (x.contiguous() for x in (P, T, A, b, nrows))
        ctx.save_for_backward(P, T, A, b, nrows)
        ctx.refiner = refiner
        return refiner.forward(P, T, A, b, nrows)

    @staticmethod
    def backward(ctx, grad_loss):
        P, T, A, b, nrows = ctx.saved_tensors
        dP, dT = ctx.refiner.backward(P, T, A, b, nrows, grad_loss.float())
        return dP, dT, None, None, None, None


def refine_loss(P, T, A, b, nrows, refiner: Refiner):
    """Per-segment loss with a hand-written CUDA backward (autograd-aware)."""
    return RefineLoss.apply(P, T, A, b, nrows, refiner)

"""torch.autograd.Function wrappers over the amgh C ABI (differentiation pattern).

StateSolve:   y = K u = A^-1 M_yu u (Sec. 2, Eq. solutionopdef); its backward
              is the adjoint K^T ybar = M_yu^T A^-T ybar, one more AMG-CG solve.
ReducedCost:  J(u) = 1/2 (K u - y_d)^T M_y (K u - y_d) + beta/2 u^T M_u u
              (Eq. functional with the state eliminated); its backward is the
              adjoint gradient M_yu^T A^-T M_y (y - y_d) + beta M_u u, which
              equals H u - b with H and b of Eq. firstorderpractice.
Both run entirely in the CUDA library; torch only carries the tensors.
"""
from __future__ import annotations

import torch


class StateSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, prob):
        ctx.prob = prob
        return prob.state_only(u.contiguous())

    @staticmethod
    def backward(ctx, ybar):
        return ctx.prob.state_adjoint(ybar.contiguous()), None


class ReducedCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, prob):
        u = u.contiguous()
        y, J = prob.state_solve(u)
        ctx.prob = prob
        ctx.save_for_backward(u, y)
        return torch.tensor(J, dtype=u.dtype, device=u.device)

    @staticmethod
    def backward(ctx, gJ):
        u, y = ctx.saved_tensors
        g = ctx.prob.gradient(u, y)
        return gJ * g, None


def state_solve(u, prob):
    """Differentiable y = A^-1 M_yu u."""
    return StateSolve.apply(u, prob)


def reduced_cost(u, prob):
    """Differentiable reduced cost J(u) with the adjoint-solve gradient."""
    return ReducedCost.apply(u, prob)

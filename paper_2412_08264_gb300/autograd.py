"""The lower-level solve as a torch.autograd.Function with a hand-written backward.

forward(theta)      x^_k(theta) for every pair (bl_lower_solve, warm-started), returned packed.
backward(grad_x)    the implicit-function adjoint (eqs. (2.4)-(2.7)): for each pair solve
                    H_k w_k = grad_x_k with the recycled CG of the engine (its recycle space carries
                    over between calls), then dL/dtheta = sum_k J_k w_k with
                    J_k = -(D^2_{theta x} Phi_k)^T (bl_hypergrad).
The upstream gradient may be any function of x^ (not only 1/2 ||x^ - x*||^2); the recycle state can be
checkpointed with Engine.state_dict / load_state_dict between outer steps.
"""
from __future__ import annotations

import torch

from .outer import Engine


class LowerLevelSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, engine: Engine):
        th = theta.detach().to(torch.float64).contiguous()
        x, _ = engine.lower(th)
        engine.xhat = x
        ctx.engine = engine
        return x.clone()

    @staticmethod
    def backward(ctx, grad_x: torch.Tensor):
        engine: Engine = ctx.engine
        g = grad_x.detach().to(engine.P.dtype).contiguous()
        # the point (theta, x^) of the forward solve is still the library's current point
        mean, per, _, _ = engine.hypergrad_at_point(g=g, per_pair=True)
        return per.sum(0), None


def lower_level_solve(theta: torch.Tensor, engine: Engine) -> torch.Tensor:
    return LowerLevelSolve.apply(theta, engine)

"""torch.autograd.Function over the C ABI: J(gamma) forward, dJ/dgamma from the exact discrete
adjoint (Sec. 2.4) in backward.

The forward stores whatever the adjoint needs on the device (binomial checkpoints and the tape
of the last segment); the backward runs the reverse sweep.  A solver holds one forward run at a
time, so when the solver has run forward again since (or its adjoint was already taken), the
backward first repeats this output's forward from the saved design.  Every operation runs in the
CUDA library; this module only hands tensors across.
"""
from __future__ import annotations

import torch

from . import lks as _lks


class LKSObjective(torch.autograd.Function):
    """J = objective of Sec. 2.5 after Alg. 1 on design gamma; grad = dJ/dgamma."""

    @staticmethod
    def forward(ctx, gamma: torch.Tensor, solver: "_lks.Solver") -> torch.Tensor:
        g = gamma.detach().to(torch.float64).contiguous().clone()
        solver.set_design(g)
        J = solver.forward()
        ctx.solver = solver
        ctx.generation = solver.generation
        ctx.gamma = g
        ctx.meta = (gamma.shape, gamma.device)
        return torch.tensor(J, dtype=torch.float64, device=gamma.device)

    @staticmethod
    def backward(ctx, grad_J: torch.Tensor):
        shape, device = ctx.meta
        solver = ctx.solver
        if solver.generation != ctx.generation or not solver.adjoint_ready:
            solver.set_design(ctx.gamma)
            solver.forward()
            ctx.generation = solver.generation
        g = torch.empty(shape, dtype=torch.float64, device=device)
        solver.adjoint(out=g)
        return grad_J.to(torch.float64) * g, None


def objective(gamma: torch.Tensor, solver: "_lks.Solver") -> torch.Tensor:
    """J(gamma) as a differentiable scalar (float64)."""
    return LKSObjective.apply(gamma, solver)

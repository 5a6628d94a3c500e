"""Differentiable compact-multigrid solve of the diffusion problem.

``diffusion_solve(k, g, cfg)`` returns the decoded finest-level solution u of
-div(k grad u) = g (A(k) u = h^d g, zero Dirichlet) computed by compact FMG on
the GPU, as a ``torch.autograd.Function``:

* forward: one compact FMG solve; the solver's compact state u~ (a few bits per
  DoF) is kept as the checkpoint, not the decoded u;
* backward: the adjoint system A lam = dJ/du (A is symmetric) is solved by a
  second compact FMG solve; u is decoded again from the checkpoint; the
  hand-written gradient kernel (cmg_gradient) forms dJ/dk and dJ/dg = h^d lam.

Marshalling only: every step runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import cmg


class DiffusionSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, k: torch.Tensor, g: torch.Tensor, cfg) -> torch.Tensor:
        # k: binary32 nodal coefficient, (2^L + 1)^d with the boundary; g: float64
        # nodal right-hand side on the interior, (2^L - 1)^d
        k = k.detach().contiguous()
        g = g.detach().contiguous()
        solver = cmg.Solver(cfg)
        solver.set_coefficient(k.reshape(-1))
        solver.set_rhs_nodal(g.reshape(-1))
        solver.fmg_solve()
        u = solver.decode_solution().reshape(g.shape)
        ctx.solver = solver  # the compact checkpoint
        ctx.cfg = cfg
        ctx.kshape = k.shape
        ctx.save_for_backward(k)
        return u

    @staticmethod
    def backward(ctx, grad_u: torch.Tensor):
        (k,) = ctx.saved_tensors
        cfg = ctx.cfg
        d, L = cfg.dim, cfg.L_max
        # adjoint: A lam = grad_u, posed as A lam = h^d g' with g' = 2^(d L) grad_u (exact)
        rhs = (grad_u.detach().to(torch.float64) * float(2 ** (d * L))).contiguous().reshape(-1)
        adj = cmg.Solver(cfg)
        adj.set_coefficient(k.reshape(-1))
        adj.set_rhs_nodal(rhs)
        adj.fmg_solve()
        lam = adj.decode_solution().reshape(-1)
        u = ctx.solver.decode_solution().reshape(-1)  # decoded again from the compact checkpoint
        dk, dg = ctx.solver.gradient(u, lam, want_dg=True)
        return dk.reshape(ctx.kshape).to(k.dtype), dg.reshape(grad_u.shape), None


def diffusion_solve(k: torch.Tensor, g: torch.Tensor, cfg) -> torch.Tensor:
    """u = A(k)^-1 h^d g by compact FMG, differentiable in k and g."""
    return DiffusionSolve.apply(k, g, cfg)

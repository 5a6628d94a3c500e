"""Differentiable compact-multigrid solve of the diffusion problem.

``diffusion_solve(k, g, cfg)`` returns the decoded finest-level solution u of
-div(k grad u) = g (A(k) u = h^d g, zero Dirichlet) computed by compact FMG on
the GPU, as a ``torch.autograd.Function``:

* forward: one compact FMG solve; only the compact sections u~_1..u~_L (a few
  bits per DoF, cmg_state_save) are kept as the checkpoint, in host memory, and
  the solver context with its residual, correction and temporaries is closed
  before forward returns;
* backward: the adjoint system A lam = dJ/du (A is symmetric) is solved by a
  second compact FMG solve; a context is rebuilt from the checkpoint
  (cmg_state_load) and u is decoded from it again; the hand-written gradient
  kernel (cmg_gradient) forms dJ/dk and dJ/dg = h^d lam.

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
        ctx.checkpoint = solver.state_save()  # the compact u~ sections only
        solver.close()
        ctx.cfg = cfg
        ctx.kshape = k.shape
        ctx.save_for_backward(k)
        return u

    @staticmethod
    def backward(ctx, grad_u: torch.Tensor):
        (k,) = ctx.saved_tensors
        cfg = ctx.cfg
        d, L = cfg.dim, cfg.L_max
        # adjoint: A lam = grad_u, posed as A lam = h^d 2^(d L) grad_u (the library
        # applies the power-of-two scale)
        rhs = grad_u.detach().to(torch.float64).contiguous().reshape(-1)
        adj = cmg.Solver(cfg)
        adj.set_coefficient(k.reshape(-1))
        adj.set_rhs_nodal(rhs, d * L)
        adj.fmg_solve()
        lam = adj.decode_solution().reshape(-1)
        adj.close()
        fwd = cmg.Solver(cfg)  # rebuilt from the compact checkpoint
        fwd.set_coefficient(k.reshape(-1))
        fwd.state_load(ctx.checkpoint)
        u = fwd.decode_solution().reshape(-1)
        dk, dg = fwd.gradient(u, lam, want_dg=True)
        fwd.close()
        ctx.checkpoint = None
        return dk.reshape(ctx.kshape).to(k.dtype), dg.reshape(grad_u.shape), None


def diffusion_solve(k: torch.Tensor, g: torch.Tensor, cfg) -> torch.Tensor:
    """u = A(k)^-1 h^d g by compact FMG, differentiable in k and g."""
    return DiffusionSolve.apply(k, g, cfg)

"""Differentiable LS solve: u(m) for plane waves, with the adjoint solve as backward.

The scattered field u of the plane wave u_I = exp(i omega d.p) solves
(I + omega^2 K M) u = -omega^2 K (m u_I) (Eq. LS_d).  For a real loss L(u),
with g = dL/dRe u + i dL/dIm u (torch's gradient of a complex tensor),
dL/dm = Re(g^H du/dm) and du/dm_x = -omega^2 A^{-1} K e_x (u + u_I)_x, so
dL/dm = Re((-omega^2 K mu) . (u + u_I)) with A^T mu = conj(g)
(A^T = I + omega^2 M K, K symmetric).  Forward and backward both run in the
CUDA library: lss_set_medium / lss_factor / lss_plane_wave_rhs / lss_solve,
then lss_adjoint_solve (transposed preconditioner, reused factors) and
lss_medium_gradient.
"""
from __future__ import annotations

import numpy as np
import torch

from .solver import GmresOptions, LSSolver


class LSSolve(torch.autograd.Function):
    """u = LSSolve.apply(m, solver, dirs, opts, memory_cap): scattered fields,
    R x n x n.  The forward fields are kept on the device for the backward
    unless they take more than memory_cap bytes (None: a quarter of the
    device memory free at the forward); then the backward recomputes them by
    a second forward solve.  The backward refactors for this medium when the
    solver has been given another one since the forward."""

    @staticmethod
    def forward(ctx, m: torch.Tensor, solver: LSSolver, dirs, opts: GmresOptions | None = None,
                memory_cap: int | None = None):
        solver.set_medium(m.detach())
        solver.factor()
        g = solver.plane_wave_rhs(dirs)
        u, _ = solver.solve(g, opts)
        ctx.solver, ctx.dirs, ctx.opts = solver, np.asarray(dirs, dtype=np.float64).reshape(-1, 2), opts
        ctx.version = solver.medium_version
        cap = memory_cap if memory_cap is not None else torch.cuda.mem_get_info(u.device)[0] // 4
        ctx.recompute = u.numel() * u.element_size() > cap
        ctx.save_for_backward(m.detach(), u if not ctx.recompute else torch.empty(0, device=u.device))
        return u

    @staticmethod
    def backward(ctx, grad_u: torch.Tensor):
        m, u = ctx.saved_tensors
        solver = ctx.solver
        if solver.medium_version != ctx.version:   # another medium was set since the forward
            solver.set_medium(m)
            solver.factor()
            ctx.version = solver.medium_version
        if ctx.recompute:
            u, _ = solver.solve(solver.plane_wave_rhs(ctx.dirs), ctx.opts)
        mu, _ = solver.adjoint_solve(torch.conj(grad_u).resolve_conj().contiguous(), ctx.opts)
        grad_m = solver.medium_gradient(mu, u, ctx.dirs)
        return grad_m, None, None, None, None


def ls_solve(m: torch.Tensor, solver: LSSolver, dirs, opts: GmresOptions | None = None,
             memory_cap: int | None = None) -> torch.Tensor:
    """Differentiable scattered fields of plane waves with directions `dirs` in medium m
    (forward fields recomputed in the backward when they exceed memory_cap bytes)."""
    return LSSolve.apply(m, solver, dirs, opts, memory_cap)

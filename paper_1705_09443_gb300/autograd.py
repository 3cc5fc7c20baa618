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
    """u = LSSolve.apply(m, solver, dirs, opts): scattered fields, R x n x n."""

    @staticmethod
    def forward(ctx, m: torch.Tensor, solver: LSSolver, dirs, opts: GmresOptions | None = None):
        solver.set_medium(m.detach())
        solver.factor()
        g = solver.plane_wave_rhs(dirs)
        u, _ = solver.solve(g, opts)
        ctx.solver, ctx.dirs, ctx.opts = solver, np.asarray(dirs, dtype=np.float64).reshape(-1, 2), opts
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, grad_u: torch.Tensor):
        (u,) = ctx.saved_tensors
        solver = ctx.solver
        mu, _ = solver.adjoint_solve(torch.conj(grad_u).resolve_conj().contiguous(), ctx.opts)
        grad_m = solver.medium_gradient(mu, u, ctx.dirs)
        return grad_m, None, None, None


def ls_solve(m: torch.Tensor, solver: LSSolver, dirs, opts: GmresOptions | None = None) -> torch.Tensor:
    """Differentiable scattered fields of plane waves with directions `dirs` in medium m."""
    return LSSolve.apply(m, solver, dirs, opts)

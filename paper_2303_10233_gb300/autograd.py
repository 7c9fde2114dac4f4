"""torch.autograd.Function around the GPU solver with a hand-written adjoint.

Forward: u, p = solve K(nu) [u; p] = b(f, nu) (eth_solve).
Backward: for upstream gradients (g_u, g_p) the adjoint system
K(nu)^T [l_u; l_p] = [g_u; g_p] is solved on the GPU (eth_solve_adjoint:
the same MINRES for symmetric Stokes, the two-stage PCD GMRES on
[F^T B^T; B 0] with PCD built on F1^T for Oseen) and

    dL/df_nodal = M_v D_I l_u,      dL/dnu = -(D_I l_u)^T A u

are formed by eth_adjoint_gradients.  The forward pressure is canonical (its
constant Q1 and P0 components removed), so the gradient reaching the adjoint
system is the projected g_p; eth_solve_adjoint performs that projection itself
and reports a removed component as ETH_EINCONSISTENT, which is expected here.
Only argument marshalling happens in this module.
"""
from __future__ import annotations

import torch

from . import eth


class EthSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f_nodal, nu, grid, ubc, wind, opts):
        nu_v = float(nu)
        grid.set_coefficients(nu_v, wind)
        grid.set_rhs(f_nodal.detach().contiguous(), ubc)
        u, p, st = grid.solve(**opts)
        if st["status"] not in (0,):
            raise eth.EthError(st["status"], f"forward solve did not converge: {st}")
        ctx.grid, ctx.opts, ctx.nu, ctx.wind, ctx.ubc = grid, opts, nu_v, wind, ubc
        ctx.nu_is_tensor = torch.is_tensor(nu)
        ctx.save_for_backward(u)
        return u, p

    @staticmethod
    def backward(ctx, gu, gp):
        grid = ctx.grid
        (u,) = ctx.saved_tensors
        grid.set_coefficients(ctx.nu, ctx.wind)
        gu = torch.zeros_like(u) if gu is None else gu.contiguous()
        if gp is None:
            gp = torch.zeros(grid.n1 + grid.n0, dtype=torch.float64, device=u.device)
        lu, lp, st = grid.solve_adjoint(gu, gp.contiguous(), **ctx.opts)
        if st["status"] not in (0, 6):   # 6: the pressure gradient's null-space part was projected out
            raise eth.EthError(st["status"], f"adjoint solve did not converge: {st}")
        gf, gnu = grid.adjoint_gradients(lu, u)
        gnu_t = torch.tensor(gnu, dtype=torch.float64, device=u.device) if ctx.nu_is_tensor else None
        return gf, gnu_t, None, None, None, None


def solve(f_nodal, nu, grid, ubc, wind=None, **opts):
    """Differentiable solve: returns (u, p); gradients flow to f_nodal and nu."""
    return EthSolve.apply(f_nodal, nu, grid, ubc, wind, opts)

"""Adjoint gradients of J = ||u - u_t||^2 (test infrastructure only).

The discrete state solves K(nu) x = b(f, nu) (Dirichlet eliminated, see
``problem``).  With the adjoint K^T lam = dJ/dx = [2(u - u_t); 0]:

    dJ/df_nodal = M_v D_I lam_u            (b_u = D_I M_v f + ...)
    dJ/dnu      = -(D_I lam_u)^T A u       (dK/dnu and db/dnu act through nu*A)

where u is the full velocity (boundary values included) and M_v, A are the
per-component Q2 mass and Laplacian.  Both K and K^T have the pressure null
space span{e1, e0}; the adjoint right-hand side has a zero pressure part, so
the adjoint system is consistent and lam_u is unique.
"""
from __future__ import annotations

import numpy as np

from . import direct, problem, fem


def objective(sys, x, u_target):
    u = x[: sys.g.nu]
    d = u - u_target
    return float(np.dot(d, d))


def solve_state(sys, f_nodal, ubc):
    b = sys.rhs(f_nodal, ubc)
    x, _ = direct.solve(sys, b)
    return x, b


def gradients(sys, f_nodal, ubc, u_target):
    """(J, grad_f (2*nv), grad_nu, lam) by the exact (direct) adjoint."""
    g = sys.g
    x, _ = solve_state(sys, f_nodal, ubc)
    u = x[: g.nu]
    rhs = np.concatenate([2.0 * (u - u_target), np.zeros(g.np_)])
    lam, _ = direct.solve_transpose(sys, rhs)
    lu = sys.DI @ lam[: g.nu]
    grad_f = np.concatenate([sys.Mv @ lu[: g.nv], sys.Mv @ lu[g.nv:]])
    Au = np.concatenate([sys.A @ u[: g.nv], sys.A @ u[g.nv:]])
    grad_nu = -float(np.dot(lu, Au))
    return objective(sys, x, u_target), grad_f, grad_nu, lam


def fd_objective(g, nu, wind, f_nodal, ubc, u_target):
    """J evaluated by a fresh assembly + direct solve (for finite differences)."""
    sys = problem.System(g, nu, wind)
    x, _ = solve_state(sys, f_nodal, ubc)
    return objective(sys, x, u_target)

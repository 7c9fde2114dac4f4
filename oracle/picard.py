"""Picard (fixed-point) linearisation of the steady Navier-Stokes problem (test infrastructure only).

Sec. 3: the Oseen systems the method solves arise from the Picard iteration for
steady incompressible Navier-Stokes flow.  Given the velocity iterate u_k, the next
iterate solves the Oseen problem whose convection uses the wind w = u_k:

    [ nu A + N(u_k)   B^T ] [u_{k+1}]   [f]
    [ B               0   ] [p_{k+1}] = [g],

with the Dirichlet data of the problem and, from u_0 = 0, a first step that is the
Stokes problem (N(0) = 0).  Every step here is an exact (bordered direct) solve of
``problem.System`` with the current wind.  The nonlinear residual of an iterate
(u, p) is the relative residual of the Oseen system assembled with wind u itself,
||b(u) - K(u) [u; p]|| / ||b(u)||; it vanishes at a discrete Navier-Stokes solution.
"""
from __future__ import annotations

import numpy as np

from . import direct, fem, problem


def nonlinear_residual(g: fem.Grid, nu, f_nodal, ubc, x):
    """||b(u) - K(u) x|| / ||b(u)|| with K(u), b(u) the Oseen system linearised at u = x[:nu]."""
    s = problem.System(g, nu, np.array(x[: g.nu], copy=True))
    b = s.rhs(f_nodal, ubc)
    return np.linalg.norm(b - s.K @ x) / np.linalg.norm(b)


def picard(g: fem.Grid, nu, f_nodal, ubc, steps):
    """Iterates x_1..x_steps (canonical pressure) and their nonlinear residuals; x_1 is the
    Stokes solution (zero wind)."""
    xs, res = [], []
    wind = np.zeros(g.nu)
    for _ in range(steps):
        s = problem.System(g, nu, wind)
        b = s.rhs(f_nodal, ubc)
        x, _ = direct.solve(s, b)
        x = s.canonical(x)
        xs.append(x)
        res.append(nonlinear_residual(g, nu, f_nodal, ubc, x))
        wind = np.array(x[: g.nu], copy=True)
    return xs, res

"""Saddle-point systems with Dirichlet velocity eliminated (test infrastructure only).

Stokes (Sec. 2, Eq. saddle_point) and Oseen (Sec. 3, Eq. oseen-system):

    K = [ F   B^T ]      F = nu*A (Stokes) or nu*A + N(w) (Oseen), per component,
        [ B   0   ]      B = [B1; B0] from b(u, p) = -int p div u.

Dirichlet treatment: the full Q2 lattice is kept.  Boundary velocity rows of K
are identity rows and boundary velocity columns are zero in every other row,
so K stays symmetric for Stokes.  The boundary values move to the right-hand
side: f_I = (M_v f_nodal - F u_b)_I, g = -B u_b.  The body force enters through
the consistent Q2 mass matrix.

For enclosed flow the pressure null space of K is spanned by e1 = [0; 1_{n_k}; 0]
and e0 = [0; 0; 1_{n_0}] (constant Q1 and constant P0 pressures separately,
Sec. 3 Test problem 4); k = e1 - e0 (Eq. pressure_null_vector).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem


class System:
    """Assembled FP64 Stokes/Oseen system on a uniform grid."""

    def __init__(self, g: fem.Grid, nu=1.0, wind=None):
        self.g = g
        self.nu = float(nu)
        self.wind = None if wind is None else np.asarray(wind, dtype=np.float64)
        self.A = fem.stiffness_q2(g)
        self.Mv = fem.mass_q2(g)
        self.N = fem.convection_q2(g, self.wind) if self.wind is not None else None
        Fs = self.nu * self.A
        if self.N is not None:
            Fs = Fs + self.N
        self.Fs = Fs.tocsr()                                   # scalar F, no BCs
        self.B1, self.B0 = fem.divergence(g)
        self.B = sp.vstack([self.B1, self.B0]).tocsr()
        self.MQ, self.Qk, self.R, self.Q0 = fem.pressure_mass(g)
        self.intr = ~g.bnd                                     # interior Q2 nodes
        di = self.intr.astype(np.float64)
        self.DIs = sp.diags(di)
        self.DBs = sp.diags(1.0 - di)
        self.DI = sp.block_diag([self.DIs, self.DIs]).tocsr()
        self.DB = sp.block_diag([self.DBs, self.DBs]).tocsr()
        FsI = (self.DIs @ self.Fs @ self.DIs + self.DBs).tocsr()
        AsI = (self.DIs @ (self.nu * self.A) @ self.DIs + self.DBs).tocsr()
        self.F = sp.block_diag([FsI, FsI]).tocsr()             # velocity block of K
        self.Anu = sp.block_diag([AsI, AsI]).tocsr()           # nu*A with BC rows
        self.BI = (self.B @ self.DI).tocsr()
        self.B1I = (self.B1 @ self.DI).tocsr()
        self.B0I = (self.B0 @ self.DI).tocsr()
        self.K = sp.bmat([[self.F, self.BI.T], [self.BI, None]]).tocsr()
        self.K1 = sp.bmat([[self.F, self.B1I.T], [self.B1I, None]]).tocsr()  # reduced system
        nu_, n1, n0 = g.nu, g.n1, g.n0
        self.e1 = np.concatenate([np.zeros(nu_), np.ones(n1), np.zeros(n0)])
        self.e0 = np.concatenate([np.zeros(nu_), np.zeros(n1), np.ones(n0)])
        self.k = fem.null_vector_k(g)

    # ---------------------------------------------------------------- RHS
    def rhs(self, f_nodal, ubc):
        """b = [D_I (M_v f - F u_b) + D_B u_b; -B D_B u_b]."""
        g = self.g
        f_nodal = np.asarray(f_nodal, dtype=np.float64)
        ub = self.DB @ np.asarray(ubc, dtype=np.float64)
        Mf = np.concatenate([self.Mv @ f_nodal[: g.nv], self.Mv @ f_nodal[g.nv:]])
        Fub = np.concatenate([self.Fs @ ub[: g.nv], self.Fs @ ub[g.nv:]])
        bu = self.DI @ (Mf - Fub) + ub
        bp = -(self.B @ ub)
        return np.concatenate([bu, bp])

    # ---------------------------------------------------------------- helpers
    def split(self, x):
        g = self.g
        return x[: g.nu], x[g.nu: g.nu + g.n1], x[g.nu + g.n1:]

    def canonical(self, x):
        """Remove the e1 and e0 components (Euclidean): sum p1 = sum p0 = 0."""
        g = self.g
        y = np.array(x, dtype=np.float64, copy=True)
        y[g.nu: g.nu + g.n1] -= y[g.nu: g.nu + g.n1].mean()
        y[g.nu + g.n1:] -= y[g.nu + g.n1:].mean()
        return y

    def project_rhs(self, b):
        """Make b consistent: remove its components along e1 and e0."""
        return self.canonical(b)

    def residual(self, x, b):
        return b - self.K @ x

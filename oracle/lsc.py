"""Least-squares commutator (LSC) preconditioner for the two-field pressure
(test infrastructure only).

Sec. 3.2, Eq. lsc-definition: the Schur complement B F^{-1} B^T of the Oseen system
is approximated by

    M_S = (B H^{-1} B^T) (B M^{-1} F H^{-1} B^T)^{-1} (B M^{-1} B^T),

built from B = [B1; B0] (the full Q1 + P0 frame), the velocity block F and a
diagonal velocity mass M; H = D^{-1/2} M D^{-1/2} with a diagonal D that adjusts the
rows of tangential velocity unknowns next to Dirichlet walls.  Eq. nse-precon-lsc
uses it in the block upper-triangular preconditioner

    M_3 = [ F  B^T ; 0  -M_S ].

Readings (the paper defers the details to the Elman-Silvester-Wathen book):
* M is the diagonal of the consistent Q2 velocity mass matrix (as in the PCD's Ap).
* D is diagonal with entry ``omega`` for the tangential velocity component at the
  interior Q2 nodes next to a wall (u_x next to the bottom and top walls, u_y next
  to the left and right walls) and 1 elsewhere; omega = 1 gives H = M, plain LSC.
* For enclosed flow B^T annihilates e1 and e0 (constant pressure in either field), so
  both B X B^T products are singular on span{e1, e0}; their solves return the
  solution orthogonal to e1 and e0 (Euclidean) after removing the right-hand side's
  components along them, as for the other singular pressure solves here.

M_S^{-1} r = (B M^{-1} B^T)^+ (B M^{-1} F H^{-1} B^T) (B H^{-1} B^T)^+ r.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import krylov, problem


def tangential_weights(g, omega):
    """Diagonal of D over the velocity unknowns [u_x; u_y]."""
    N = g.N
    j, i = np.divmod(np.arange(g.nv), N)
    dx = np.ones(g.nv)
    dy = np.ones(g.nv)
    interior = ~g.bnd
    next_to_bottom_top = interior & ((j == 1) | (j == N - 2))
    next_to_sides = interior & ((i == 1) | (i == N - 2))
    dx[next_to_bottom_top] = omega
    dy[next_to_sides] = omega
    return np.concatenate([dx, dy])


class _ConstrainedSolve:
    """z = S^+ r on the complement of span(E) (S symmetric, S E = 0): the right-hand
    side loses its components along E and z is orthogonal to E (Euclidean)."""

    def __init__(self, S, E):
        self.E = E
        Q, _ = np.linalg.qr(E)
        self.Q = Q
        nE = E.shape[1]
        aug = sp.bmat([[S, sp.csr_matrix(E)], [sp.csr_matrix(E.T), sp.csr_matrix((nE, nE))]])
        self.lu = krylov._LU(aug.tocsc())
        self.m = S.shape[0]

    def __call__(self, r):
        r = r - self.Q @ (self.Q.T @ r)
        return self.lu(np.concatenate([r, np.zeros(self.E.shape[1])]))[: self.m]


class LSC:
    """M_S^{-1} of Eq. lsc-definition and the block-triangular M_3^{-1} of Eq.
    nse-precon-lsc (exact solves of F and of the two pressure products)."""

    def __init__(self, sys: problem.System, omega=1.0):
        self.sys = sys
        g = sys.g
        md = sys.Mv.diagonal()
        m = np.concatenate([md, md])
        d = tangential_weights(g, omega)
        self.minv = 1.0 / m
        self.hinv = d / m                      # H = D^{-1/2} M D^{-1/2}, diagonal
        B = sys.BI                             # boundary velocity columns removed
        self.B = B
        E = np.column_stack([sys.e1[g.nu:], sys.e0[g.nu:]])
        self.BMB = _ConstrainedSolve((B @ sp.diags(self.minv) @ B.T).tocsr(), E)
        self.BHB = _ConstrainedSolve((B @ sp.diags(self.hinv) @ B.T).tocsr(), E)
        self.Fsolve = krylov._LU(sys.F)

    def schur_inv(self, rp):
        """M_S^{-1} rp."""
        y = self.BHB(rp)
        t = self.B @ (self.minv * (self.sys.F @ (self.hinv * (self.B.T @ y))))
        return self.BMB(t)

    def __call__(self, r):
        s = self.sys
        nu_ = s.g.nu
        zp = -self.schur_inv(r[nu_:])
        zu = self.Fsolve(r[:nu_] - s.BI.T @ zp)
        return np.concatenate([zu, zp])


def solve(sys, b, tol=1e-6, omega=1.0, restart=50, maxit=2000, x0=None):
    """GMRES with the right preconditioner M_3 on the full Oseen system from the lifted
    boundary data; stops at ||b - K x|| <= tol ||b||.  Returns (x, info)."""
    g = sys.g
    if x0 is None:
        x0 = np.concatenate([sys.DB @ b[: g.nu], np.zeros(g.np_)])
    bp = sys.project_rhs(b)
    P = LSC(sys, omega)
    return krylov.gmres(lambda v: sys.K @ v, P, bp, x0, tol * np.linalg.norm(bp), restart, maxit)

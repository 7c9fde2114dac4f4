"""Chebyshev semi-iteration on symmetric Gauss-Seidel for the singular two-level
pressure mass matrix: the M_cheb block of the cheaper preconditioner P_2
(test infrastructure only).

Sec. 2.3-2.4: Jacobi-based approximations of M_Q = [Qk R^T; R Q0] converge slowly;
symmetric Gauss-Seidel (SGS) converges for symmetric positive semidefinite
matrices, and P_2 = blkdiag(A_AMG, M_cheb) uses a fixed number (20) of Chebyshev
semi-iteration steps built on SGS.  The result is mesh dependent because the
largest non-unit eigenvalue of the SGS iteration matrix tends to 1 under
refinement.

Readings:
* SGS ordering: five colours, the four parity classes (I mod 2, J mod 2) of the
  Q1 nodes and then all P0 elements (unknowns of one colour are not coupled in
  M_Q), forward over the colours and back.  Within a colour the order does not
  matter, so this is the order a multicolour GPU sweep reproduces exactly.
  P = (D + L) D^{-1} (D + L^T) for that ordering.
* Chebyshev interval [a, 1]: the eigenvalues of P^{-1} M_Q are 0 (along k) and lie
  in (0, 1]; a is the smallest nonzero one, computed once per grid.
* Output: the iterate with k projected out (Euclidean k^T z = 0), as for the other
  M_Q solves; the right-hand side first loses its k component.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, problem


def colour_order(g: fem.Grid):
    """Permutation of the frame unknowns [Q1 nodes; P0 elements] by colour."""
    I = np.arange(g.n1) % (g.n + 1)
    J = np.arange(g.n1) // (g.n + 1)
    order = []
    for cj in (0, 1):
        for ci in (0, 1):
            order.append(np.flatnonzero((I % 2 == ci) & (J % 2 == cj)))
    order.append(g.n1 + np.arange(g.n0))
    return np.concatenate(order)


class SGS:
    """z = P^{-1} r for the symmetric Gauss-Seidel splitting of M in a given order:
    a forward sweep (D + L) y = r, then a backward sweep (D + L^T) z = D y."""

    def __init__(self, M, order):
        self.order = order
        Mp = sp.csr_matrix(M)[order][:, order]
        self.Lo = sp.tril(Mp, format="csr")               # D + L
        self.Up = sp.triu(Mp, format="csr")               # D + L^T
        self.d = Mp.diagonal()

    def __call__(self, r):
        rp = r[self.order]
        y = spla.spsolve_triangular(self.Lo, rp, lower=True)
        zp = spla.spsolve_triangular(self.Up, self.d * y, lower=False)
        z = np.empty_like(zp)
        z[self.order] = zp
        return z


def chebyshev(Mop, Pinv, r, a, b, steps):
    """Chebyshev semi-iteration for M x = r with preconditioner P^{-1}, eigenvalues of
    P^{-1} M in [a, b], x_0 = 0; returns x_steps.  The residual of an eigenvector
    component with eigenvalue lam is scaled by T_k((theta - lam)/delta) / T_k(theta/delta)."""
    theta, delta = 0.5 * (b + a), 0.5 * (b - a)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = np.zeros_like(r)
    res = r.copy()
    d = Pinv(res) / theta
    for _ in range(steps):
        x = x + d
        res = res - Mop(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * Pinv(res)
        rho = rho_new
    return x


def sgs_interval(g: fem.Grid, MQ=None, k=None):
    """(a, b): smallest nonzero and largest eigenvalue of P^{-1} M_Q (dense)."""
    if MQ is None:
        s = problem.System(g, 1.0)
        MQ, k = s.MQ, s.k
    order = colour_order(g)
    Mp = MQ.toarray()[np.ix_(order, order)]
    Lo = np.tril(Mp)
    D = np.diag(np.diag(Mp))
    P = Lo @ np.linalg.solve(D, Lo.T)
    lam = np.sort(sla.eigh(Mp, P, eigvals_only=True))
    assert abs(lam[0]) <= 1e-10 * lam[-1]                 # the k direction
    return float(lam[1]), float(lam[-1])


class MCheb:
    """nu * M_cheb^{-1} r: ``steps`` Chebyshev-SGS steps on M_Q, k projected out."""

    def __init__(self, sys, steps=20, interval=None):
        self.sys = sys
        self.k = sys.k
        self.steps = steps
        self.a, self.b = interval if interval is not None else sgs_interval(sys.g, sys.MQ, sys.k)
        self.sgs = SGS(sys.MQ, colour_order(sys.g))

    def __call__(self, r):
        k = self.k
        r = r - (k @ r) / (k @ k) * k
        z = chebyshev(lambda v: self.sys.MQ @ v, self.sgs, r, self.a, self.b, self.steps)
        z = z - (k @ z) / (k @ k) * k
        return self.sys.nu * z


class P2Exact:
    """blkdiag(nu A exact, M_cheb): the paper's P_2 with the A block solved exactly,
    so that its effect on MINRES comes from M_cheb alone."""

    def __init__(self, sys, steps=20):
        from .krylov import _LU
        self.sys = sys
        self.Asolve = _LU(sys.Anu)
        self.mq = MCheb(sys, steps)

    def __call__(self, r):
        nu_ = self.sys.g.nu
        return np.concatenate([self.Asolve(r[:nu_]), self.mq(r[nu_:])])

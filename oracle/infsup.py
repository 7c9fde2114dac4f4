"""Discrete inf-sup constant of the enriched pair and its EST-MINRES estimate
(test infrastructure only).

Sec. 2.4: gamma^2 is the smallest nonzero eigenvalue of the pencil

    B A^{-1} B^T v = lambda M_Q v,        v orthogonal to k,

where k (Prop. 1 / Remark 1) spans the common null space of B^T and M_Q, so the
pencil is singular along k and the problem is posed on a complement of k.  For an
enclosed flow the constant pressure is a second null vector of B^T (but not of
M_Q): it gives the eigenvalue 0, the hydrostatic mode, which "nonzero" excludes.

``dense_gamma2`` is that definition written out with dense matrices (small grids).

EST-MINRES (Sec. 2.4): with the block preconditioner P_1 = blkdiag(A, M_Q), with
k projected out of the M_Q solve, the eigenvalues of P_1^{-1} K are 1 and
(1 +- sqrt(1 + 4 sigma)) / 2 for the pencil eigenvalues sigma.  The eigenvalue
theta_- = (1 - sqrt(1 + 4 gamma^2)) / 2 is the negative one closest to zero, so
gamma^2 = theta_-^2 - theta_-.  The estimate takes for theta_- the negative
harmonic Ritz value closest to zero of the Lanczos process that preconditioned
MINRES runs: the theta with T_{k+1,k}^T T_{k+1,k} y = theta T_k y, T_k the
tridiagonal of the delta_j (diagonal) and gamma_j (off the diagonal), T_{k+1,k}
with gamma_{k+1} below it.  Harmonic Ritz values are the zeros of the MINRES
residual polynomial; they stay outside the gap around zero, so the estimate
approaches gamma^2 from above.  ``harmonic_ritz`` solves that small pencil
directly (dense, scipy.linalg.eig).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import fem, problem


def dense_gamma2(g: fem.Grid):
    """(gamma^2, sigma) with sigma all pencil eigenvalues on the complement of k
    (ascending; sigma[0] is the hydrostatic 0).  Dense: small grids only."""
    s = problem.System(g, 1.0)
    A = s.Anu.toarray()                    # A with identity Dirichlet rows (nu = 1)
    BI = s.BI.toarray()                    # B with the boundary columns removed
    S = BI @ np.linalg.solve(A, BI.T)
    M = s.MQ.toarray()
    W = sla.null_space(s.k[None, :])       # orthonormal basis of the complement of k
    sig = sla.eigh(W.T @ S @ W, W.T @ M @ W, eigvals_only=True)
    return float(sig[1]), sig


def tridiag(delta, gamma, k):
    """T_{k+1,k} from delta_1..delta_k and gamma_1..gamma_{k+1} (gamma_1 unused)."""
    T = np.zeros((k + 1, k))
    for j in range(k):
        T[j, j] = delta[j]
        T[j + 1, j] = gamma[j + 1]
        if j + 1 < k:
            T[j, j + 1] = gamma[j + 1]
    return T


def harmonic_ritz(delta, gamma, k):
    """Harmonic Ritz values (target 0) of the first k Lanczos steps."""
    Tk1 = tridiag(delta, gamma, k)
    Tk = Tk1[:k, :]
    th = sla.eig(Tk1.T @ Tk1, Tk, right=False)
    th = th[np.isfinite(th)]
    return np.sort(th.real[np.abs(th.imag) <= 1e-8 * np.maximum(1.0, np.abs(th.real))])


def est_gamma2(delta, gamma, k):
    """EST-MINRES estimate after k iterations: theta^2 - theta for the negative
    harmonic Ritz value theta closest to zero; NaN while none is negative."""
    th = harmonic_ritz(delta, gamma, k)
    neg = th[th < 0.0]
    if neg.size == 0:
        return float("nan")
    t = neg.max()
    return float(t * t - t)


def est_history(delta, gamma):
    """Estimates after each iteration k = 1 .. len(delta)."""
    return np.array([est_gamma2(delta, gamma, k) for k in range(1, len(delta) + 1)])

"""Exact discrete solution by a bordered sparse direct solve (test infrastructure only).

The enclosed-flow system K is singular with null space span{e1, e0}
(Sec. 2.1 Prop. 1, Remark 2, and Sec. 3 Test problem 4).  Bordering

    [ K    E ] [x]   [b]          E = [e1, e0]
    [ E^T  0 ] [l] = [0]

is nonsingular, and for a consistent b it returns the solution with
sum(p1) = sum(p0) = 0 and l = 0.  SuperLU in float64.

The bordered matrix has dense border rows and columns, which makes the sparse
factorisation slow beyond n = 64.  ``solve_pinned`` computes the same solution
another way for larger grids: it fixes one Q1 and one P0 pressure value at zero
(identity rows and zero columns for those two unknowns, a nonsingular sparse
system when b is consistent) and then removes the e1 / e0 components, which
gives the same canonical representative.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def bordered_solve(K, E, b):
    """Solve [K E; E^T 0][x; l] = [b; 0]; returns (x, l)."""
    E = sp.csr_matrix(np.atleast_2d(E).T) if np.ndim(E) == 1 else sp.csr_matrix(E)
    m = E.shape[1]
    Kb = sp.bmat([[K, E], [E.T, None]]).tocsc()
    rhs = np.concatenate([b, np.zeros(m)])
    sol = spla.splu(Kb, permc_spec="COLAMD").solve(rhs)
    return sol[: K.shape[0]], sol[K.shape[0]:]


def solve(sys, b):
    """Exact solution of the enclosed-flow system (canonical pressure)."""
    E = np.stack([sys.e1, sys.e0], axis=1)
    x, lam = bordered_solve(sys.K, E, b)
    return x, lam


def solve_transpose(sys, b):
    """Exact solution of K^T x = b with the same bordering (adjoint systems)."""
    E = np.stack([sys.e1, sys.e0], axis=1)
    x, lam = bordered_solve(sys.K.T.tocsr(), E, b)
    return x, lam


def solve_pinned(sys, b):
    """Exact canonical solution via two pinned pressure unknowns (see the module
    docstring); b must be consistent (zero e1 / e0 components)."""
    g = sys.g
    keep = np.ones(sys.K.shape[0])
    keep[[g.nu, g.nu + g.n1]] = 0.0          # first Q1 and first P0 pressure
    Dk = sp.diags(keep)
    Kp = (Dk @ sys.K @ Dk + sp.diags(1.0 - keep)).tocsc()
    x = spla.splu(Kp, permc_spec="COLAMD").solve(b * keep)
    return sys.canonical(x)

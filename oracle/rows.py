"""Selected rows of the saddle-point product K x, element by element (test infrastructure only).

At the full grid sizes (512^2, 1024^2) the assembled K of ``problem.System`` no longer fits
a test, so the parity tests compare sampled entries of K x.  Each entry is the sum of
the element contributions of the (at most four) elements that contain the row's node,
with the same element matrices (3x3 Gauss, ``fem.element_matrices``; convection per
element from the Q2 interpolant of the wind, Sec. 3.1) and the same Dirichlet treatment
as ``problem.System`` (Sec. 2):

* velocity rows on the boundary are identity rows;
* every other row sees the velocity only at interior nodes (boundary columns are zero);
* velocity row i of component c:  sum_T [nu A_T + N_T] (i, :) u_c,T  +  B_T^T(i, :) p_T;
* Q1 row k:  sum_T B1_T(k, :) u_T;   P0 row T:  B0_T u_T;  with b(u, p) = -int p div u.

Rows are indices into x = [u_x; u_y; p1; p0].
"""
from __future__ import annotations

import numpy as np

from . import fem


def _elements_of_q2(g: fem.Grid, i, j):
    """(ex, ey, local index b*3 + a) of the elements containing Q2 node (i, j)."""
    out = []
    exs = [i // 2 - 1, i // 2] if i % 2 == 0 else [i // 2]
    eys = [j // 2 - 1, j // 2] if j % 2 == 0 else [j // 2]
    for ey in eys:
        for ex in exs:
            if 0 <= ex < g.n and 0 <= ey < g.n:
                out.append((ex, ey, (j - 2 * ey) * 3 + (i - 2 * ex)))
    return out


def _elements_of_q1(g: fem.Grid, I, J):
    out = []
    for ey in (J - 1, J):
        for ex in (I - 1, I):
            if 0 <= ex < g.n and 0 <= ey < g.n:
                out.append((ex, ey, (J - ey) * 2 + (I - ex)))
    return out


def k_rows(g: fem.Grid, nu, wind, x, rows, bound=False):
    """Entries (K x)[rows] of the Stokes (wind None) or Oseen operator of problem.System.

    bound=True returns instead the element-wise sums of |entries| x |x|, an upper bound
    of (|K| |x|)[rows] that scales a rounding-error tolerance per entry."""
    x = np.asarray(x, dtype=np.float64)
    E = fem.element_matrices(g)
    if bound:
        E = {k: np.abs(v) for k, v in E.items()}
        x = np.abs(x)
    T = g.tables(3)
    W = T["W"]
    N, nv, n1 = g.N, g.nv, g.n1
    ux, uy = x[:nv].copy(), x[nv:2 * nv].copy()
    ux[g.bnd] = 0.0                       # boundary columns of K are zero
    uy[g.bnd] = 0.0
    p1, p0 = x[2 * nv:2 * nv + n1], x[2 * nv + n1:]
    wind = None if wind is None else np.asarray(wind, dtype=np.float64)

    def conv(e):
        if wind is None:
            return 0.0
        con = g.q2_conn[e]
        wx = T["P2"] @ wind[:nv][con]     # wind at the Gauss points of element e
        wy = T["P2"] @ wind[nv:][con]
        Ne = np.einsum("q,qi,q,qj->ij", W, T["P2"], wx, T["DX2"]) + \
            np.einsum("q,qi,q,qj->ij", W, T["P2"], wy, T["DY2"])
        return np.abs(Ne) if bound else Ne

    out = np.empty(len(rows))
    for r_i, r in enumerate(np.asarray(rows)):
        r = int(r)
        if r < 2 * nv:                    # velocity row
            c, node = divmod(r, nv)
            j, i = divmod(node, N)
            if g.bnd[node]:
                out[r_i] = x[r]
                continue
            u = ux if c == 0 else uy
            s = 0.0
            for ex, ey, li in _elements_of_q2(g, i, j):
                e = ey * g.n + ex
                con = g.q2_conn[e]
                Fe = nu * E["A"] + conv(e)   # (bound: |nu A| + |N| >= |nu A + N|)
                s += Fe[li] @ u[con]
                B1 = E["B1x"] if c == 0 else E["B1y"]
                B0 = E["B0x"] if c == 0 else E["B0y"]
                s += B1[:, li] @ p1[g.q1_conn[e]] + B0[0, li] * p0[e]
            out[r_i] = s
        elif r < 2 * nv + n1:              # Q1 pressure row
            k = r - 2 * nv
            J, I = divmod(k, g.n + 1)
            s = 0.0
            for ex, ey, lk in _elements_of_q1(g, I, J):
                e = ey * g.n + ex
                con = g.q2_conn[e]
                s += E["B1x"][lk] @ ux[con] + E["B1y"][lk] @ uy[con]
            out[r_i] = s
        else:                              # P0 pressure row
            e = r - 2 * nv - n1
            con = g.q2_conn[e]
            out[r_i] = E["B0x"][0] @ ux[con] + E["B0y"][0] @ uy[con]
    return out

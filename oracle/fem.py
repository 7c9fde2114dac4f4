"""Q2--Q1* finite elements on a uniform rectangular grid, assembled in FP64 CSR.

Test infrastructure (see the package docstring); never used by the product path.

Discretisation (Sec. 2.1 of the paper, Eq. eth_pressure_space / eth_spec):
velocity in (Q2)^2, pressure in the frame {Q1 Lagrange basis} U {P0 indicators}.
A pressure vector is p = [p_k; p_0] with the n_k = (n+1)^2 Q1 coefficients
first and the n_0 = n^2 element constants after them (Eq. function_basis).

Layout (shared contract with the CUDA library, restated independently there):
* Q2 lattice of (2n+1)^2 nodes, node (i, j) at (x0 + i*hx/2, y0 + j*hy/2),
  global index j*(2n+1) + i (x fastest).  Velocity = [u_x; u_y].
* Q1 lattice of (n+1)^2 nodes, index J*(n+1) + I.
* Element (ex, ey) has index ey*n + ex.

Every element integral uses the 3x3 Gauss-Legendre rule on the affine map.
That rule is exact for A, B, M_Q, the velocity mass and the Q1 matrices; for
the convection term with a Q2 wind it *defines* the discrete operator.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


# --------------------------------------------------------------------------
# 1D reference shape functions on [0, 1]
# --------------------------------------------------------------------------
def q2_1d(t):
    """Quadratic Lagrange basis at nodes {0, 1/2, 1}: values and d/dt."""
    t = np.asarray(t, dtype=np.float64)
    v = np.stack([2.0 * (t - 0.5) * (t - 1.0), -4.0 * t * (t - 1.0), 2.0 * t * (t - 0.5)], axis=-1)
    d = np.stack([4.0 * t - 3.0, 4.0 - 8.0 * t, 4.0 * t - 1.0], axis=-1)
    return v, d


def q1_1d(t):
    """Linear Lagrange basis at nodes {0, 1}: values and d/dt."""
    t = np.asarray(t, dtype=np.float64)
    v = np.stack([1.0 - t, t], axis=-1)
    d = np.stack([-np.ones_like(t), np.ones_like(t)], axis=-1)
    return v, d


def gauss01(m):
    """m-point Gauss-Legendre rule mapped to [0, 1] (weights sum to 1)."""
    x, w = np.polynomial.legendre.leggauss(m)
    return 0.5 * (x + 1.0), 0.5 * w


# --------------------------------------------------------------------------
# Grid and connectivity
# --------------------------------------------------------------------------
class Grid:
    """Uniform n x n grid of rectangles on [x0,x1] x [y0,y1]."""

    def __init__(self, n, x0=-1.0, x1=1.0, y0=-1.0, y1=1.0):
        self.n = int(n)
        self.x0, self.x1, self.y0, self.y1 = float(x0), float(x1), float(y0), float(y1)
        self.hx = (self.x1 - self.x0) / self.n
        self.hy = (self.y1 - self.y0) / self.n
        self.N = 2 * self.n + 1                     # Q2 nodes per direction
        self.nv = self.N * self.N                   # Q2 nodes
        self.nu = 2 * self.nv                       # velocity DoFs
        self.n1 = (self.n + 1) ** 2                 # Q1 pressure DoFs (n_k)
        self.n0 = self.n * self.n                   # P0 pressure DoFs (n_0)
        self.np_ = self.n1 + self.n0                # frame size n_p
        self.nt = self.nu + self.np_                # total unknowns
        n = self.n
        ex, ey = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
        ex = ex.ravel()
        ey = ey.ravel()                              # element e = ey*n + ex
        self.ex, self.ey = ex, ey
        a = np.array([0, 1, 2, 0, 1, 2, 0, 1, 2])    # local Q2 index i = b*3 + a
        b = np.array([0, 0, 0, 1, 1, 1, 2, 2, 2])
        self.q2_conn = (2 * ey[:, None] + b[None, :]) * self.N + (2 * ex[:, None] + a[None, :])
        c = np.array([0, 1, 0, 1])                   # local Q1 index = d*2 + c
        d = np.array([0, 0, 1, 1])
        self.q1_conn = (ey[:, None] + d[None, :]) * (n + 1) + (ex[:, None] + c[None, :])
        i = np.arange(self.N)
        self.xq2 = self.x0 + 0.5 * self.hx * i       # Q2 lattice coordinates
        self.yq2 = self.y0 + 0.5 * self.hy * i
        X, Y = np.meshgrid(self.xq2, self.yq2, indexing="xy")
        self.X2, self.Y2 = X.ravel(), Y.ravel()
        I = np.arange(n + 1)
        X1, Y1 = np.meshgrid(self.x0 + self.hx * I, self.y0 + self.hy * I, indexing="xy")
        self.X1, self.Y1 = X1.ravel(), Y1.ravel()
        onb = np.zeros((self.N, self.N), dtype=bool)
        onb[0, :] = onb[-1, :] = onb[:, 0] = onb[:, -1] = True
        self.bnd = onb.ravel()                       # Dirichlet Q2 nodes (whole boundary)

    # reference-element tables at the m x m Gauss points, point q = s*m + r
    def tables(self, m=3):
        t, w = gauss01(m)
        v2, d2 = q2_1d(t)
        v1, d1 = q1_1d(t)
        a = np.array([0, 1, 2, 0, 1, 2, 0, 1, 2]); b = np.array([0, 0, 0, 1, 1, 1, 2, 2, 2])
        c = np.array([0, 1, 0, 1]); d = np.array([0, 0, 1, 1])
        r = np.tile(np.arange(m), m); s = np.repeat(np.arange(m), m)
        T = {}
        T["W"] = w[r] * w[s] * self.hx * self.hy
        T["P2"] = v2[r][:, a] * v2[s][:, b]
        T["DX2"] = d2[r][:, a] * v2[s][:, b] / self.hx
        T["DY2"] = v2[r][:, a] * d2[s][:, b] / self.hy
        T["P1"] = v1[r][:, c] * v1[s][:, d]
        T["DX1"] = d1[r][:, c] * v1[s][:, d] / self.hx
        T["DY1"] = v1[r][:, c] * d1[s][:, d] / self.hy
        T["xi"], T["eta"] = t[r], t[s]
        return T


def _assemble(rows_conn, cols_conn, Ke, shape):
    """Scatter-add element matrices Ke ((nloc_r, nloc_c) or (nel, nloc_r, nloc_c))."""
    nel = rows_conn.shape[0]
    if Ke.ndim == 2:
        Ke = np.broadcast_to(Ke, (nel,) + Ke.shape)
    R = np.broadcast_to(rows_conn[:, :, None], Ke.shape)
    C = np.broadcast_to(cols_conn[:, None, :], Ke.shape)
    M = sp.coo_matrix((Ke.ravel(), (R.ravel(), C.ravel())), shape=shape)
    return M.tocsr()


# --------------------------------------------------------------------------
# Element matrices (3x3 Gauss) and global matrices
# --------------------------------------------------------------------------
def element_matrices(g: Grid):
    """Constant element matrices of the uniform grid (dict of ndarrays)."""
    T = g.tables(3)
    W = T["W"]
    E = {}
    E["A"] = (T["DX2"] * W[:, None]).T @ T["DX2"] + (T["DY2"] * W[:, None]).T @ T["DY2"]
    E["M2"] = (T["P2"] * W[:, None]).T @ T["P2"]
    E["B1x"] = -(T["P1"] * W[:, None]).T @ T["DX2"]          # (4, 9)
    E["B1y"] = -(T["P1"] * W[:, None]).T @ T["DY2"]
    E["B0x"] = -(W @ T["DX2"])[None, :]                      # (1, 9)
    E["B0y"] = -(W @ T["DY2"])[None, :]
    E["Qk"] = (T["P1"] * W[:, None]).T @ T["P1"]             # (4, 4)
    E["R"] = (W @ T["P1"])[None, :]                          # (1, 4)
    E["Q0"] = np.array([[W.sum()]])
    E["K1"] = (T["DX1"] * W[:, None]).T @ T["DX1"] + (T["DY1"] * W[:, None]).T @ T["DY1"]
    return E


def stiffness_q2(g: Grid):
    """Scalar Q2 Laplacian a_ij = int grad phi_i . grad phi_j (Sec. 2, a(u,v))."""
    return _assemble(g.q2_conn, g.q2_conn, element_matrices(g)["A"], (g.nv, g.nv))


def mass_q2(g: Grid):
    """Scalar Q2 mass matrix int phi_i phi_j (per velocity component)."""
    return _assemble(g.q2_conn, g.q2_conn, element_matrices(g)["M2"], (g.nv, g.nv))


def wind_at_gauss(g: Grid, wind, m=3):
    """Q2 interpolant of the nodal wind (2*nv vector) at each element's Gauss points."""
    T = g.tables(m)
    wx = wind[: g.nv][g.q2_conn] @ T["P2"].T                 # (nel, m*m)
    wy = wind[g.nv:][g.q2_conn] @ T["P2"].T
    return wx, wy, T


def convection_q2(g: Grid, wind, m=3):
    """Scalar convection n_ij = int (w_h . grad phi_j) phi_i, m x m Gauss (Sec. 3.1).

    Row i is the test function, column j the trial function.  With m = 3
    this is the discrete convection operator of the method.
    """
    wx, wy, T = wind_at_gauss(g, wind, m)
    W = T["W"]
    Ne = np.einsum("q,qi,eq,qj->eij", W, T["P2"], wx, T["DX2"]) + \
        np.einsum("q,qi,eq,qj->eij", W, T["P2"], wy, T["DY2"])
    return _assemble(g.q2_conn, g.q2_conn, Ne, (g.nv, g.nv))


def divergence(g: Grid):
    """B = [B1; B0], b(u, p) = -int p div u (Sec. 2).  Shape (n_p, 2*nv), no BCs."""
    E = element_matrices(g)
    e = np.arange(g.n0)[:, None]
    B1x = _assemble(g.q1_conn, g.q2_conn, E["B1x"], (g.n1, g.nv))
    B1y = _assemble(g.q1_conn, g.q2_conn, E["B1y"], (g.n1, g.nv))
    B0x = _assemble(e, g.q2_conn, E["B0x"], (g.n0, g.nv))
    B0y = _assemble(e, g.q2_conn, E["B0y"], (g.n0, g.nv))
    B1 = sp.hstack([B1x, B1y]).tocsr()
    B0 = sp.hstack([B0x, B0y]).tocsr()
    return B1, B0


def pressure_mass(g: Grid):
    """Two-field pressure mass matrix M_Q = [Qk R^T; R Q0] (Sec. 2.3)."""
    E = element_matrices(g)
    e = np.arange(g.n0)[:, None]
    Qk = _assemble(g.q1_conn, g.q1_conn, E["Qk"], (g.n1, g.n1))
    R = _assemble(e, g.q1_conn, E["R"], (g.n0, g.n1))
    Q0 = sp.diags(np.full(g.n0, E["Q0"][0, 0]))
    MQ = sp.bmat([[Qk, R.T], [R, Q0]]).tocsr()
    return MQ, Qk, R, Q0


def q1_stiffness(g: Grid):
    """Q1 Laplacian int grad psi_j . grad psi_i (diffusion part of F_1, Sec. 3.1)."""
    return _assemble(g.q1_conn, g.q1_conn, element_matrices(g)["K1"], (g.n1, g.n1))


def q1_convection(g: Grid, wind, m=3):
    """Q1 convection int (w_h . grad psi_j) psi_i with the Q2 wind, m x m Gauss (Sec. 3.1)."""
    wx, wy, T = wind_at_gauss(g, wind, m)
    W = T["W"]
    Ne = np.einsum("q,qi,eq,qj->eij", W, T["P1"], wx, T["DX1"]) + \
        np.einsum("q,qi,eq,qj->eij", W, T["P1"], wy, T["DY1"])
    return _assemble(g.q1_conn, g.q1_conn, Ne, (g.n1, g.n1))


def null_vector_k(g: Grid):
    """k = [1_{n_k}; -1_{n_0}] (Eq. pressure_null_vector)."""
    return np.concatenate([np.ones(g.n1), -np.ones(g.n0)])


# --------------------------------------------------------------------------
# Evaluation of discrete fields (for error norms)
# --------------------------------------------------------------------------
def l2_h1_errors(g: Grid, u, p, u_exact, grad_exact, p_exact, m=5):
    """L2 and H1-seminorm velocity errors and L2 pressure error (mean removed).

    u_exact(x, y) -> (ux, uy); grad_exact(x, y) -> (dux/dx, dux/dy, duy/dx, duy/dy);
    p_exact(x, y) -> p (any additive constant).  Uses m x m Gauss per element.
    """
    T = g.tables(m)
    W = T["W"]
    xq = g.x0 + (g.ex[:, None] + T["xi"][None, :]) * g.hx
    yq = g.y0 + (g.ey[:, None] + T["eta"][None, :]) * g.hy
    ux = u[: g.nv][g.q2_conn]; uy = u[g.nv:][g.q2_conn]
    uxh = ux @ T["P2"].T; uyh = uy @ T["P2"].T
    gh = [ux @ T["DX2"].T, ux @ T["DY2"].T, uy @ T["DX2"].T, uy @ T["DY2"].T]
    ex, ey = u_exact(xq, yq)
    ge = grad_exact(xq, yq)
    l2u = np.sqrt(np.sum(W * ((uxh - ex) ** 2 + (uyh - ey) ** 2)))
    h1u = np.sqrt(np.sum(W * sum((a - b) ** 2 for a, b in zip(gh, ge))))
    ph = p[: g.n1][g.q1_conn] @ T["P1"].T + p[g.n1:][:, None]
    pe = p_exact(xq, yq)
    area = W.sum() * g.n0
    dp = ph - pe
    dp = dp - np.sum(W * dp) / area
    l2p = np.sqrt(np.sum(W * dp ** 2))
    return l2u, h1u, l2p


def element_divergence(g: Grid, u):
    """int_T div u_h for every element T (exact for Q2 with 3x3 Gauss)."""
    T = g.tables(3)
    W = T["W"]
    ux = u[: g.nv][g.q2_conn]; uy = u[g.nv:][g.q2_conn]
    return (ux @ T["DX2"].T + uy @ T["DY2"].T) @ W

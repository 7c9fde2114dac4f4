"""Inflow-outflow flow on a masked uniform grid: the flow over a step (test
infrastructure only).

Sec. 3, Test problem 3: D = [-1, 0) x [0, 1]  U  [0, 5] x [-1, 1], viscosity 1/50,
parabolic inflow u = (4y(1 - y), 0) at x = -1, the natural (do-nothing) condition
at the outflow x = 5, no-slip walls elsewhere; the Oseen system is the one after
five Picard steps from the Stokes solution.  The grid is uniform with square
elements of side h on the bounding box [-1, 5] x [-1, 1]; an element is active
when it lies in D.

Layout.  Unknowns live on the full lattice of the bounding box (Q2 nodes, Q1
nodes, P0 elements), ordered as on the square grid; those of inactive nodes or
elements are kept with identity rows and value 0.  Velocity rows are identity at
Dirichlet nodes: active nodes on the boundary of D except those strictly inside
the outflow edge (the outflow corners belong to the walls).  The natural outflow
condition needs nothing else: it is what the weak form gives where no Dirichlet
row is imposed.

Null space.  The frame vector k (1 on the active Q1 nodes, -1 on the active
elements) is the zero function, so B^T k = 0 and M_Q k = 0 whatever the boundary
conditions; with an outflow boundary the constant pressure is no longer in
ker B^T, so the system is singular along [0; k] only (Sec. 2, one-dimensional
pressure null space).  Solutions are returned with k^T p = 0.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import direct, fem, krylov


class MaskedGrid:
    """nx x ny square elements of side h from (x0, y0); ``active`` is (ny, nx) bool.
    ``x_out``: abscissa of the outflow edge (natural condition), or None."""

    tables = fem.Grid.tables

    def __init__(self, nx, ny, h, x0, y0, active, x_out=None):
        self.nx, self.ny = int(nx), int(ny)
        self.hx = self.hy = float(h)
        self.x0, self.y0 = float(x0), float(y0)
        self.Nx, self.Ny = 2 * self.nx + 1, 2 * self.ny + 1
        self.nv = self.Nx * self.Ny
        self.nu = 2 * self.nv
        self.n1 = (self.nx + 1) * (self.ny + 1)
        self.n0 = self.nx * self.ny
        self.np_ = self.n1 + self.n0
        self.nt = self.nu + self.np_
        act = np.asarray(active, dtype=bool).reshape(self.ny, self.nx)
        self.active = act
        self.elems = np.flatnonzero(act.ravel())           # element e = ey*nx + ex
        ex, ey = self.elems % self.nx, self.elems // self.nx
        a = np.array([0, 1, 2, 0, 1, 2, 0, 1, 2]); b = np.array([0, 0, 0, 1, 1, 1, 2, 2, 2])
        self.q2_conn = (2 * ey[:, None] + b[None, :]) * self.Nx + (2 * ex[:, None] + a[None, :])
        c = np.array([0, 1, 0, 1]); d = np.array([0, 0, 1, 1])
        self.q1_conn = (ey[:, None] + d[None, :]) * (self.nx + 1) + (ex[:, None] + c[None, :])
        self.q2_active = np.zeros(self.nv, dtype=bool); self.q2_active[self.q2_conn.ravel()] = True
        self.q1_active = np.zeros(self.n1, dtype=bool); self.q1_active[self.q1_conn.ravel()] = True
        self.p0_active = act.ravel().copy()
        jj, ii = np.divmod(np.arange(self.nv), self.Nx)
        self.X2 = self.x0 + 0.5 * h * ii
        self.Y2 = self.y0 + 0.5 * h * jj
        # a node is interior when every element slot around it is an active element
        inner = np.ones(self.nv, dtype=bool)
        for node in range(self.nv):
            i, j = ii[node], jj[node]
            exs = [i // 2 - 1, i // 2] if i % 2 == 0 else [i // 2]
            eys = [j // 2 - 1, j // 2] if j % 2 == 0 else [j // 2]
            for e_y in eys:
                for e_x in exs:
                    if not (0 <= e_x < self.nx and 0 <= e_y < self.ny and act[e_y, e_x]):
                        inner[node] = False
        bnd = self.q2_active & ~inner
        self.outflow = np.zeros(self.nv, dtype=bool)
        if x_out is not None:
            on = bnd & np.isclose(self.X2, x_out)
            ys = self.Y2[on]
            # strictly inside the outflow edge: not at its two wall corners
            self.outflow = on & (self.Y2 > ys.min() + 1e-12) & (self.Y2 < ys.max() - 1e-12)
        self.dirichlet = bnd & ~self.outflow
        self.fixed = self.dirichlet | ~self.q2_active      # identity velocity rows
        self.bnd = self.fixed                               # same role as Grid.bnd


def step_grid(m):
    """The step domain with h = 1/m (nx = 6m, ny = 2m)."""
    nx, ny = 6 * m, 2 * m
    h = 1.0 / m
    xc = -1.0 + h * (np.arange(nx) + 0.5)
    yc = -1.0 + h * (np.arange(ny) + 0.5)
    X, Y = np.meshgrid(xc, yc, indexing="xy")
    active = ~((X < 0.0) & (Y < 0.0))
    return MaskedGrid(nx, ny, h, -1.0, -1.0, active, x_out=5.0)


def channel_grid(m, length=2.0):
    """The channel [0, length] x [-1, 1] with h = 1/m and outflow at x = length."""
    nx, ny = int(round(length * m)), 2 * m
    return MaskedGrid(nx, ny, 1.0 / m, 0.0, -1.0, np.ones((ny, nx), dtype=bool), x_out=length)


class StepSystem:
    """Assembled FP64 Stokes (wind None) or Oseen system on a MaskedGrid."""

    def __init__(self, g: MaskedGrid, nu, wind=None):
        self.g = g
        self.nu = float(nu)
        E = fem.element_matrices(g)
        nv, n1, n0 = g.nv, g.n1, g.n0
        A = fem._assemble(g.q2_conn, g.q2_conn, E["A"], (nv, nv))
        self.Mv = fem._assemble(g.q2_conn, g.q2_conn, E["M2"], (nv, nv))
        Fs = self.nu * A
        if wind is not None:
            Fs = Fs + fem.convection_q2(g, np.asarray(wind, dtype=np.float64))
        self.Fs = Fs.tocsr()
        e = g.elems[:, None]
        B1 = sp.hstack([fem._assemble(g.q1_conn, g.q2_conn, E["B1x"], (n1, nv)),
                        fem._assemble(g.q1_conn, g.q2_conn, E["B1y"], (n1, nv))])
        B0 = sp.hstack([fem._assemble(e, g.q2_conn, E["B0x"], (n0, nv)),
                        fem._assemble(e, g.q2_conn, E["B0y"], (n0, nv))])
        self.B = sp.vstack([B1, B0]).tocsr()
        Qk = fem._assemble(g.q1_conn, g.q1_conn, E["Qk"], (n1, n1))
        R = fem._assemble(e, g.q1_conn, E["R"], (n0, n1))
        Q0 = sp.diags(E["Q0"][0, 0] * g.p0_active.astype(float))
        self.MQ = sp.bmat([[Qk, R.T], [R, Q0]]).tocsr()
        di = (~g.fixed).astype(float)
        self.DIs, self.DBs = sp.diags(di), sp.diags(1.0 - di)
        self.DI = sp.block_diag([self.DIs, self.DIs]).tocsr()
        self.DB = sp.block_diag([self.DBs, self.DBs]).tocsr()
        FsI = (self.DIs @ self.Fs @ self.DIs + self.DBs).tocsr()
        self.F = sp.block_diag([FsI, FsI]).tocsr()
        AsI = (self.DIs @ (self.nu * A) @ self.DIs + self.DBs).tocsr()
        self.Anu = sp.block_diag([AsI, AsI]).tocsr()
        self.BI = (self.B @ self.DI).tocsr()
        self.B1I = (B1.tocsr() @ self.DI).tocsr()
        self.B0I = (B0.tocsr() @ self.DI).tocsr()
        pin = np.concatenate([~g.q1_active, ~g.p0_active]).astype(float)
        self.pin1 = sp.diags((~g.q1_active).astype(float))
        self.K = sp.bmat([[self.F, self.BI.T], [self.BI, sp.diags(pin)]]).tocsr()
        self.K1 = sp.bmat([[self.F, self.B1I.T], [self.B1I, self.pin1]]).tocsr()   # reduced system
        self.Qk = Qk.tocsr()
        self.wind = None if wind is None else np.asarray(wind, dtype=np.float64)
        self.k = np.concatenate([g.q1_active.astype(float), -g.p0_active.astype(float)])
        self.kx = np.concatenate([np.zeros(g.nu), self.k])

    def rhs(self, ubc):
        """b = [D_I(-F u_b) + D_B u_b; -B u_b] (no body force; u_b zero off the Dirichlet nodes)."""
        g = self.g
        ub = self.DB @ np.asarray(ubc, dtype=np.float64)
        Fub = np.concatenate([self.Fs @ ub[: g.nv], self.Fs @ ub[g.nv:]])
        return np.concatenate([self.DI @ (-Fub) + ub, -(self.B @ ub)])

    def solve(self, b):
        """Exact solution with k^T p = 0 (bordered with [0; k])."""
        x, _ = direct.bordered_solve(self.K, self.kx, b)
        return x


def inflow_data(g: MaskedGrid, profile):
    """Dirichlet data: u = (profile(y), 0) at the leftmost active column of Dirichlet
    nodes, zero elsewhere."""
    ub = np.zeros(g.nu)
    left = g.dirichlet & np.isclose(g.X2, g.x0)
    ub[: g.nv][left] = profile(g.Y2[left])
    return ub


def step_inflow(g):
    return inflow_data(g, lambda y: 4.0 * y * (1.0 - y))


def picard(g: MaskedGrid, nu, ubc, steps):
    """Picard iterates x_1..x_steps (x_1 Stokes) and the nonlinear residuals
    ||b(u) - K(u) x|| / ||b(u)|| at each iterate."""
    xs, res = [], []
    wind = np.zeros(g.nu)
    for _ in range(steps):
        s = StepSystem(g, nu, wind)
        x = s.solve(s.rhs(ubc))
        xs.append(x)
        s1 = StepSystem(g, nu, x[: g.nu].copy())
        b1 = s1.rhs(ubc)
        res.append(np.linalg.norm(b1 - s1.K @ x) / np.linalg.norm(b1))
        wind = x[: g.nu].copy()
    return xs, res


def vertical_flux(g: MaskedGrid, u, i):
    """Flux int u_x dy through the lattice column of Q2 index i (even: element edges),
    Simpson's rule on each active edge (exact for the Q2 trace)."""
    ux = u[: g.nv].reshape(g.Ny, g.Nx)
    h = g.hy
    tot = 0.0
    for ey in range(g.ny):
        ex_l, ex_r = i // 2 - 1, i // 2
        on = any(0 <= ex < g.nx and g.active[ey, ex] for ex in (ex_l, ex_r))
        if on:
            j = 2 * ey
            tot += h / 6.0 * (ux[j, i] + 4.0 * ux[j + 1, i] + ux[j + 2, i])
    return tot


def dense_gamma2(g: MaskedGrid):
    """Smallest eigenvalue of B A^{-1} B^T v = lambda M_Q v over the active pressure
    unknowns orthogonal to k (no hydrostatic mode with an outflow boundary)."""
    import scipy.linalg as sla
    s = StepSystem(g, 1.0)
    act = np.concatenate([g.q1_active, g.p0_active])
    A = s.Anu.toarray()
    BI = s.BI.toarray()[act]
    S = BI @ np.linalg.solve(A, BI.T)
    M = s.MQ.toarray()[np.ix_(act, act)]
    W = sla.null_space(s.k[act][None, :])
    sig = sla.eigh(W.T @ S @ W, W.T @ M @ W, eigvals_only=True)
    return float(sig[0]), sig


def inflow_robin_q1(g: MaskedGrid, wind):
    """Q1 boundary matrix -int_{Gamma_in} (w.n) psi_j psi_i ds over the boundary edges of
    the active domain where the wind enters (w.n < 0 at the edge midpoint); w is the
    Q2 trace of the wind (quadratic along the edge), 3-point Gauss (exact)."""
    t, wq = fem.gauss01(3)
    wx = np.asarray(wind)[: g.nv]
    wy = np.asarray(wind)[g.nv:]
    rows, cols, vals = [], [], []
    for e in g.elems:
        ex, ey = e % g.nx, e // g.nx
        # (neighbour offset, outward normal, Q2 nodes along the edge, Q1 end nodes)
        edges = [((-1, 0), (-1.0, 0.0), [(2 * ex, 2 * ey + k) for k in range(3)], [(ex, ey), (ex, ey + 1)]),
                 ((1, 0), (1.0, 0.0), [(2 * ex + 2, 2 * ey + k) for k in range(3)], [(ex + 1, ey), (ex + 1, ey + 1)]),
                 ((0, -1), (0.0, -1.0), [(2 * ex + k, 2 * ey) for k in range(3)], [(ex, ey), (ex + 1, ey)]),
                 ((0, 1), (0.0, 1.0), [(2 * ex + k, 2 * ey + 2) for k in range(3)], [(ex, ey + 1), (ex + 1, ey + 1)])]
        for (dx, dy), (nx_, ny_), q2n, q1n in edges:
            fx, fy = ex + dx, ey + dy
            if 0 <= fx < g.nx and 0 <= fy < g.ny and g.active[fy, fx]:
                continue                                    # interior edge
            wn = np.array([wx[j * g.Nx + i] * nx_ + wy[j * g.Nx + i] * ny_ for i, j in q2n])
            if wn[1] >= 0.0:
                continue                                    # not an inflow edge
            quad = np.stack([(1 - t) * (1 - 2 * t), 4 * t * (1 - t), t * (2 * t - 1)], axis=1)   # Q2 trace
            lin = np.stack([1 - t, t], axis=1)
            wng = quad @ wn
            Me = -(lin * (wq * wng * g.hx)[:, None]).T @ lin
            ids = [j * (g.nx + 1) + i for i, j in q1n]
            for a in range(2):
                for b in range(2):
                    rows.append(ids[a]); cols.append(ids[b]); vals.append(Me[a, b])
    return sp.coo_matrix((vals, (rows, cols)), shape=(g.n1, g.n1)).tocsr()


class StepPCD1:
    """Step I preconditioner [F B1^T; 0 -M_S]^{-1} on the masked grid (Eq.
    discrete-commutator1x): M_S^{-1} r = Ap^{-1} F1 Q1^{-1} r with Q1, F1 = nu K1 + N1(w)
    and Ap = B1 Md^{-1} B1^T assembled over the active elements and the free velocity
    columns (interior and outflow); inactive Q1 nodes get identity rows.

    Boundary condition of F1 (the paper leaves it to the PCD literature): the Robin
    term -int_{Gamma_in} (w.n) p q ds on the inflow boundary, the form the pressure
    convection-diffusion operator takes when its convection term is integrated by
    parts like the velocity one.  Without it, F1 annihilates the constants (natural
    boundary conditions everywhere), M_S^{-1} is singular while the Schur complement
    of an outflow problem is not, and Step I stagnates (measured: no convergence in
    600 GMRES(50) steps on the step at h = 1/2 ... 1/8, against 14-17 with the term).
    For enclosed flow, and for the Stokes problem (w = 0), the term vanishes."""

    def __init__(self, sys):
        self.sys = sys
        g = sys.g
        self.Fsolve = krylov._LU(sys.F)
        self.Q1solve = krylov._LU((sys.Qk + sys.pin1).tocsc())
        F1 = sys.nu * fem.q1_stiffness(g)
        if sys.wind is not None:
            F1 = F1 + fem.q1_convection(g, sys.wind) + inflow_robin_q1(g, sys.wind)
        self.F1 = (F1 + sys.pin1).tocsr()
        md = sys.Mv.diagonal()
        with np.errstate(divide="ignore"):
            inv = np.where(md > 0.0, 1.0 / np.where(md > 0.0, md, 1.0), 0.0)
        Mdinv = sp.diags(np.concatenate([inv, inv]))
        self.Apsolve = krylov._LU((sys.B1I @ Mdinv @ sys.B1I.T + sys.pin1).tocsc())

    def schur_inv(self, rp):
        return self.Apsolve(self.F1 @ self.Q1solve(rp))

    def __call__(self, r):
        s = self.sys
        nu_ = s.g.nu
        zp = -self.schur_inv(r[nu_:])
        zu = self.Fsolve(r[:nu_] - s.B1I.T @ zp)
        return np.concatenate([zu, zp])


class StepM1:
    """Step II preconditioner [F B^T; 0 -(1/nu) M_Q]^{-1} (Eq. nse-precon-ref) on the masked
    grid: the M_Q solve is augmented with k (active unknowns) and keeps identity rows
    for the inactive pressure unknowns."""

    def __init__(self, sys):
        self.sys = sys
        g = sys.g
        self.Fsolve = krylov._LU(sys.F)
        pin = sp.diags(np.concatenate([~g.q1_active, ~g.p0_active]).astype(float))
        k = sys.k
        aug = sp.bmat([[sys.MQ + pin, sp.csr_matrix(k[:, None])], [sp.csr_matrix(k[None, :]), None]])
        self.lu = krylov._LU(aug.tocsc())

    def __call__(self, r):
        s = self.sys
        nu_ = s.g.nu
        zp = -s.nu * self.lu(np.concatenate([r[nu_:], [0.0]]))[:-1]
        zu = self.Fsolve(r[:nu_] - s.BI.T @ zp)
        return np.concatenate([zu, zp])


def two_stage(sys, b, eta=1e-6, c=10.0, restart=50, maxit=2000):
    """The two-stage PCD method of Sec. 3.1 on the masked grid (Step I on the reduced Q1
    system with StepPCD1, Step II on the full system with StepM1)."""
    return krylov.two_stage(sys, b, eta, c, restart, maxit, pcd_cls=StepPCD1, m1_cls=StepM1)


class StepLSC:
    """The LSC preconditioner M_3 (Sec. 3.2, Eq. lsc-definition and nse-precon-lsc) on
    the masked grid, with H = M (plain LSC): both frame products B M^{-1} B^T are
    singular along k alone (outflow), inactive pressure unknowns keep identity rows."""

    def __init__(self, sys):
        from . import lsc
        self.sys = sys
        g = sys.g
        md = sys.Mv.diagonal()
        m = np.concatenate([md, md])
        self.minv = np.where(m > 0.0, 1.0 / np.where(m > 0.0, m, 1.0), 0.0)
        self.B = sys.BI
        pin = sp.diags(np.concatenate([~g.q1_active, ~g.p0_active]).astype(float))
        S = (self.B @ sp.diags(self.minv) @ self.B.T + pin).tocsr()
        self.BMB = lsc._ConstrainedSolve(S, sys.k[:, None])
        self.Fsolve = krylov._LU(sys.F)

    def schur_inv(self, rp):
        y = self.BMB(rp)
        t = self.B @ (self.minv * (self.sys.F @ (self.minv * (self.B.T @ y))))
        return self.BMB(t)

    def __call__(self, r):
        s = self.sys
        nu_ = s.g.nu
        zp = -self.schur_inv(r[nu_:])
        zu = self.Fsolve(r[:nu_] - s.BI.T @ zp)
        return np.concatenate([zu, zp])


def lsc_solve(sys, b, tol=1e-6, restart=50, maxit=2000):
    """GMRES with the right preconditioner M_3 (LSC) on the full masked-grid system from
    the lifted boundary data; stops at ||b - K x|| <= tol ||b||."""
    g = sys.g
    x0 = np.concatenate([sys.DB @ b[: g.nu], np.zeros(g.np_)])
    return krylov.gmres(lambda v: sys.K @ v, StepLSC(sys), b, x0, tol * np.linalg.norm(b), restart, maxit)


"""Seeded synthetic inputs for the enriched Taylor--Hood solvers.

This module holds no arithmetic of the solution method: it only draws random
parameters and evaluates analytic fields (stream functions, manufactured
solutions, lid data) at the Q2 lattice nodes.  Both the CUDA path and the CPU
oracle consume its output, so it must stay free of any discretisation code.

Node layout: the Q2 lattice of a uniform n x n grid on [x0,x1] x [y0,y1] has
(2n+1)^2 nodes, node (i, j) at (x0 + i*hx/2, y0 + j*hy/2), flat index
j*(2n+1) + i.  Vector fields are stored as [v_x (all nodes); v_y (all nodes)].

Workloads (all on [-1, 1]^2):
* ``cavity``      -- regularised lid-driven cavity (Sec. 2.4 Test problem 1 and
                     Sec. 3 Test problem 4): u = (1 - x^4, 0) on y = 1, zero on
                     the other walls, zero body force.
* ``mms``         -- manufactured smooth Stokes solution from a seeded sum of six
                     sine stream-function modes and a four-mode zero-mean
                     pressure, body force f = -nu lap u + grad p.
* ``oseen_wind``  -- divergence-free wind, the curl of an eight-mode sine stream
                     function vanishing on the boundary, scaled to unit maximum
                     nodal speed.
* ``batch``       -- 64 mixed Stokes/Oseen instances of uneven size and viscosity.
* ``diff``        -- the differentiation problem (Oseen 256^2, nu = 1/200).
* ``tridiagonal`` -- random symmetric tridiagonal coefficients (diagonal and
                     positive off-diagonal), the shape of a Lanczos record.
* ``step``        -- the flow over a step (Sec. 3, Test problem 3): the element
                     mask of D = [-1, 0) x [0, 1] U [0, 5] x [-1, 1] on the box
                     [-1, 5] x [-1, 1] with square elements of side 1/m, and the
                     parabolic inflow u = (4y(1 - y), 0) at x = -1.
* ``channel``     -- the channel [0, L] x [-1, 1] with the inflow (1 - y^2, 0).
"""
from __future__ import annotations

import numpy as np


def lattice(n, x0=-1.0, x1=1.0, y0=-1.0, y1=1.0):
    """Coordinates (X, Y) of the Q2 lattice nodes, flattened x-fastest."""
    N = 2 * n + 1
    xs = x0 + (x1 - x0) * np.arange(N) / (2 * n)
    ys = y0 + (y1 - y0) * np.arange(N) / (2 * n)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    return X.ravel(), Y.ravel()


def boundary_mask(n):
    N = 2 * n + 1
    m = np.zeros((N, N), dtype=bool)
    m[0, :] = m[-1, :] = m[:, 0] = m[:, -1] = True
    return m.ravel()


def sizes(n):
    """(N_v, n_u, n_k, n_0, N_t) for an n x n grid."""
    nv = (2 * n + 1) ** 2
    n1 = (n + 1) ** 2
    n0 = n * n
    return nv, 2 * nv, n1, n0, 2 * nv + n1 + n0


# ---------------------------------------------------------------------------
def cavity(n, nu=1.0):
    """Lid-driven cavity: u = (1 - x^4, 0) on the lid y = 1 (corners give 0)."""
    X, Y = lattice(n)
    nv = X.size
    ubc = np.zeros(2 * nv)
    top = np.isclose(Y, 1.0)
    ubc[:nv][top] = 1.0 - X[top] ** 4
    return {"name": f"cavity{n}", "n": n, "nu": float(nu), "wind": None,
            "f_nodal": np.zeros(2 * nv), "ubc": ubc}


class SineStream:
    """psi = sum_m a_m sin(k_m pi (x+1)/2) sin(l_m pi (y+1)/2) and its curl."""

    def __init__(self, a, k, l):
        self.a = np.asarray(a, dtype=np.float64)
        self.al = np.asarray(k, dtype=np.float64) * np.pi / 2.0
        self.be = np.asarray(l, dtype=np.float64) * np.pi / 2.0

    def velocity(self, x, y):
        """u = (d psi/dy, -d psi/dx)."""
        x = np.asarray(x)[..., None] + 1.0
        y = np.asarray(y)[..., None] + 1.0
        ux = np.sum(self.a * self.be * np.sin(self.al * x) * np.cos(self.be * y), axis=-1)
        uy = np.sum(-self.a * self.al * np.cos(self.al * x) * np.sin(self.be * y), axis=-1)
        return ux, uy

    def grad(self, x, y):
        """(dux/dx, dux/dy, duy/dx, duy/dy)."""
        x = np.asarray(x)[..., None] + 1.0
        y = np.asarray(y)[..., None] + 1.0
        a, al, be = self.a, self.al, self.be
        sx, cx, sy, cy = np.sin(al * x), np.cos(al * x), np.sin(be * y), np.cos(be * y)
        return (np.sum(a * be * al * cx * cy, -1), np.sum(-a * be * be * sx * sy, -1),
                np.sum(a * al * al * sx * sy, -1), np.sum(-a * al * be * cx * cy, -1))

    def laplacian(self, x, y):
        """Each sine mode is an eigenfunction: lap u = -(al^2 + be^2) u per mode."""
        x = np.asarray(x)[..., None] + 1.0
        y = np.asarray(y)[..., None] + 1.0
        a, al, be = self.a, self.al, self.be
        lam = -(al * al + be * be)
        lx = np.sum(lam * a * be * np.sin(al * x) * np.cos(be * y), -1)
        ly = np.sum(lam * -a * al * np.cos(al * x) * np.sin(be * y), -1)
        return lx, ly


class SinePressure:
    """p = sum_m b_m sin(pi k'_m x) cos(pi l'_m y) (zero mean on [-1,1]^2)."""

    def __init__(self, b, k, l):
        self.b = np.asarray(b, dtype=np.float64)
        self.k = np.asarray(k, dtype=np.float64) * np.pi
        self.l = np.asarray(l, dtype=np.float64) * np.pi

    def __call__(self, x, y):
        x = np.asarray(x)[..., None]; y = np.asarray(y)[..., None]
        return np.sum(self.b * np.sin(self.k * x) * np.cos(self.l * y), -1)

    def grad(self, x, y):
        x = np.asarray(x)[..., None]; y = np.asarray(y)[..., None]
        b, k, l = self.b, self.k, self.l
        return (np.sum(b * k * np.cos(k * x) * np.cos(l * y), -1),
                np.sum(-b * l * np.sin(k * x) * np.sin(l * y), -1))


def mms(n, seed=0, nu=1.0):
    """Manufactured Stokes solution (seeded), body force f = -nu lap u + grad p."""
    rng = np.random.default_rng(seed)
    k = rng.integers(1, 5, size=6)
    l = rng.integers(1, 5, size=6)
    a = rng.standard_normal(6) / (k * k + l * l)
    kp = rng.integers(1, 4, size=4)
    lp = rng.integers(1, 4, size=4)
    b = rng.standard_normal(4)
    psi = SineStream(a, k, l)
    pr = SinePressure(b, kp, lp)
    X, Y = lattice(n)
    ux, uy = psi.velocity(X, Y)
    lx, ly = psi.laplacian(X, Y)
    px, py = pr.grad(X, Y)
    f = np.concatenate([-nu * lx + px, -nu * ly + py])
    bnd = boundary_mask(n)
    ubc = np.concatenate([np.where(bnd, ux, 0.0), np.where(bnd, uy, 0.0)])
    return {"name": f"mms{n}", "n": n, "nu": float(nu), "wind": None, "f_nodal": f,
            "ubc": ubc, "u_exact": np.concatenate([ux, uy]),
            "exact": {"u": psi.velocity, "grad": psi.grad, "p": pr}}


def oseen_wind(n, seed=1, modes=8, kmax=6):
    """Unit-max-speed divergence-free wind from a seeded sine stream function."""
    rng = np.random.default_rng(seed)
    k = rng.integers(1, kmax + 1, size=modes)
    l = rng.integers(1, kmax + 1, size=modes)
    c = rng.standard_normal(modes)
    psi = SineStream(c, k, l)
    X, Y = lattice(n)
    wx, wy = psi.velocity(X, Y)
    s = np.sqrt(wx * wx + wy * wy).max()
    return np.concatenate([wx, wy]) / s


def oseen_cavity(n, nu=1.0 / 100.0, seed=1):
    """Oseen problem: cavity lid BCs, zero body force, seeded wind."""
    w = cavity(n, nu)
    w["name"] = f"oseen{n}"
    w["wind"] = oseen_wind(n, seed)
    return w


def batch(seed=2, count=64, sizes_choice=(32, 64, 128, 256)):
    """Uneven batch: n ~ U{sizes}, nu = 10^U(-3,-1), even i Stokes, odd i Oseen."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes_choice), size=count)
    nus = 10.0 ** rng.uniform(-3.0, -1.0, size=count)
    out = []
    for i in range(count):
        n = int(ns[i])
        nv = (2 * n + 1) ** 2
        fr = np.random.default_rng(seed * 100003 + i)
        f = fr.standard_normal(2 * nv)
        inst = {"name": f"batch{i}", "n": n, "nu": float(nus[i]), "f_nodal": f,
                "ubc": np.zeros(2 * nv),
                "wind": oseen_wind(n, 1000 + i) if i % 2 == 1 else None}
        out.append(inst)
    return out


def diff(n=256, nu=1.0 / 200.0):
    """Differentiation problem: Oseen cavity, smooth body force and target field."""
    w = cavity(n, nu)
    w["name"] = f"diff{n}"
    w["wind"] = oseen_wind(n, 3)
    f = mms(n, seed=4)
    w["f_nodal"] = f["u_exact"].copy()
    w["u_target"] = mms(n, seed=5)["u_exact"].copy()
    return w


def tridiagonal(k, seed=0):
    """(delta, gamma): k diagonal entries uniform on [-1, 2] and k off-diagonal
    entries uniform on [0.05, 1] (gamma[j-1] couples rows j and j+1; the last one
    sits below a k x k block)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 2.0, k), rng.uniform(0.05, 1.0, k)


def _box_lattice(nx, ny, h, x0, y0):
    xs = x0 + 0.5 * h * np.arange(2 * nx + 1)
    ys = y0 + 0.5 * h * np.arange(2 * ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    return X.ravel(), Y.ravel()


def _inflow(nx, ny, h, x0, y0, active, profile):
    """u = (profile(y), 0) on the nodes of the box's left edge that touch an active
    element (the inflow boundary), zero elsewhere."""
    X, Y = _box_lattice(nx, ny, h, x0, y0)
    N = 2 * nx + 1
    ub = np.zeros(2 * X.size)
    act = np.asarray(active, dtype=bool).reshape(ny, nx)
    for j in range(2 * ny + 1):
        eys = [j // 2] if j % 2 else [j // 2 - 1, j // 2]
        if any(0 <= ey < ny and act[ey, 0] for ey in eys):
            ub[j * N] = profile(Y[j * N])
    return ub


def step(m, nu=1.0 / 50.0):
    """The step problem with h = 1/m: nx = 6m, ny = 2m elements on [-1, 5] x [-1, 1]."""
    nx, ny, h = 6 * m, 2 * m, 1.0 / m
    xc = -1.0 + h * (np.arange(nx) + 0.5)
    yc = -1.0 + h * (np.arange(ny) + 0.5)
    XC, YC = np.meshgrid(xc, yc, indexing="xy")
    active = ~((XC < 0.0) & (YC < 0.0))
    ubc = _inflow(nx, ny, h, -1.0, -1.0, active, lambda y: 4.0 * y * (1.0 - y))
    return {"nx": nx, "ny": ny, "h": h, "x0": -1.0, "y0": -1.0, "active": active, "nu": float(nu), "ubc": ubc,
            "outflow": True}


def channel(m, length=2.0, nu=0.02):
    """[0, length] x [-1, 1] with h = 1/m, inflow u = (1 - y^2, 0) at x = 0, outflow at x = length."""
    nx, ny, h = int(round(length * m)), 2 * m, 1.0 / m
    active = np.ones((ny, nx), dtype=bool)
    ubc = _inflow(nx, ny, h, 0.0, -1.0, active, lambda y: 1.0 - y ** 2)
    return {"nx": nx, "ny": ny, "h": h, "x0": 0.0, "y0": -1.0, "active": active, "nu": float(nu), "ubc": ubc,
            "outflow": True}

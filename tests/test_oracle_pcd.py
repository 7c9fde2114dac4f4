"""Pins of the oracle's Q1 pressure convection-diffusion (PCD) Schur block.

Sec. 3.1 derives the Step I Schur approximation from the commutator statement
(Eq. discrete-commutator1): when (Q1^{-1} B1)(M^{-1} F) equals
(Q1^{-1} F1)(Q1^{-1} B1), with M the diagonal of the velocity mass matrix, the
rearrangement B1 F^{-1} B1^T = Q1 F1^{-1} (B1 M^{-1} B1^T) (Eq.
discrete-commutator1x) is exact algebra.  So on a problem built to have a zero
commutator, M_S^{-1} = Ap^+ F1 Q1^{-1} must invert the true Schur complement
S1 = B1 F^{-1} B1^T exactly.  That fixes the order of the three factors, the
mass diagonal inside Ap and the interior-column restriction of B1: a swapped
order, a lumped (row-sum) mass or a B1 with boundary columns fails it.  The
convection-diffusion matrix F1 itself is pinned separately against the weak
form nu (grad phi_j, grad phi_i) + (w . grad phi_j, phi_i) of the paper,
integrated exactly for a linear wind; a missing convection term, a sign flip or
a missing viscosity fails that one.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import sympy

from oracle import fem, krylov, problem
from paper_2303_10233_gb300 import workloads as W

xs, ys = sympy.symbols("x y")


def _interior_velocity(g):
    return np.concatenate([~g.bnd, ~g.bnd])


def _zero_commutator_case(n, seed):
    """An Oseen system whose F and F1 make the discrete commutator vanish.

    F1 = Q1 G_p with G_p = 3 I + 0.5 P R (P the Euclidean projector orthogonal to
    q = Q1 1, so G_p^T q = 3 q and Q1 G_p Q1^{-1} maps mean-free vectors to
    mean-free vectors).  On the interior velocity unknowns F = M G_v with
    G_v = B^+ (Q1 G_p Q1^{-1} B) + (I - B^+ B), so that B G_v = Q1 G_p Q1^{-1} B,
    which is B M^{-1} F = F1 Q1^{-1} B: the commutator of Eq. discrete-commutator1
    is zero."""
    w = W.oseen_cavity(n, nu=1 / 50, seed=1)
    g = fem.Grid(n)
    s = problem.System(g, w["nu"], w["wind"])
    I = _interior_velocity(g)
    Bh = s.B1I.toarray()[:, I]
    md = s.Mv.diagonal()
    Mh = np.diag(np.concatenate([md, md])[I])
    Q1 = s.Qk.toarray()
    q = Q1 @ np.ones(g.n1)
    rng = np.random.default_rng(seed)
    P = np.eye(g.n1) - np.outer(q, q) / (q @ q)
    Gp = 3.0 * np.eye(g.n1) + 0.5 * P @ rng.standard_normal((g.n1, g.n1))
    F1 = Q1 @ Gp
    Bp = np.linalg.pinv(Bh)
    Gv = Bp @ (Q1 @ Gp @ np.linalg.solve(Q1, Bh)) + (np.eye(Bh.shape[1]) - Bp @ Bh)
    Fh = Mh @ Gv
    return s, Bh, Mh, Q1, F1, Fh


@pytest.mark.parametrize("n", [2, 4])
def test_pcd_exact_when_commutator_vanishes(n):
    s, Bh, Mh, Q1, F1, Fh = _zero_commutator_case(n, seed=n)
    # the construction: (Q1^-1 B1)(M^-1 F) - (Q1^-1 F1)(Q1^-1 B1) = 0
    C = np.linalg.solve(Q1, Bh) @ np.linalg.solve(Mh, Fh) - np.linalg.solve(Q1, F1) @ np.linalg.solve(Q1, Bh)
    assert abs(C).max() < 1e-9 * abs(np.linalg.solve(Q1, Bh)).max() * abs(np.linalg.solve(Mh, Fh)).max()
    S1 = Bh @ np.linalg.solve(Fh, Bh.T)            # the true Schur complement of Step I
    pcd = krylov.PCD1(s)
    pcd.F1 = sp.csr_matrix(F1)
    rng = np.random.default_rng(10 + n)
    for _ in range(3):
        y = rng.standard_normal(s.g.n1)
        y -= y.mean()
        z = pcd.schur_inv(S1 @ y)
        assert np.linalg.norm((z - z.mean()) - y) < 1e-8 * np.linalg.norm(y)
    # planted mistakes in the composition fail the same identity
    y = rng.standard_normal(s.g.n1)
    y -= y.mean()
    r = S1 @ y
    swapped = pcd.Q1solve(pcd.F1 @ pcd.Apsolve(r))           # Q1^-1 F1 Ap^-1
    assert np.linalg.norm((swapped - swapped.mean()) - y) > 1e-3 * np.linalg.norm(y)
    ml = np.asarray(s.Mv.sum(axis=1)).ravel()                  # lumped (row-sum) mass
    Ap_l = (s.B1I @ sp.diags(np.concatenate([1 / ml, 1 / ml])) @ s.B1I.T).tocsr()
    lumped = krylov.NullSolve(Ap_l)(pcd.F1 @ pcd.Q1solve(r))
    assert np.linalg.norm(lumped - y) > 1e-3 * np.linalg.norm(y)
    Ap_b = (s.B1 @ sp.diags(1 / np.concatenate([s.Mv.diagonal()] * 2)) @ s.B1.T).tocsr()
    bcols = krylov.NullSolve(Ap_b)(pcd.F1 @ pcd.Q1solve(r))   # boundary velocity columns kept
    assert np.linalg.norm(bcols - y) > 1e-3 * np.linalg.norm(y)


def test_pcd_f1_is_the_pressure_convection_diffusion_form():
    dom = (-1.0, 1.0, -1.0, 1.0)
    n, nu = 3, 0.37
    g = fem.Grid(n, *dom)
    wx, wy = 0.6 + 0.4 * ys - 0.3 * xs, -0.2 + 0.5 * xs + 0.1 * ys
    nod = lambda e, X, Y: np.array([float(e.subs({xs: a, ys: b})) for a, b in zip(X, Y)])
    wind = np.concatenate([nod(wx, g.X2, g.Y2), nod(wy, g.X2, g.Y2)])
    s = problem.System(g, nu, wind)
    pcd = krylov.PCD1(s)
    P = 1 + xs - 2 * xs * ys
    Qf = 2 - ys + xs * ys
    p, qv = nod(P, g.X1, g.Y1), nod(Qf, g.X1, g.Y1)
    form = nu * (sympy.diff(P, xs) * sympy.diff(Qf, xs) + sympy.diff(P, ys) * sympy.diff(Qf, ys)) + \
        (wx * sympy.diff(Qf, xs) + wy * sympy.diff(Qf, ys)) * P
    exact = float(sympy.integrate(sympy.integrate(form, (xs, -1, 1)), (ys, -1, 1)))
    assert abs(p @ (pcd.F1 @ qv) - exact) < 1e-11 * max(1.0, abs(exact))
    # Md of Ap is the diagonal of the consistent velocity mass (the Sec. 3.1 footnote)
    md = s.Mv.diagonal()
    Ap = (s.B1I @ sp.diags(np.concatenate([1 / md, 1 / md])) @ s.B1I.T).toarray()
    assert abs(pcd.Ap.toarray() - Ap).max() < 1e-13 * abs(Ap).max()


def test_pcd_step1_not_slower_under_refinement():
    """Sec. 3.1: the Step I residual reduction is robust under refinement (typically
    fewer steps on finer grids).  Exact blocks, the Oseen cavity, nu = 1/50."""
    its = []
    for n in (8, 16, 32):
        w = W.oseen_cavity(n, nu=1 / 50, seed=1)
        g = fem.Grid(n)
        s = problem.System(g, w["nu"], w["wind"])
        b = s.rhs(w["f_nodal"], w["ubc"])
        _, info = krylov.two_stage(s, b, eta=1e-6, c=10.0, restart=200, maxit=400)
        its.append(info["its1"])
    assert max(its) - min(its) <= 3, its

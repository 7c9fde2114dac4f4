"""Pins of the oracle's solvers: exact solutions, convergence rates, theory.

* MMS: textbook Q2-Q1 rates (L2 velocity h^3, H1 velocity h^2, L2 pressure h^2)
  for the direct solve; element-wise mass conservation (Sec. 2.1).
* MINRES (Algorithm 1): with P_ideal (Sec. 2) the preconditioned matrix has the
  three nonzero eigenvalues 1, (1 +- sqrt 5)/2, so MINRES ends in 3 steps;
  with P_1 it reproduces the direct solution and its count is flat in n
  (Tables 1 and 3 pattern).
* GMRES: with the exact Schur complement the block-triangular preconditioned
  operator has a degree-2 minimal polynomial, so GMRES ends in 2 steps.
* Two-stage PCD (Sec. 3.1): Prop. 2 bound at the switch; final residual <= eta.
* Adjoint: gradients match central finite differences.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import adjoint, direct, fem, krylov, problem
from paper_2303_10233_gb300 import workloads as W


def _system(w):
    g = fem.Grid(w["n"])
    s = problem.System(g, w["nu"], w["wind"])
    return g, s, s.rhs(w["f_nodal"], w["ubc"])


def test_mms_convergence_rates_and_conservation():
    errs = []
    for n in (8, 16, 32):
        w = W.mms(n, seed=0)
        g, s, b = _system(w)
        x, lam = direct.solve(s, b)
        assert np.linalg.norm(b - s.K @ x) < 1e-12 * np.linalg.norm(b)
        assert abs(lam).max() < 1e-12
        u, p = x[: g.nu], x[g.nu:]
        ex = w["exact"]
        errs.append(fem.l2_h1_errors(g, u, p, ex["u"], ex["grad"], ex["p"]))
        # element-wise conservation: int_T div u_h = 0 (boundary data lifted exactly)
        assert abs(fem.element_divergence(g, u)).max() < 1e-12
    errs = np.array(errs)
    r = errs[:-1] / errs[1:]
    assert np.all(r[:, 0] > 7.0) and np.all(r[:, 0] < 9.5), r
    assert np.all(r[:, 1] > 3.6) and np.all(r[:, 1] < 4.5), r
    assert np.all(r[:, 2] > 3.5) and np.all(r[:, 2] < 5.5), r


def test_rhs_is_consistent_for_enclosed_flow():
    for w in (W.cavity(8), W.mms(8), W.oseen_cavity(8)):
        g, s, b = _system(w)
        assert abs(b[g.nu: g.nu + g.n1].sum()) < 1e-13
        assert abs(b[g.nu + g.n1:].sum()) < 1e-13


@pytest.mark.parametrize("n", [4, 8])
def test_minres_ideal_preconditioner_three_steps(n):
    g, s, b = _system(W.cavity(n))
    x0 = np.concatenate([s.DB @ b[: g.nu], np.zeros(g.np_)])
    x, info = krylov.minres(lambda v: s.K @ v, krylov.PIdeal(s), b, x0, tol=1e-12, maxit=10)
    assert info["its"] <= 3
    assert info["eta"][3] < 1e-10 * info["eta"][0]


def test_minres_p1_matches_direct_and_is_mesh_independent():
    its = []
    for n in (4, 8, 16, 32):
        g, s, b = _system(W.cavity(n))
        xd, _ = direct.solve(s, b)
        x0 = np.concatenate([s.DB @ b[: g.nu], np.zeros(g.np_)])
        x, info = krylov.minres(lambda v: s.K @ v, krylov.P1(s), b, x0, tol=1e-10)
        its.append(info["its"])
        assert np.linalg.norm(s.canonical(x) - xd) < 1e-7 * np.linalg.norm(xd)
        h = np.array(info["eta"])
        assert np.all(np.diff(h) <= 1e-12 * h[0])          # |eta| is non-increasing
    assert max(its) - min(its) <= 8, its


def test_gmres_exact_schur_two_steps():
    g, s, b = _system(W.oseen_cavity(4, nu=0.05))
    F = s.F.toarray()
    BI = s.BI.toarray()
    S = BI @ np.linalg.solve(F, BI.T)
    Spinv = np.linalg.pinv(S, rcond=1e-10)

    def Minv(r):
        zp = -Spinv @ r[g.nu:]
        return np.concatenate([np.linalg.solve(F, r[: g.nu] - BI.T @ zp), zp])

    x0 = np.concatenate([s.DB @ b[: g.nu], np.zeros(g.np_)])
    x, info = krylov.gmres(lambda v: s.K @ v, Minv, b, x0, 1e-10 * np.linalg.norm(b), restart=10, maxit=10)
    assert info["its"] <= 2
    xd, _ = direct.solve(s, b)
    assert np.linalg.norm(s.canonical(x) - xd) < 1e-8 * np.linalg.norm(xd)


def test_two_stage_prop2_and_accuracy():
    for n in (8, 16):
        g, s, b = _system(W.oseen_cavity(n, nu=1 / 100))
        eta = 1e-8
        x, info = krylov.two_stage(s, b, eta=eta, c=10.0)
        assert np.linalg.norm(b - s.K @ x) <= eta * np.linalg.norm(b) * 1.0001
        assert info["z_star_sq"] <= info["prop2_bound"] * (1 + 1e-9)
        xd, _ = direct.solve(s, b)
        assert np.linalg.norm(s.canonical(x) - xd) < 1e-5 * np.linalg.norm(xd)


def test_adjoint_gradients_match_central_differences():
    n = 6
    w = W.diff(n, nu=1 / 200)
    g = fem.Grid(n)
    s = problem.System(g, w["nu"], w["wind"])
    J, gf, gnu, _ = adjoint.gradients(s, w["f_nodal"], w["ubc"], w["u_target"])
    rng = np.random.default_rng(7)
    eps = 1e-4
    for _ in range(3):
        d = rng.standard_normal(g.nu); d /= np.linalg.norm(d)
        Jp = adjoint.fd_objective(g, w["nu"], w["wind"], w["f_nodal"] + eps * d, w["ubc"], w["u_target"])
        Jm = adjoint.fd_objective(g, w["nu"], w["wind"], w["f_nodal"] - eps * d, w["ubc"], w["u_target"])
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - gf @ d) <= 1e-6 * max(1.0, abs(fd))
    h = 1e-4 * w["nu"]                                # relative step in nu
    Jp = adjoint.fd_objective(g, w["nu"] + h, w["wind"], w["f_nodal"], w["ubc"], w["u_target"])
    Jm = adjoint.fd_objective(g, w["nu"] - h, w["wind"], w["f_nodal"], w["ubc"], w["u_target"])
    fd = (Jp - Jm) / (2 * h)
    assert abs(fd - gnu) <= 1e-5 * abs(fd)


def test_batch_workload_totals():
    insts = W.batch()
    assert len(insts) == 64
    tot = sum(W.sizes(i["n"])[4] for i in insts)
    assert 5e6 < tot < 30e6
    assert all(i["wind"] is None for i in insts[0::2])
    assert all(i["wind"] is not None for i in insts[1::2])


def test_picard_pins():
    """Picard iteration (Sec. 3): the first step with zero wind is the Stokes solution;
    at a low Reynolds number the iteration contracts, its nonlinear residual falls
    monotonically to roundoff, and the limit satisfies the discrete Navier-Stokes
    equations K(u) x = b(u) with the wind equal to its own velocity."""
    from oracle import picard
    from paper_2303_10233_gb300 import workloads as W
    n = 8
    w = W.cavity(n, nu=0.2)
    g = fem.Grid(n)
    xs, res = picard.picard(g, w["nu"], w["f_nodal"], w["ubc"], 14)
    s0 = problem.System(g, w["nu"])
    xst, _ = direct.solve(s0, s0.rhs(w["f_nodal"], w["ubc"]))
    assert np.linalg.norm(xs[0] - xst) <= 1e-12 * np.linalg.norm(xst)
    assert all(b < a for a, b in zip(res[:10], res[1:11]))
    assert res[-1] <= 1e-11 < res[0]
    # at the limit, one more Oseen solve with the limit's own wind reproduces it
    s = problem.System(g, w["nu"], xs[-1][: g.nu].copy())
    x1, _ = direct.solve(s, s.rhs(w["f_nodal"], w["ubc"]))
    assert np.linalg.norm(s.canonical(x1) - xs[-1]) <= 1e-9 * np.linalg.norm(xs[-1])


@pytest.mark.parametrize("w", [W.mms(8, seed=0), W.oseen_cavity(16, nu=1 / 200, seed=1)])
def test_pinned_direct_solve_equals_bordered(w):
    """The pinned-pressure factorisation used at the larger test grids returns the same
    canonical solution as the bordered solve (unique modulo span{e1, e0})."""
    g, s, b = _system(w)
    xb, _ = direct.solve(s, b)
    xp = direct.solve_pinned(s, b)
    assert np.linalg.norm(xp - xb) <= 1e-10 * np.linalg.norm(xb)
    assert np.linalg.norm(b - s.K @ xp) <= 1e-12 * np.linalg.norm(b)

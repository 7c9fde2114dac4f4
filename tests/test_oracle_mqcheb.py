"""Pins of the oracle's Chebyshev-SGS approximation of M_Q (the M_cheb block of P_2).

* Chebyshev semi-iteration: for r = M v with M v = lam P v, the residual after k
  steps is exactly T_k((theta - lam)/delta) / T_k(theta/delta) r (Chebyshev
  polynomials evaluated by a library routine, not by the recurrence).
* SGS: the sweep implementation equals (D + L) D^{-1} (D + L^T) in the colour order;
  each colour is an independent set of M_Q (so a multicolour sweep is exact); the
  eigenvalues of P^{-1} M_Q lie in [0, 1] with the single zero along k.
* Many steps reproduce M_Q^+ (k projected out).
* The paper's statements: the smallest nonzero SGS eigenvalue falls like h^2 (the
  largest non-unit eigenvalue of the iteration matrix tends to 1), so MINRES with
  P_2 degrades under refinement and its inf-sup estimate with it, while on a coarse
  grid P_2 behaves like P_1.
"""
import numpy as np
import pytest
import scipy.linalg as sla
from numpy.polynomial import chebyshev as C

from oracle import fem, infsup, krylov, mqcheb, problem
from paper_2303_10233_gb300 import workloads as W


def test_chebyshev_residual_polynomial():
    rng = np.random.default_rng(0)
    n = 12
    X = rng.standard_normal((n, n))
    M = X @ X.T + n * np.eye(n)
    Lo = np.tril(M)
    D = np.diag(np.diag(M))
    P = Lo @ np.linalg.solve(D, Lo.T)
    lam, V = sla.eigh(M, P)
    a, b = lam.min() * 0.9, lam.max() * 1.05
    theta, delta = 0.5 * (b + a), 0.5 * (b - a)
    for idx in (0, 5, n - 1):
        r = M @ V[:, idx]
        for k in (1, 5, 20):
            x = mqcheb.chebyshev(lambda v: M @ v, lambda v: np.linalg.solve(P, v), r, a, b, k)
            e = np.zeros(k + 1); e[k] = 1.0
            Rk = C.chebval((theta - lam[idx]) / delta, e) / C.chebval(theta / delta, e)
            assert np.allclose(r - M @ x, Rk * r, rtol=1e-9, atol=1e-11 * np.abs(r).max())


def test_sgs_sweeps_and_colours():
    g = fem.Grid(6)
    s = problem.System(g, 1.0)
    order = mqcheb.colour_order(g)
    assert np.array_equal(np.sort(order), np.arange(g.np_))
    Mp = s.MQ.toarray()[np.ix_(order, order)]
    # every colour is an independent set: its diagonal block is diagonal
    I = np.arange(g.n1) % (g.n + 1); J = np.arange(g.n1) // (g.n + 1)
    sizes = [np.count_nonzero((I % 2 == ci) & (J % 2 == cj)) for cj in (0, 1) for ci in (0, 1)] + [g.n0]
    start = 0
    for sz in sizes:
        blk = Mp[start:start + sz, start:start + sz]
        assert np.count_nonzero(blk - np.diag(np.diag(blk))) == 0
        start += sz
    Lo = np.tril(Mp)
    P = Lo @ np.linalg.solve(np.diag(np.diag(Mp)), Lo.T)
    sgs = mqcheb.SGS(s.MQ, order)
    r = np.random.default_rng(2).standard_normal(g.np_)
    z = sgs(r)
    assert np.allclose(z[order], np.linalg.solve(P, r[order]), rtol=1e-12, atol=1e-12 * np.abs(z).max())
    lam = np.sort(sla.eigh(Mp, P, eigvals_only=True))
    assert abs(lam[0]) <= 1e-12 and lam[1] > 0.0 and lam[-1] <= 1.0 + 1e-12


def test_many_steps_reproduce_mq_pseudoinverse():
    g = fem.Grid(8)
    s = problem.System(g, 0.5)
    r = np.random.default_rng(3).standard_normal(g.np_)
    ex = s.nu * krylov.MQSolve(s)(r - (s.k @ r) / (s.k @ s.k) * s.k)
    got = mqcheb.MCheb(s, 300)(r)
    assert np.linalg.norm(got - ex) <= 1e-10 * np.linalg.norm(ex)
    assert abs(s.k @ got) <= 1e-12 * np.linalg.norm(got)


def test_sgs_interval_falls_like_h2():
    a = [mqcheb.sgs_interval(fem.Grid(n))[0] for n in (4, 8, 16)]
    assert 3.0 <= a[0] / a[1] <= 5.0 and 3.0 <= a[1] / a[2] <= 5.0, a


def test_p2_degrades_under_refinement():
    res = {}
    for n in (4, 16):
        w = W.cavity(n)
        g = fem.Grid(n)
        s = problem.System(g, w["nu"])
        b = s.rhs(w["f_nodal"], w["ubc"])
        x0 = np.concatenate([s.DB @ b[: g.nu], np.zeros(g.np_)])
        for name, P in (("p1", krylov.P1(s)), ("p2", mqcheb.P2Exact(s, 20))):
            _, info = krylov.minres(lambda v: s.K @ v, P, s.project_rhs(b), x0, tol=1e-8, maxit=1000)
            res[(n, name)] = (info["its"], infsup.est_history(info["delta"], info["gamma"])[-1])
    (i1, e1), (i2, e2) = res[(4, "p1")], res[(4, "p2")]
    assert abs(i1 - i2) <= 1 and abs(e1 - e2) <= 0.01 * e1
    (i1, e1), (i2, e2) = res[(16, "p1")], res[(16, "p2")]
    assert i2 >= i1 + 5 and e2 <= 0.9 * e1, res

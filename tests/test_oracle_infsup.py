"""Pins of the oracle's inf-sup constant and EST-MINRES estimate (Sec. 2.4).

* Closed forms: for K = [A B^T; B 0] with diagonal A, B = [diag(b) 0] and the
  preconditioner blkdiag(A, M), M diagonal, the pencil eigenvalues are
  sigma_i = b_i^2 / (a_i m_i); EST-MINRES must reach min sigma_i, from above.
* The harmonic Ritz values from the Lanczos scalars equal those of the
  Petrov-Galerkin condition (M V y - theta V y) orthogonal to M V, solved on an
  explicit Krylov basis built by repeated multiplication.
* The FEM pencil: one zero eigenvalue (the hydrostatic mode), all others in
  (0, 1] (for u in H^1_0, ||div u|| <= |u|_1), the largest tending to 1; the
  dense gamma^2 agrees with the EST-MINRES estimate of preconditioned MINRES with
  the exact P_1, which reaches it from above within about 25 iterations.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import fem, infsup, krylov, problem
from paper_2303_10233_gb300 import workloads as W


def _synthetic(nu_, npr, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.5, 2.0, nu_)
    bb = rng.uniform(0.3, 1.2, npr)
    m = rng.uniform(0.5, 2.0, npr)
    B = np.zeros((npr, nu_))
    B[np.arange(npr), np.arange(npr)] = bb
    K = np.block([[np.diag(a), B.T], [B, np.zeros((npr, npr))]])
    pdiag = np.concatenate([a, m])
    rhs = rng.standard_normal(nu_ + npr)
    return K, pdiag, rhs, bb ** 2 / (a[:npr] * m)


def test_est_closed_form_from_above():
    K, pdiag, rhs, sigma = _synthetic(30, 20, 3)
    x, info = krylov.minres(lambda v: K @ v, lambda r: r / pdiag, rhs, np.zeros(len(rhs)), tol=1e-14,
                            maxit=200)
    h = infsup.est_history(info["delta"], info["gamma"])
    g2 = sigma.min()
    fin = h[np.isfinite(h)]
    assert fin.size > 0
    assert np.all(fin >= g2 * (1 - 1e-9)), (fin.min(), g2)
    assert abs(h[-1] - g2) <= 1e-8 * g2, (h[-1], g2)


def test_harmonic_ritz_matches_petrov_galerkin():
    K, pdiag, rhs, _ = _synthetic(12, 8, 5)
    P = np.diag(pdiag)
    x, info = krylov.minres(lambda v: K @ v, lambda r: r / pdiag, rhs, np.zeros(len(rhs)), tol=1e-14)
    M = np.linalg.solve(P, K)
    z = rhs / pdiag
    for k in (2, 3, 5):
        cols = [z]
        for _ in range(k - 1):
            cols.append(M @ cols[-1])
        V, _ = np.linalg.qr(np.array(cols).T)
        MV = M @ V
        th = sla.eig(MV.T @ P @ MV, MV.T @ P @ V, right=False)
        ref = np.sort(th.real)
        got = infsup.harmonic_ritz(info["delta"], info["gamma"], k)
        assert got.shape == ref.shape
        assert np.allclose(got, ref, rtol=1e-8, atol=1e-10), (k, got, ref)


@pytest.mark.parametrize("n", [4, 8])
def test_dense_pencil_spectrum(n):
    g = fem.Grid(n)
    g2, sig = infsup.dense_gamma2(g)
    assert sig.size == g.n1 + g.n0 - 1
    assert abs(sig[0]) <= 1e-12                     # hydrostatic mode
    assert sig[1] > 0.1 and g2 == sig[1]
    assert sig[-1] <= 1.0 + 1e-12                   # ||div u|| <= |u|_1 on H^1_0
    assert sig[-1] >= 0.99
    s = problem.System(g, 1.0)
    assert np.abs(s.BI.T @ s.e1[g.nu:]).max() <= 1e-12   # constants are in ker B^T
    assert np.abs(s.BI.T @ s.e0[g.nu:]).max() <= 1e-12


def test_largest_pencil_eigenvalue_tends_to_one():
    tops = [infsup.dense_gamma2(fem.Grid(n))[1][-1] for n in (4, 8)]
    assert tops[0] < tops[1] <= 1.0 + 1e-12
    assert 1.0 - tops[1] < 0.25 * (1.0 - tops[0])


@pytest.mark.parametrize("n", [4, 8])
def test_est_minres_exact_p1_reaches_dense_gamma2(n):
    w = W.cavity(n)
    g = fem.Grid(n)
    s = problem.System(g, w["nu"])
    b = s.rhs(w["f_nodal"], w["ubc"])
    x, info = krylov.minres(lambda v: s.K @ v, krylov.P1(s), b, np.zeros(g.nt), tol=1e-10)
    h = infsup.est_history(info["delta"], info["gamma"])
    g2, _ = infsup.dense_gamma2(g)
    fin = h[np.isfinite(h)]
    assert np.all(fin >= g2 * (1 - 1e-8))
    assert abs(h[-1] - g2) <= 1e-6 * g2, (h[-1], g2)
    assert abs(h[min(24, len(h) - 1)] - g2) <= 1e-2 * g2


def test_est_nan_before_negative_ritz_value():
    # one Lanczos step on a positive 1x1 block: no negative harmonic Ritz value
    assert np.isnan(infsup.est_gamma2([2.0], [1.0, 0.5], 1))
    # delta = -1, gamma_2 = 0: theta = -1 exactly, gamma^2 = 2
    assert infsup.est_gamma2([-1.0], [1.0, 0.0], 1) == pytest.approx(2.0, rel=1e-14)

"""Pins of the oracle's least-squares commutator preconditioner (Sec. 3.2).

* Exactness when F is a multiple of the diagonal mass: with F = c M the LSC
  formula collapses to (1/c) B M^{-1} B^T = B F^{-1} B^T, for any diagonal D.
* The middle factor is the least-squares commutator: with D = I,
  M_S^{-1} (B M^{-1} B^T) y = X y where X minimises ||M^{-1/2}(F M^{-1} B^T - B^T X)||
  (solved column by column with a least-squares routine on the dense matrices).
* The wall weights of D sit on the tangential component at the nodes next to a wall.
* The paper's remark that LSC works for Q2-Q1*: GMRES with M_3 on the Oseen cavity
  needs nearly mesh-independent iteration counts, fewer than with M_1.
"""
import copy

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, krylov, lsc, problem
from paper_2303_10233_gb300 import workloads as W


def _system(n, nu=0.01):
    w = W.oseen_cavity(n, nu=nu, seed=1)
    g = fem.Grid(n)
    return g, problem.System(g, w["nu"], w["wind"]), w


def _complement(g, rng):
    s = problem.System(g, 1.0)
    E = np.column_stack([s.e1[g.nu:], s.e0[g.nu:]])
    Q, _ = np.linalg.qr(E)
    r = rng.standard_normal(g.np_)
    return r - Q @ (Q.T @ r)


@pytest.mark.parametrize("omega", [1.0, 10.0])
def test_exact_for_scaled_mass(omega):
    g, s, _ = _system(6)
    md = s.Mv.diagonal()
    m = np.concatenate([md, md])
    c = 3.7
    intr = np.concatenate([~g.bnd, ~g.bnd]).astype(float)
    s2 = copy.copy(s)
    s2.F = sp.diags(c * m * intr + (1.0 - intr)).tocsr()   # identity Dirichlet rows
    P = lsc.LSC(s2, omega)
    B = s.BI.toarray()
    S = B @ np.diag(1.0 / (c * m)) @ B.T                  # B F^{-1} B^T
    Sp = np.linalg.pinv(S, rcond=1e-10, hermitian=True)
    rng = np.random.default_rng(0)
    for _ in range(3):
        r = _complement(g, rng)
        assert np.allclose(P.schur_inv(r), Sp @ r, rtol=1e-9, atol=1e-9 * np.abs(Sp @ r).max())


@pytest.mark.parametrize("omega", [1.0, 10.0])
def test_middle_factor_is_least_squares_commutator(omega):
    """X minimises the M^{-1}-weighted ||F H^{-1} B^T - B^T X|| and M_S^{-1} = X (B H^{-1} B^T)^+;
    with omega != 1 this also fixes the order of the two outer factors."""
    g, s, _ = _system(4)
    P = lsc.LSC(s, omega)
    md = s.Mv.diagonal()
    m = np.concatenate([md, md])
    hinv = lsc.tangential_weights(g, omega) / m
    B = s.BI.toarray()
    F = s.F.toarray()
    intr = np.concatenate([~g.bnd, ~g.bnd])
    Wr = np.diag(1.0 / np.sqrt(m))[intr]
    A_ls = Wr @ B.T
    R_ls = Wr @ F @ np.diag(hinv) @ B.T
    X = np.linalg.lstsq(A_ls, R_ls, rcond=None)[0]
    BHB = B @ np.diag(hinv) @ B.T
    rng = np.random.default_rng(1)
    for _ in range(3):
        y = _complement(g, rng)
        got = P.schur_inv(BHB @ y)
        ref = X @ y
        assert np.allclose(got, ref, rtol=1e-8, atol=1e-10 * np.abs(ref).max())


def test_tangential_weights():
    g = fem.Grid(2)                  # 5 x 5 Q2 nodes, interior 3 x 3
    d = lsc.tangential_weights(g, 7.0)
    dx, dy = d[: g.nv].reshape(5, 5), d[g.nv:].reshape(5, 5)   # [j, i]
    ex = np.ones((5, 5)); ex[1, 1:4] = 7.0; ex[3, 1:4] = 7.0
    ey = np.ones((5, 5)); ey[1:4, 1] = 7.0; ey[1:4, 3] = 7.0
    assert np.array_equal(dx, ex) and np.array_equal(dy, ey)


def test_lsc_gmres_mesh_robust_and_better_than_m1():
    its, its_m1 = [], []
    for n in (8, 16, 32):
        g, s, w = _system(n, nu=0.01)
        b = s.rhs(w["f_nodal"], w["ubc"])
        x, info = lsc.solve(s, b, tol=1e-6, restart=200)
        bp = s.project_rhs(b)
        assert np.linalg.norm(bp - s.K @ x) <= 1e-6 * np.linalg.norm(bp) * 1.0001
        its.append(info["its"])
        x0 = np.concatenate([s.DB @ b[: g.nu], np.zeros(g.np_)])
        _, info1 = krylov.gmres(lambda v: s.K @ v, krylov.M1(s), bp, x0, 1e-6 * np.linalg.norm(bp), 200, 2000)
        its_m1.append(info1["its"])
    assert max(its) <= 40 and its[-1] <= 1.5 * its[0], its
    assert all(a < b for a, b in zip(its, its_m1)), (its, its_m1)


@pytest.mark.parametrize("n", [4, 8])
def test_frame_operator_blocks_are_laplacians(n):
    """The LSC solves with S = B M^{-1} B^T on the frame: its exact block-diagonal part is
    a mesh-independent preconditioner, and the blocks are spectrally equivalent to the
    Q1 Laplacian (Q1 block) and to the cell-centred 5-point Laplacian (P0 block), so each
    can be replaced by a Laplacian V-cycle (the basis of a multigrid LSC solve)."""
    import scipy.linalg as sla
    g = fem.Grid(n)
    s = problem.System(g, 1.0)
    md = s.Mv.diagonal()
    m = np.concatenate([md, md])
    B = s.BI.toarray()
    S = B @ np.diag(1.0 / m) @ B.T
    n1 = g.n1
    W = sla.null_space(np.column_stack([s.e1[g.nu:], s.e0[g.nu:]]).T)
    Pb = np.zeros_like(S)
    Pb[:n1, :n1] = S[:n1, :n1]
    Pb[n1:, n1:] = S[n1:, n1:]
    lam = sla.eigh(W.T @ S @ W, W.T @ Pb @ W, eigvals_only=True)
    assert lam.max() / lam.min() <= 5.0
    K1 = fem.q1_stiffness(g).toarray()
    W1 = sla.null_space(np.ones((1, n1)))
    l1 = sla.eigh(W1.T @ S[:n1, :n1] @ W1, W1.T @ K1 @ W1, eigvals_only=True)
    assert 0.4 <= l1.min() and l1.max() <= 1.6
    L5 = np.zeros((g.n0, g.n0))
    for e in range(g.n0):
        ex, ey = e % n, e // n
        for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            if 0 <= ex + dx < n and 0 <= ey + dy < n:
                L5[e, e] += 1.0
                L5[e, (ey + dy) * n + ex + dx] -= 1.0
    W0 = sla.null_space(np.ones((1, g.n0)))
    l0 = sla.eigh(W0.T @ S[n1:, n1:] @ W0, W0.T @ L5 @ W0, eigvals_only=True)
    assert 3.0 <= l0.min() and l0.max() <= 5.0

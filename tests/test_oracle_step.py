"""Pins of the masked-grid inflow-outflow oracle (Sec. 3, Test problem 3).

* With every element active and no outflow, the masked assembly reproduces the
  square-grid system (itself pinned in test_oracle_fem.py) entry by entry.
* Poiseuille flow in a channel with a natural outflow is reproduced exactly:
  u = (1 - y^2, 0) lies in Q2 and p = 2 nu (L - x) in Q1, and the do-nothing
  condition holds for it (du_x/dx = 0 and p = 0 at x = L).
* On the step, P0 pressure makes every element conserve mass, so the flux through
  every vertical grid line equals the inflow flux int_0^1 4y(1-y) dy = 2/3.
* The null space is one-dimensional: [0; k] (no hydrostatic mode with an outflow).
* The paper's statements about this problem: the centroid pressures are an order of
  magnitude smaller than the vertex pressures, and the inf-sup constant of the
  step domain with its long channel is much smaller than that of the square.
"""
import numpy as np
import pytest

from oracle import fem, infsup, problem, step


def test_full_mask_reproduces_square_system():
    n = 6
    g = step.MaskedGrid(n, n, 2.0 / n, -1.0, -1.0, np.ones((n, n), dtype=bool), x_out=None)
    gs = fem.Grid(n)
    rng = np.random.default_rng(0)
    wind = rng.standard_normal(gs.nu)
    a = step.StepSystem(g, 0.03, wind)
    b = problem.System(gs, 0.03, wind)
    assert np.array_equal(g.fixed, gs.bnd)
    assert abs(a.K - b.K).max() <= 1e-14 * abs(b.K).max()
    assert abs(a.MQ - b.MQ).max() <= 1e-15


@pytest.mark.parametrize("m", [2, 4])
def test_poiseuille_exact(m):
    L, nu = 2.0, 0.02
    g = step.channel_grid(m, L)
    s = step.StepSystem(g, nu)
    ub = step.inflow_data(g, lambda y: 1.0 - y ** 2)
    x = s.solve(s.rhs(ub))
    u, p1, p0 = x[: g.nu], x[g.nu: g.nu + g.n1], x[g.nu + g.n1:]
    assert np.abs(u - np.concatenate([1.0 - g.Y2 ** 2, np.zeros(g.nv)])).max() <= 1e-12
    XI = g.x0 + g.hx * (np.arange(g.n1) % (g.nx + 1))
    for t, e in enumerate(g.elems):        # pressure function p1 + p0 at the element's vertices
        nodes = g.q1_conn[t]
        assert np.abs(p1[nodes] + p0[e] - 2.0 * nu * (L - XI[nodes])).max() <= 1e-12


@pytest.mark.parametrize("m", [2, 4])
def test_step_flux_and_elementwise_conservation(m):
    g = step.step_grid(m)
    ub = step.step_inflow(g)
    xs, res = step.picard(g, 1.0 / 50.0, ub, 5)
    s = step.StepSystem(g, 1.0 / 50.0)
    for x in (xs[0], xs[-1]):
        u = x[: g.nu]
        fl = np.array([step.vertical_flux(g, u, i) for i in range(0, g.Nx, 2)])
        assert np.abs(fl - 2.0 / 3.0).max() <= 1e-12, fl
        div0 = (s.B @ u)[g.n1:][g.p0_active]              # -int_T div u_h
        assert np.abs(div0).max() <= 1e-13
    assert all(r1 < 0.6 * r0 for r0, r1 in zip(res, res[1:])), res


def test_null_space_is_k_only():
    g = step.step_grid(1)
    s = step.StepSystem(g, 1.0 / 50.0, np.random.default_rng(1).standard_normal(g.nu))
    sv = np.linalg.svd(s.K.toarray(), compute_uv=False)
    assert sv[-1] <= 1e-12 * sv[0] and sv[-2] >= 1e-6 * sv[0]
    assert np.abs(s.K @ s.kx).max() <= 1e-13


def test_centroid_pressures_an_order_smaller():
    g = step.step_grid(4)
    xs, _ = step.picard(g, 1.0 / 50.0, step.step_inflow(g), 5)
    x = xs[-1]
    p1 = x[g.nu: g.nu + g.n1][g.q1_active]
    p0 = x[g.nu + g.n1:][g.p0_active]
    c = p0.mean()                      # frame split with zero-mean centroid part
    assert np.abs(p0 - c).max() <= 0.1 * np.abs(p1 + c).max()


def test_step_infsup_much_smaller_than_square():
    g1, _ = step.dense_gamma2(step.step_grid(1))
    g2, _ = step.dense_gamma2(step.step_grid(2))
    sq, _ = infsup.dense_gamma2(fem.Grid(8))
    assert abs(g1 - g2) <= 0.01 * g2
    assert g2 <= 0.2 * sq and g2 > 0.0


def test_inflow_robin_closed_form():
    """For a constant wind (c, 0) entering a channel at x = 0, the inflow boundary matrix
    is the 1D Q1 mass of the inflow edge times c: total c * (edge length) = 2c, symmetric,
    nothing on the edges the wind leaves through or runs along, and nothing for zero wind."""
    g = step.channel_grid(3, 2.0)
    c = 0.7
    wind = np.concatenate([np.full(g.nv, c), np.zeros(g.nv)])
    R = step.inflow_robin_q1(g, wind).toarray()
    assert abs(R.sum() - 2.0 * c) <= 1e-13 and np.allclose(R, R.T, atol=1e-15)
    I = np.arange(g.n1) % (g.nx + 1)
    assert np.abs(R[I != 0]).max() == 0.0 and np.abs(R[:, I != 0]).max() == 0.0
    h = g.hy
    col = R[np.ix_(I == 0, I == 0)]
    assert np.isclose(col[0, 0], c * h / 3.0) and np.isclose(col[1, 1], 2.0 * c * h / 3.0)
    assert np.isclose(col[0, 1], c * h / 6.0)
    # reversed, the wind enters through the right edge instead
    Rr = step.inflow_robin_q1(g, -wind).toarray()
    assert np.abs(Rr[I != g.nx]).max() == 0.0 and abs(Rr.sum() - 2.0 * c) <= 1e-13
    assert np.abs(step.inflow_robin_q1(g, 0.0 * wind).toarray()).max() == 0.0


def test_pcd_needs_the_inflow_term():
    """With natural conditions only (no inflow term: the Stokes system) the PCD Schur
    approximation annihilates the Q1 mass image of the constants; with the Oseen wind
    and its inflow term it does not (the reason for the reading)."""
    g = step.step_grid(2)
    one = g.q1_active.astype(float)
    s0 = step.StepSystem(g, 1.0 / 50.0)
    z0 = step.StepPCD1(s0).schur_inv(s0.Qk @ one)
    assert np.abs(z0).max() <= 1e-10
    xs, _ = step.picard(g, 1.0 / 50.0, step.step_inflow(g), 2)
    s1 = step.StepSystem(g, 1.0 / 50.0, xs[-1][: g.nu].copy())
    z1 = step.StepPCD1(s1).schur_inv(s1.Qk @ one)
    assert np.abs(z1).max() >= 1e-3


def test_step_two_stage_pcd():
    """The two-stage method (Sec. 3.1) on the Oseen step problem after five Picard steps:
    converges to the direct solution, Prop. 2 holds at the switch, and Step I needs a
    mesh-independent number of iterations (the paper's PCD histories are mesh independent)."""
    its1 = []
    for m in (2, 4):
        g = step.step_grid(m)
        ub = step.step_inflow(g)
        xs, _ = step.picard(g, 1.0 / 50.0, ub, 5)
        s = step.StepSystem(g, 1.0 / 50.0, xs[-1][: g.nu].copy())
        b = s.rhs(ub)
        x, info = step.two_stage(s, b, eta=1e-6, c=10.0)
        assert np.linalg.norm(b - s.K @ x) <= 1e-6 * np.linalg.norm(b) * 1.0001
        xd = s.solve(b)
        xc = x - (s.kx @ x) / (s.kx @ s.kx) * s.kx
        assert np.linalg.norm(xc - xd) <= 1e-4 * np.linalg.norm(xd)
        assert info["z_star_sq"] <= info["prop2_bound"] * (1.0 + 1e-10)
        its1.append(info["its1"])
    assert max(its1) <= 25 and abs(its1[1] - its1[0]) <= 5, its1


def test_step_lsc_mesh_robust():
    """GMRES with the LSC preconditioner M_3 on the Oseen step problem reaches the direct
    solution in a mesh-independent number of steps (the paper: LSC gives good results
    for Q2-Q1*)."""
    its = []
    for m in (2, 4, 8):
        g = step.step_grid(m)
        ub = step.step_inflow(g)
        xs, _ = step.picard(g, 1.0 / 50.0, ub, 5)
        s = step.StepSystem(g, 1.0 / 50.0, xs[-1][: g.nu].copy())
        b = s.rhs(ub)
        x, info = step.lsc_solve(s, b, tol=1e-6)
        assert np.linalg.norm(b - s.K @ x) <= 1e-6 * np.linalg.norm(b) * 1.0001
        xd = s.solve(b)
        xc = x - (s.kx @ x) / (s.kx @ s.kx) * s.kx
        assert np.linalg.norm(xc - xd) <= 1e-4 * np.linalg.norm(xd)
        its.append(info["its"])
    assert max(its) <= 20 and max(its) - min(its) <= 4, its


@pytest.mark.parametrize("m", [1, 2])
def test_step_est_minres_reaches_dense_gamma2(m):
    """EST-MINRES (Sec. 2.4) on the Stokes step problem with the exact blocks
    blkdiag(A, M_Q) (M_Q augmented with k, identity rows for inactive unknowns) reaches
    the dense inf-sup constant of the step from above: a second route to the value
    compared with the square's."""
    import scipy.sparse as sp
    from oracle import krylov
    g = step.step_grid(m)
    s = step.StepSystem(g, 1.0)
    b = s.rhs(step.step_inflow(g))
    Alu = krylov._LU(s.Anu)
    pin = sp.diags(np.concatenate([~g.q1_active, ~g.p0_active]).astype(float))
    aug = sp.bmat([[s.MQ + pin, sp.csr_matrix(s.k[:, None])], [sp.csr_matrix(s.k[None, :]), None]])
    Mlu = krylov._LU(aug.tocsc())
    P = lambda r: np.concatenate([Alu(r[: g.nu]), Mlu(np.concatenate([r[g.nu:], [0.0]]))[:-1]])
    x0 = np.concatenate([s.DB @ b[: g.nu], np.zeros(g.np_)])
    _, info = krylov.minres(lambda v: s.K @ v, P, b, x0, tol=1e-12, maxit=2000)
    h = infsup.est_history(info["delta"], info["gamma"])
    g2, _ = step.dense_gamma2(g)
    fin = h[np.isfinite(h)]
    assert np.all(fin >= g2 * (1 - 1e-8))
    assert abs(h[-1] - g2) <= 1e-6 * g2

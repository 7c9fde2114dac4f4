"""Pins of the oracle's discretisation against closed forms and exact integrals.

Everything here is independent of the oracle's own quadrature code: the
expected values are textbook closed forms of the 1D quadratic/linear Lagrange
element matrices, or exact symbolic integrals (sympy) of polynomial fields
that the Q2 / Q1 / P0 spaces represent exactly.
"""
import numpy as np
import pytest

from oracle import fem, problem
from paper_2303_10233_gb300 import workloads as W

sympy = pytest.importorskip("sympy")
xs, ys = sympy.symbols("x y")


# 1D closed forms on [0, h] for the quadratic Lagrange element at {0, h/2, h}
K2 = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / 3.0      # times 1/h
M2 = np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) / 30.0      # times h
M1 = np.array([[2, 1], [1, 2]]) / 6.0                           # linear mass, times h
# int_0^1 N_c(t) L_a'(t) dt and int_0^1 N_d(t) L_b(t) dt (N linear, L quadratic)
C12 = np.array([[-5, 4, 1], [-1, -4, 5]]) / 6.0
G12 = np.array([[1, 2, 0], [0, 2, 1]]) / 6.0


@pytest.mark.parametrize("dom", [(-1, 1, -1, 1), (0.0, 2.0, -1.0, 0.5)])
def test_element_matrices_closed_form(dom):
    g = fem.Grid(3, *dom)
    hx, hy = g.hx, g.hy
    E = fem.element_matrices(g)
    # local index i = b*3 + a  ->  kron(y-matrix, x-matrix)
    A = np.kron(M2 * hy, K2 / hx) + np.kron(K2 / hy, M2 * hx)
    np.testing.assert_allclose(E["A"], A, rtol=0, atol=1e-13)
    np.testing.assert_allclose(E["M2"], np.kron(M2 * hy, M2 * hx), atol=1e-15)
    np.testing.assert_allclose(E["Qk"], np.kron(M1 * hy, M1 * hx), atol=1e-15)
    np.testing.assert_allclose(E["B1x"], -np.kron(G12 * hy, C12), atol=1e-14)
    np.testing.assert_allclose(E["B1y"], -np.kron(C12, G12 * hx), atol=1e-14)
    np.testing.assert_allclose(E["R"], np.full((1, 4), hx * hy / 4), atol=1e-15)
    assert abs(E["Q0"][0, 0] - hx * hy) < 1e-15
    # int_T d(phi)/dx = hy * (L_a(1) - L_a(0)) * int L_b
    la = np.array([-1.0, 0.0, 1.0]); lb = np.array([1.0, 4.0, 1.0]) / 6.0
    np.testing.assert_allclose(E["B0x"][0], -np.kron(lb * hy, la), atol=1e-14)
    np.testing.assert_allclose(E["B0y"][0], -np.kron(la, lb * hx), atol=1e-14)


def _nodal(expr, X, Y):
    f = sympy.lambdify((xs, ys), expr, "numpy")
    return np.broadcast_to(np.asarray(f(X, Y), dtype=np.float64), X.shape).copy()


def _integrate(expr, dom):
    x0, x1, y0, y1 = [sympy.nsimplify(v) for v in dom]
    return float(sympy.integrate(expr, (xs, x0, x1), (ys, y0, y1)))


DOM = (0.0, 2.0, -1.0, 0.5)
U = xs**2 * ys + 3 * xs * ys**2 - ys          # in Q2 (degree <= 2 per variable)
V = xs * ys**2 - 2 * xs**2 + xs * ys


def test_q2_bilinear_forms_exact():
    g = fem.Grid(4, *DOM)
    u = _nodal(U, g.X2, g.Y2)
    v = _nodal(V, g.X2, g.Y2)
    A = fem.stiffness_q2(g)
    M = fem.mass_q2(g)
    ea = _integrate(sympy.diff(U, xs) * sympy.diff(V, xs) + sympy.diff(U, ys) * sympy.diff(V, ys), DOM)
    em = _integrate(U * V, DOM)
    assert abs(u @ (A @ v) - ea) < 1e-12 * max(1, abs(ea))
    assert abs(u @ (M @ v) - em) < 1e-12 * max(1, abs(em))
    assert abs(A @ np.ones(g.nv)).max() < 1e-12          # constants in null(A)


def test_divergence_exact_q1_and_p0():
    g = fem.Grid(3, *DOM)
    ux, uy = U, V
    u = np.concatenate([_nodal(ux, g.X2, g.Y2), _nodal(uy, g.X2, g.Y2)])
    Q = 1 + 2 * xs - xs * ys                       # bilinear -> exact in Q1
    q1 = _nodal(Q, g.X1, g.Y1)
    B1, B0 = fem.divergence(g)
    div = sympy.diff(ux, xs) + sympy.diff(uy, ys)
    assert abs(q1 @ (B1 @ u) + _integrate(Q * div, DOM)) < 1e-12
    # P0 part: (B0 u)_e = -int_{T_e} div u, element by element
    b0 = B0 @ u
    for e in range(g.n0):
        ex, ey = e % g.n, e // g.n
        d = (g.x0 + ex * g.hx, g.x0 + (ex + 1) * g.hx, g.y0 + ey * g.hy, g.y0 + (ey + 1) * g.hy)
        assert abs(b0[e] + _integrate(div, d)) < 1e-12


def _wind(expr_x, expr_y, g):
    return np.concatenate([_nodal(expr_x, g.X2, g.Y2), _nodal(expr_y, g.X2, g.Y2)])


def test_convection_exact_for_linear_wind():
    g = fem.Grid(4, *DOM)
    wx, wy = 1 + 2 * ys - xs, 0.5 - 3 * xs + ys       # linear wind: 3x3 Gauss is exact
    w = _wind(wx, wy, g)
    N = fem.convection_q2(g, w)
    u = _nodal(U, g.X2, g.Y2); v = _nodal(V, g.X2, g.Y2)
    exact = _integrate((wx * sympy.diff(V, xs) + wy * sympy.diff(V, ys)) * U, DOM)
    assert abs(u @ (N @ v) - exact) < 1e-11 * max(1, abs(exact))
    # the rule defines N for a Q2 wind; for a linear wind 3x3 and 4x4 agree
    N4 = fem.convection_q2(g, w, m=4)
    assert abs(N - N4).max() < 1e-13
    # Q1 convection with the same wind
    N1 = fem.q1_convection(g, w)
    P = 1 + xs - 2 * xs * ys; Qf = 2 - ys + xs * ys
    p = _nodal(P, g.X1, g.Y1); q = _nodal(Qf, g.X1, g.Y1)
    e1 = _integrate((wx * sympy.diff(Qf, xs) + wy * sympy.diff(Qf, ys)) * P, DOM)
    assert abs(p @ (N1 @ q) - e1) < 1e-11 * max(1, abs(e1))


def test_convection_rule_matters_for_quadratic_wind():
    g = fem.Grid(4, *DOM)
    w = _wind(xs**2 * ys**2, -xs * ys**2, g)
    N3 = fem.convection_q2(g, w, m=3)
    N5 = fem.convection_q2(g, w, m=5)
    assert abs(N3 - N5).max() > 1e-8                  # inexact for a Q2 wind


def test_convection_skew_on_interior_for_divergence_free_wind():
    g = fem.Grid(6)
    w = _wind(ys, -xs, g)                             # rotation: div w = 0, linear
    N = fem.convection_q2(g, w).toarray()
    I = ~g.bnd
    S = (N + N.T)[np.ix_(I, I)]
    assert abs(S).max() < 1e-13
    assert abs(N @ np.ones(g.nv)).max() < 1e-13        # N 1 = 0


def test_q1_matrices_exact():
    g = fem.Grid(3, *DOM)
    P = 1 + xs - 2 * xs * ys; Qf = 2 - ys + xs * ys
    p = _nodal(P, g.X1, g.Y1); q = _nodal(Qf, g.X1, g.Y1)
    _, Qk, _, _ = fem.pressure_mass(g)
    K1 = fem.q1_stiffness(g)
    assert abs(p @ (Qk @ q) - _integrate(P * Qf, DOM)) < 1e-12
    ek = _integrate(sympy.diff(P, xs) * sympy.diff(Qf, xs) + sympy.diff(P, ys) * sympy.diff(Qf, ys), DOM)
    assert abs(p @ (K1 @ q) - ek) < 1e-12


@pytest.mark.parametrize("n", [2, 4, 8])
def test_prop1_null_space_of_MQ(n):
    """Sec. 2.1 Prop. 1: null(M_Q) = span{k}; Remark 2: B^T k = 0."""
    g = fem.Grid(n)
    MQ, *_ = fem.pressure_mass(g)
    k = fem.null_vector_k(g)
    scale = abs(MQ).max()
    assert abs(MQ @ k).max() < 1e-14 * scale * 10
    sv = np.linalg.svd(MQ.toarray(), compute_uv=False)
    assert np.sum(sv < 1e-12 * sv[0]) == 1
    B1, B0 = fem.divergence(g)
    Bt_k = B1.T @ k[: g.n1] + B0.T @ k[g.n1:]
    assert abs(Bt_k).max() < 1e-14 * abs(B1).max() * 10


def test_cavity_null_space_dimension_two():
    """Enclosed flow: dim null(K) = 2 (constant Q1 and constant P0 pressures)."""
    w = W.cavity(4)
    g = fem.Grid(4)
    s = problem.System(g, w["nu"])
    sv = np.linalg.svd(s.K.toarray(), compute_uv=False)
    assert np.sum(sv < 1e-10 * sv[0]) == 2
    assert abs(s.K @ s.e1).max() < 1e-13 and abs(s.K @ s.e0).max() < 1e-13


def test_dof_counts_match_paper_table():
    """Velocity DoF counts of Table 1 (2178 at n=16, 526338 at n=256)."""
    assert fem.Grid(16).nu == 2178
    assert W.sizes(256)[1] == 526338
    assert W.sizes(16) == (1089, 2178, 289, 256, 2723)


@pytest.mark.parametrize("n,kind", [(6, "stokes"), (8, "oseen"), (10, "oseen")])
def test_k_rows_equal_assembled_rows(n, kind):
    """oracle.rows.k_rows (element by element, used for sampled full-size parity)
    equals the rows of the assembled K, boundary, interior, Q1 and P0 rows alike."""
    from oracle import rows as R
    from paper_2303_10233_gb300 import workloads as W
    w = W.oseen_cavity(n, nu=0.02, seed=4) if kind == "oseen" else W.mms(n, seed=1, nu=0.3)
    g = fem.Grid(n)
    s = problem.System(g, w["nu"], w["wind"])
    x = np.random.default_rng(n).standard_normal(g.nt)
    ref = s.K @ x
    rows = np.arange(g.nt)
    got = R.k_rows(g, w["nu"], w["wind"], x, rows)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()

"""Stokes solves on the GPU (MINRES + block-diagonal GMG / M_Q^+ preconditioner)
against the FP64 oracle: exact discrete solution (bordered direct solve),
true residual recomputed with the oracle's CSR K, element-wise conservation,
and mesh-independent iteration counts."""
import numpy as np
import pytest

from oracle import direct, fem, problem
from paper_2303_10233_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eth():
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_10233_gb300 import eth as E
    return E


def _solve(eth, w, **opts):
    G = eth.problem(w)
    u, p, st = G.solve(**opts)
    x = np.concatenate([u.cpu().numpy(), p.cpu().numpy()])
    G.close()
    return x, st


def _oracle(w):
    g = fem.Grid(w["n"])
    s = problem.System(g, w["nu"], w["wind"])
    b = s.rhs(w["f_nodal"], w["ubc"])
    return g, s, b


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cavity16_matches_direct(eth, precision):
    w = W.cavity(16)
    g, s, b = _oracle(w)
    x, st = _solve(eth, w, tol=1e-9, precision=precision)
    res = np.linalg.norm(b - s.K @ x) / np.linalg.norm(b)
    assert st["status"] == 0 and res <= 1e-9 * 1.01, (st, res)
    xd, _ = direct.solve(s, b)
    assert np.linalg.norm(s.canonical(x) - xd) <= 1e-7 * np.linalg.norm(xd)
    # canonical pressure returned: sum p1 = sum p0 = 0
    assert abs(x[g.nu: g.nu + g.n1].sum()) < 1e-9 and abs(x[g.nu + g.n1:].sum()) < 1e-9


@pytest.mark.parametrize("n", [8, 24, 64])
def test_mms_residual_and_error(eth, n):
    w = W.mms(n, seed=0)
    g, s, b = _oracle(w)
    x, st = _solve(eth, w, tol=1e-6, precision="mixed")
    res = np.linalg.norm(b - s.K @ x) / np.linalg.norm(b)
    assert res <= 1e-6 and abs(res - st["relres_true"]) <= 1e-3 * res + 1e-12
    x9, st9 = _solve(eth, w, tol=1e-10, precision="mixed")
    xd, _ = direct.solve(s, b)
    assert np.linalg.norm(s.canonical(x9) - xd) <= 1e-5 * np.linalg.norm(xd)
    # element-wise mass conservation of the solution: B0 u = g0
    r0 = (s.B0I @ x9[: g.nu]) - b[g.nu + g.n1:]
    assert np.abs(r0).max() <= 1e-8 * np.abs(b).max()


def test_iterations_mesh_independent(eth):
    its = []
    for n in (16, 32, 64, 128):
        _, st = _solve(eth, W.mms(n, seed=0), tol=1e-6, precision="fp64")
        its.append(st["iters_total"])
    assert max(its) - min(its) <= 10, its


def test_zero_rhs_and_bad_options(eth):
    w = W.cavity(8)
    w["ubc"] = np.zeros_like(w["ubc"])
    x, st = _solve(eth, w)
    assert np.abs(x).max() == 0.0
    G = eth.problem(W.cavity(8))
    with pytest.raises(eth.EthError):
        G.solve(tol=-1.0)
    G.close()


def test_cavity16_exact_blocks_match_oracle_minres(eth):
    """Config 1: MINRES with P_1 = blkdiag(A, M_Q) solved exactly (inner PCG to
    1e-12): the GPU iteration count equals the oracle's Algorithm 1 with the
    same exact blocks to within one iteration, and the solution matches."""
    from oracle import krylov
    w = W.cavity(16)
    g, s, b = _oracle(w)
    tol = 1e-8
    x, st = _solve(eth, w, tol=tol, precision="fp64", a_exact=1, mq_mode=1, inner_tol=1e-12)
    assert st["status"] == 0 and st["refine_passes"] == 1
    x0 = np.concatenate([s.DB @ b[: g.nu], np.zeros(g.np_)])
    bb = s.project_rhs(b)
    xo, info = krylov.minres(lambda v: s.K @ v, krylov.P1(s), bb, x0, tol=0.3 * tol / 1.0, maxit=500)
    assert abs(st["iters_total"] - info["its"]) <= 1, (st["iters_total"], info["its"])
    xd, _ = direct.solve(s, b)
    assert np.linalg.norm(s.canonical(x) - xd) <= 1e-6 * np.linalg.norm(xd)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_modes_match_stream_launches(eth, precision):
    """The device-side MINRES loop (conditional WHILE graph node, graph=1), host-replayed
    graphs of two iterations (graph=2) and plain stream launches (graph=0) perform the
    same arithmetic: same iteration count and the same solution, bitwise."""
    w = W.mms(40, seed=5)
    G = eth.problem(w)
    out = [G.solve(tol=1e-8, precision=precision, graph=m) for m in (0, 1, 2)]
    G.close()
    (u0, p0, s0) = out[0]
    for u, p, s in out[1:]:
        assert s["status"] == 0 and s["iters_total"] == s0["iters_total"]
        assert torch.equal(u, u0) and torch.equal(p, p0)


@pytest.mark.parametrize("kind", ["stokes", "oseen"])
def test_failure_statuses(eth, kind):
    """Failures made on the host, reported as status codes without a device fault:
    NaN in the body force -> ETH_ENAN; too few iterations -> ETH_ENOTCONV with the
    reached residual in the statistics; boundary data with a net flux (a right-hand
    side with a null-space component) -> ETH_EINCONSISTENT, returned with the solution of
    the projected system (the binding raises only for the hard failures)."""
    n = 16
    w = W.mms(n, seed=2) if kind == "stokes" else W.oseen_cavity(n, nu=1 / 50, seed=2)
    G = eth.problem(w)
    _, _, st = G.solve(tol=1e-10, maxit=3)
    assert st["status"] == 4 and st["relres_true"] > 1e-10
    f = torch.as_tensor(w["f_nodal"], device="cuda").clone()
    ub = torch.as_tensor(w["ubc"], device="cuda")
    f[7] = float("nan")
    G.set_rhs(f, ub)
    with pytest.raises(eth.EthError) as ei:
        G.solve(tol=1e-6, maxit=50)
    assert ei.value.status == 8
    g = fem.Grid(n)
    flux = np.zeros(2 * g.nv)
    left = np.isclose(g.X2, -1.0) & ~np.isclose(np.abs(g.Y2), 1.0)
    flux[: g.nv][left] = 1.0                      # inflow through the left side only
    G.set_rhs(torch.zeros(2 * g.nv, dtype=torch.float64, device="cuda"), torch.as_tensor(flux, device="cuda"))
    _, _, st = G.solve(tol=1e-6, maxit=400)
    assert st["status"] == 6   # the projected system is solved; the removal is reported
    G.close()

"""Oseen solves on the GPU (two-stage PCD GMRES, Sec. 3.1) against the FP64
oracle: exact discrete solution, true residual with the oracle's CSR K, the
Prop. 2 bound at the stage switch, and FP64 vs mixed precision."""
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


def _run(eth, w, **opts):
    G = eth.problem(w)
    u, p, st = G.solve(**opts)
    x = np.concatenate([u.cpu().numpy(), p.cpu().numpy()])
    G.close()
    return x, st


@pytest.mark.parametrize("n,nu", [(16, 1 / 100), (32, 1 / 100), (64, 1 / 50)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_oseen_matches_direct(eth, n, nu, precision):
    w = W.oseen_cavity(n, nu=nu, seed=1)
    g = fem.Grid(n)
    s = problem.System(g, w["nu"], w["wind"])
    b = s.rhs(w["f_nodal"], w["ubc"])
    x, st = _run(eth, w, tol=1e-9, precision=precision, mg_min_n=8)
    res = np.linalg.norm(b - s.K @ x) / np.linalg.norm(b)
    assert st["status"] == 0 and res <= 1e-9 * 1.01, (st, res)
    xd, _ = direct.solve(s, b)
    assert np.linalg.norm(s.canonical(x) - xd) <= 1e-6 * np.linalg.norm(xd)
    assert st["iters_stage1"] > 0 and st["iters_stage2"] >= 0
    # Prop. 2 at the switch: ||z*||^2 <= c^2 eta^2 ||f||^2 + ||r0*||^2
    assert st["prop2_lhs"] <= st["prop2_bound"] * (1 + 1e-6)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replayed_gmres_matches_stream_loop(eth, precision):
    """The graph-replayed Arnoldi step (column index read on the device, chunks of
    steps between host checks) performs the same arithmetic as the stream loop:
    same iteration counts and the same iterate, bitwise."""
    w = W.oseen_cavity(48, nu=1 / 200, seed=3)
    G = eth.problem(w)
    u0, p0, s0 = G.solve(tol=1e-8, precision=precision, graph=0)
    u1, p1, s1 = G.solve(tol=1e-8, precision=precision, graph=1)
    G.close()
    assert s0["status"] == 0 and s1["status"] == 0
    assert (s0["iters_stage1"], s0["iters_stage2"]) == (s1["iters_stage1"], s1["iters_stage2"])
    assert torch.equal(u0, u1) and torch.equal(p0, p1)


def test_adaptive_restart_and_option_checks(eth):
    """restart_max lets slow restart cycles double the restart length: a short
    GMRES(8) that cannot finish in 600 iterations converges when allowed to grow
    to 64 (cavity 32x32, nu = 1/200); out-of-range smoother damping is rejected before any device work."""
    w = W.oseen_cavity(32, nu=1 / 200, seed=2)
    G = eth.problem(w)
    _, _, sf = G.solve(tol=1e-8, restart=8, maxit=600)
    _, _, sa = G.solve(tol=1e-8, restart=8, restart_max=64, maxit=600)
    assert sa["status"] == 0 and sa["relres_true"] <= 1e-8 * 1.01
    if sf["status"] == 0:
        assert sa["iters_total"] <= sf["iters_total"]
    with pytest.raises(eth.EthError):
        G.solve(tol=1e-8, mg_omega=2.5)
    G.close()

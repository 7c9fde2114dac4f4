"""The warp-strip K apply (even/odd element arithmetic, one velocity component at
a time) against the oracle's assembled operators, element by element.

Grid sizes are chosen so that the strips of 30 owned element columns and the
warp's element rows end raggedly (n + 1 not a multiple of 30 or of the rows per
warp), including grids smaller than one strip; K, K^T and the reduced K1 are
checked for Stokes and Oseen in FP64 (1e-13 relative to the largest entry of
the oracle's product) and FP32 element arithmetic (5e-5).  A MINRES and a GMRES
solve with the strip form pinned (its fused <K z, z> reduction in MINRES)
reach the oracle's direct solution.
"""
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


def _case(kind, n):
    w = W.mms(n, seed=3, nu=0.7) if kind == "stokes" else W.oseen_cavity(n, nu=1 / 80, seed=3)
    g = fem.Grid(n)
    return w, g, problem.System(g, w["nu"], w["wind"])


@pytest.mark.parametrize("kind", ["stokes", "oseen"])
@pytest.mark.parametrize("n", [2, 6, 28, 30, 62, 96])
def test_strip_apply_matches_oracle(eth, kind, n):
    w, g, s = _case(kind, n)
    G = eth.problem(w)
    rng = np.random.default_rng(40 + n)
    x = rng.standard_normal(g.nt)
    xt = torch.as_tensor(x, device=G.device)
    n1 = g.nu + g.n1
    ops = {"K": (s.K, x), "KT": (s.K.T.tocsr(), x), "K1": (s.K1, x[:n1])}
    for rows in (4, 8, 16, 32):
        G.set_tile(rows, 2)
        for op, (A, xin) in ops.items():
            ref = A @ xin
            scale = np.abs(ref).max()
            xi = xt if op != "K1" else xt[:n1].contiguous()
            y64 = G.apply(op, xi).cpu().numpy()
            assert np.abs(y64 - ref).max() <= 1e-13 * scale, (rows, op, "fp64")
            y32 = G.apply(op, xi, fp32=True).cpu().numpy()
            assert np.abs(y32 - ref).max() <= 5e-5 * scale, (rows, op, "fp32")
    G.close()


@pytest.mark.parametrize("kind,n", [("stokes", 46), ("oseen", 32)])
def test_strip_solves_match_direct(eth, kind, n):
    w, g, s = _case(kind, n)
    b = s.rhs(w["f_nodal"], w["ubc"])
    xd, _ = direct.solve(s, b)
    G = eth.problem(w)
    G.set_tile(8, 2)
    for precision in ("fp64", "mixed"):
        u, p, st = G.solve(tol=1e-10, precision=precision, autotune=0, mg_min_n=4 if kind == "stokes" else 8)
        assert st["status"] == 0 and st["tile_persistent"] == 2, st
        x = s.canonical(np.concatenate([u.cpu().numpy(), p.cpu().numpy()]))
        assert np.linalg.norm(b - s.K @ x) <= 1e-10 * np.linalg.norm(b) * 1.01
        assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd), precision
    G.close()

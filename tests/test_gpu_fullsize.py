"""Parity at the full workload sizes, in the launch configurations the bench and the
solvers use: sampled entries of K x (the oracle computes each from the element
matrices, oracle.rows) for the Stokes 256^2 bench grid, the 1024^2 roofline grid and
the 512^2 Oseen grid, with every tile shape the autotuner may choose; and the
bench solve's true FP64 residual and pressure normalisation with the oracle's
assembled 256^2 system.  Per-entry bound: |y - y_ref| <= tol * (|K| |x|)_i with
tol = 1e-13 (FP64 element arithmetic) and 5e-5 (FP32)."""
import numpy as np
import pytest

from oracle import fem, problem, rows as R
from paper_2303_10233_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eth():
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_10233_gb300 import eth as E
    return E


def _sample(g, rng, m):
    """m random rows plus the corners, an edge midpoint and first/last pressure rows."""
    N, nv = g.N, g.nv
    special = [0, N - 1, nv - N, nv - 1, N // 2, nv + N * (N // 2) + 1,
               2 * nv, 2 * nv + g.n1 - 1, 2 * nv + g.n1, g.nt - 1]
    return np.unique(np.concatenate([rng.integers(0, g.nt, m), special]))


@pytest.mark.parametrize("n,kind", [(256, "stokes"), (1024, "stokes"), (512, "oseen")])
def test_fullsize_k_apply_sampled(eth, n, kind):
    w = W.mms(n, seed=0) if kind == "stokes" else W.oseen_cavity(n, nu=0.01, seed=1)
    g = fem.Grid(n)
    G = eth.problem(w)
    rng = np.random.default_rng(n + 7)
    x = rng.standard_normal(g.nt)
    rows = _sample(g, rng, 3000)
    ref = R.k_rows(g, w["nu"], w["wind"], x, rows)
    bnd = R.k_rows(g, w["nu"], w["wind"], x, rows, bound=True)
    xt = torch.as_tensor(x, device="cuda")
    for rows_, pers in ((0, False), (4, False), (8, False), (16, False), (8, True)):
        G.set_tile(rows_, pers)
        for fp32, tol in ((False, 1e-13), (True, 5e-5)):
            if fp32 is False and pers:
                continue   # the persistent form is FP32 only
            y = G.apply("K", xt, fp32=fp32).cpu().numpy()[rows]
            err = np.abs(y - ref)
            assert np.all(err <= tol * bnd + 1e-300), (rows_, pers, fp32, (err / bnd).max())
    G.close()


def test_fullsize_bench_solve_residual(eth):
    """The bench workload (Stokes 256^2 MMS, mixed precision, defaults): the true FP64
    residual of the returned solution, evaluated with the oracle's assembled K."""
    n = 256
    w = W.mms(n, seed=0)
    g = fem.Grid(n)
    s = problem.System(g, w["nu"], w["wind"])
    b = s.rhs(w["f_nodal"], w["ubc"])
    G = eth.problem(w)
    u, p, st = G.solve(tol=1e-6)
    G.close()
    x = np.concatenate([u.cpu().numpy(), p.cpu().numpy()])
    res = np.linalg.norm(b - s.K @ x) / np.linalg.norm(b)
    assert st["status"] == 0 and res <= 1e-6 * 1.001, (res, st)
    assert abs(st["relres_true"] - res) <= 1e-9
    _, p1, p0 = s.split(x)
    assert abs(p1.sum()) <= 1e-9 * np.abs(p1).sum() and abs(p0.sum()) <= 1e-9 * np.abs(p0).sum()
    # discretisation error against the manufactured velocity stays at the solver tolerance level
    ue = w["u_exact"]
    assert np.linalg.norm(x[: g.nu] - ue) <= 1e-5 * np.linalg.norm(ue)

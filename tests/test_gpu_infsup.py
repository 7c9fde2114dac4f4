"""EST-MINRES inf-sup estimate on the GPU (Sec. 2.4) against the oracle.

* The estimate kernel (Sturm bisection on a bordered tridiagonal) against the
  oracle's harmonic Ritz values (dense pencil) on seeded random tridiagonals.
* The Lanczos coefficients a GPU Stokes solve records with the exact blocks of
  P_1 against those of the oracle's Algorithm 1 on the same system, and the
  estimates against the oracle's dense gamma^2 (reached from above).
"""
import numpy as np
import pytest

from oracle import fem, infsup, krylov, problem
from paper_2303_10233_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eth():
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_10233_gb300 import eth as E
    return E


@pytest.mark.parametrize("k,seed", [(1, 0), (2, 1), (7, 2), (33, 3), (100, 4), (257, 5)])
def test_est_kernel_matches_oracle(eth, k, seed):
    d, gm = W.tridiagonal(k, seed)
    G = eth.Grid(4, "stokes")
    dd = torch.as_tensor(d, device="cuda")
    gg = torch.as_tensor(gm, device="cuda")
    got = G.est_infsup(dd, gg).cpu().numpy()
    G.close()
    ref = infsup.est_history(d, np.concatenate([[1.0], gm]))
    assert np.array_equal(np.isnan(got), np.isnan(ref)), (got, ref)
    f = ~np.isnan(ref)
    if f.any():
        assert np.allclose(got[f], ref[f], rtol=1e-8, atol=0.0), np.abs(got[f] / ref[f] - 1).max()


@pytest.mark.parametrize("n", [8, 16])
def test_est_minres_exact_p1(eth, n):
    w = W.cavity(n)
    g = fem.Grid(n)
    s = problem.System(g, w["nu"])
    b = s.rhs(w["f_nodal"], w["ubc"])
    G = eth.problem(w)
    u, p, st = G.solve(tol=1e-10, precision="fp64", a_exact=1, mq_mode=1, inner_tol=1e-13)
    assert st["status"] == 0
    d, gm = G.lanczos()
    est = G.est_infsup().cpu().numpy()
    d, gm = d.cpu().numpy(), gm.cpu().numpy()
    G.close()
    k = d.size
    assert 20 <= k <= st["iters_total"]
    # Algorithm 1 in the oracle from the same start (boundary values set, k projected)
    x0 = np.concatenate([s.DB @ b[: g.nu], np.zeros(g.np_)])
    xo, info = krylov.minres(lambda v: s.K @ v, krylov.P1(s), s.project_rhs(b), x0, tol=1e-12, maxit=k)
    do, go = np.array(info["delta"]), np.array(info["gamma"][1:])
    m = min(12, k, do.size)
    assert np.allclose(d[:m], do[:m], rtol=1e-7, atol=1e-9), (d[:m], do[:m])
    assert np.allclose(gm[:m], go[:m], rtol=1e-7, atol=1e-9), (gm[:m], go[:m])
    g2, _ = infsup.dense_gamma2(g)
    fin = est[np.isfinite(est)]
    assert np.all(fin >= g2 * (1 - 1e-6)), (fin.min(), g2)
    assert abs(est[-1] - g2) <= 1e-5 * g2, (est[-1], g2)
    eo = infsup.est_history(info["delta"], info["gamma"])
    m = min(20, k, eo.size)
    assert np.allclose(est[:m], eo[:m], rtol=1e-6, equal_nan=True), (est[:m], eo[:m])


def test_lanczos_record_mixed_first_pass(eth):
    """With mixed precision and refinement only the first MINRES run is recorded; its
    estimate (of the V-cycle / M_Q-approximation preconditioner) is finite and positive."""
    w = W.mms(32, seed=0)
    G = eth.problem(w)
    u, p, st = G.solve(tol=1e-10, precision="mixed")
    d, gm = G.lanczos()
    est = G.est_infsup(d, gm).cpu().numpy()
    G.close()
    assert st["refine_passes"] >= 2
    assert 0 < d.numel() < st["iters_total"]
    assert np.isfinite(est[-1]) and est[-1] > 0.0

"""Batched concurrent solves: each instance's result equals its one-at-a-time
solve (same kernels, same order of operations) and meets the tolerance with
the oracle's CSR operator."""
import numpy as np
import pytest

from oracle import fem, problem
from paper_2303_10233_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eth():
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_10233_gb300 import eth as E
    return E


def _instances():
    out = []
    rng = np.random.default_rng(5)
    for i, n in enumerate([8, 16, 32, 16, 8, 32]):
        nv = (2 * n + 1) ** 2
        inst = {"n": n, "nu": float(10 ** rng.uniform(-1.5, -0.5)), "f_nodal": rng.standard_normal(2 * nv),
                "ubc": np.zeros(2 * nv), "wind": W.oseen_wind(n, 1000 + i) if i % 2 else None}
        out.append(inst)
    return out


def test_batch_matches_single_and_oracle(eth):
    insts = _instances()
    opts = dict(tol=1e-8, precision="mixed", mg_min_n=4, maxit=3000)
    single = []
    for w in insts:
        G = eth.problem(w)
        u, p, st = G.solve(**opts)
        single.append((np.concatenate([u.cpu().numpy(), p.cpu().numpy()]), st))
        G.close()
    grids = [eth.problem(w) for w in insts]
    B = eth.Batch(grids)
    us, ps, sts, rc = B.solve(**opts)
    assert rc == 0, sts
    for w, u, p, st, (xs, st1) in zip(insts, us, ps, sts, single):
        x = np.concatenate([u.cpu().numpy(), p.cpu().numpy()])
        assert st["status"] == 0
        assert np.abs(x - xs).max() <= 1e-12 * max(1.0, np.abs(xs).max())
        g = fem.Grid(w["n"])
        s = problem.System(g, w["nu"], w["wind"])
        b = s.rhs(w["f_nodal"], w["ubc"])
        assert np.linalg.norm(b - s.K @ x) <= 1e-8 * np.linalg.norm(b) * 1.01
    B.close()
    for G in grids:
        G.close()

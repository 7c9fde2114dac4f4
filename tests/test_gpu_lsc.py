"""The LSC preconditioner M_3 on the GPU (Sec. 3.2, Eq. lsc-definition and Eq.
nse-precon-lsc) against the FP64 oracle.

* GMRES with M_3 reaches the oracle's exact discrete solution (sparse direct) on
  the Oseen cavity, in FP64 and in mixed precision.
* Its iteration counts stay close to those of the oracle's LSC with exact solves
  (oracle.lsc: exact F and exact frame-operator solves): the GPU's frame solves
  are a few V-cycle-preconditioned CG steps, its F solve one V-cycle.
* The adjoint solve with M_3 (F^T in the middle factor) matches the PCD adjoint.
* The hardest instance of the seeded uneven batch (n = 32, nu = 1.3e-3, cell
  Peclet number about 24), which the two-stage PCD method leaves above 1e-6,
  converges.
"""
import numpy as np
import pytest

from oracle import direct, fem, lsc, problem
from paper_2303_10233_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eth():
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_10233_gb300 import eth as E
    return E


def _sys(w):
    g = fem.Grid(w["n"])
    s = problem.System(g, w["nu"], w["wind"])
    return g, s, s.rhs(w["f_nodal"], w["ubc"])


@pytest.mark.parametrize("n,nu", [(16, 1 / 100), (32, 1 / 500)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_lsc_solve_matches_direct(eth, n, nu, precision):
    w = W.oseen_cavity(n, nu=nu, seed=1)
    g, s, b = _sys(w)
    xd, _ = direct.solve(s, b)
    G = eth.problem(w)
    u, p, st = G.solve(tol=1e-9, precision=precision, oseen_prec="lsc", restart=100, maxit=2000)
    G.close()
    x = s.canonical(np.concatenate([u.cpu().numpy(), p.cpu().numpy()]))
    res = np.linalg.norm(b - s.K @ x) / np.linalg.norm(b)
    assert st["status"] == 0 and res <= 1e-9 * 1.01, (st, res)
    assert st["iters_stage1"] == 0 and st["iters_stage2"] == st["iters_total"] > 0
    assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)


def test_lsc_iterations_close_to_exact_lsc(eth):
    out = []
    for n in (16, 32, 64):
        w = W.oseen_cavity(n, nu=1 / 100, seed=1)
        g, s, b = _sys(w)
        _, info = lsc.solve(s, b, tol=1e-6, restart=200, maxit=400)
        G = eth.problem(w)
        _, _, st = G.solve(tol=1e-6, oseen_prec="lsc", restart=200, maxit=400)
        G.close()
        assert st["status"] == 0, st
        out.append((n, info["its"], st["iters_total"]))
    print("LSC iterations (n, oracle exact blocks, GPU):", out)
    for n, ref, its in out:
        assert its <= 1.5 * ref + 5, out
    assert out[-1][2] <= 1.6 * out[0][2] + 5, out   # mesh-robust


def test_lsc_adjoint_matches_pcd_adjoint(eth):
    w = W.diff(16, nu=1 / 200)
    G = eth.problem(w)
    rng = np.random.default_rng(3)
    ru = torch.as_tensor(rng.standard_normal(2 * G.nv), device=G.device)
    rp = torch.zeros(G.n1 + G.n0, dtype=torch.float64, device=G.device)
    tight = dict(tol=1e-11, precision="fp64", maxit=3000, restart=100)
    l1, p1, s1 = G.solve_adjoint(ru, rp, **tight)
    l2, p2, s2 = G.solve_adjoint(ru, rp, oseen_prec="lsc", **tight)
    G.close()
    assert s1["status"] == 0 and s2["status"] == 0, (s1, s2)
    assert float(torch.linalg.norm(l1 - l2)) <= 1e-8 * float(torch.linalg.norm(l1))


def test_lsc_converges_on_the_hardest_batch_instance(eth):
    insts = W.batch(seed=2)
    w = insts[57]
    assert w["n"] == 32 and w["wind"] is not None
    g, s, b = _sys(w)
    G = eth.problem(w)
    u, p, st = G.solve(tol=1e-6, oseen_prec="lsc", restart=150, maxit=3000)
    G.close()
    x = np.concatenate([u.cpu().numpy(), p.cpu().numpy()])
    res = np.linalg.norm(b - s.K @ x) / np.linalg.norm(b)
    print(f"batch instance 57 (nu = {w['nu']:.3g}): LSC its {st['iters_total']}, relres {res:.2e}")
    assert st["status"] == 0 and res <= 1e-6 * 1.01, (st, res)

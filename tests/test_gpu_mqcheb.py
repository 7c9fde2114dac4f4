"""The multicolour Chebyshev-SGS approximation of M_Q on the GPU (the M_cheb block
of P_2, Sec. 2.3-2.4) against oracle/mqcheb.py.

* With the oracle's interval [a, 1] the GPU's 20-step output equals the oracle's
  sweep-by-sweep computation element by element (FP64 1e-10, FP32 1e-4): the five
  colours are independent sets of M_Q, so the multicolour sweep is the oracle's SGS.
* Many steps reproduce M_Q^+ (k projected out, the augmented-system solve).
* The default lower end 0.655 / n^2 stays within a few per cent of the oracle's
  exact smallest nonzero eigenvalue of P^{-1} M_Q.
* MINRES with blkdiag(GMG V-cycle, M_cheb) reaches the direct solution, and its
  iteration count grows under refinement (the paper's observation for P_2), while
  the default V-cycle approximation of M_Q keeps it flat.
"""
import numpy as np
import pytest

from oracle import direct, fem, krylov, mqcheb, problem
from paper_2303_10233_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eth():
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_10233_gb300 import eth as E
    return E


@pytest.mark.parametrize("n", [8, 16])
def test_mqcheb_matches_oracle(eth, n):
    g = fem.Grid(n)
    s = problem.System(g, 1.0)
    a, b = mqcheb.sgs_interval(g, s.MQ, s.k)
    ref_op = mqcheb.MCheb(s, steps=20, interval=(a, b))
    G = eth.problem(W.cavity(n))
    rng = np.random.default_rng(n)
    for _ in range(2):
        r = rng.standard_normal(g.np_)
        ref = ref_op(r)
        rt = torch.as_tensor(r, device=G.device)
        z = G.apply_mqcheb(rt, steps=20, a=a, b=b).cpu().numpy()
        assert np.abs(z - ref).max() <= 1e-10 * np.abs(ref).max()
        assert abs(z @ s.k) <= 1e-10 * np.abs(z).sum()
        z32 = G.apply_mqcheb(rt, steps=20, a=a, b=b, fp32=True).cpu().numpy()
        assert np.abs(z32 - ref).max() <= 1e-4 * np.abs(ref).max()
    # many steps: M_Q^+ (k projected out)
    r = rng.standard_normal(g.np_)
    exact = krylov.MQSolve(s)(r - (s.k @ r) / (s.k @ s.k) * s.k)
    z = G.apply_mqcheb(torch.as_tensor(r, device=G.device), steps=400, a=a, b=b).cpu().numpy()
    assert np.linalg.norm(z - exact) <= 1e-7 * np.linalg.norm(exact)
    G.close()


def test_default_interval_end_close_to_exact():
    for n in (8, 16):
        g = fem.Grid(n)
        a, _ = mqcheb.sgs_interval(g)
        assert abs(0.655 / n ** 2 - a) <= 0.03 * a, (n, a)


def test_minres_with_mcheb_block(eth):
    its = []
    for n in (16, 32, 64):
        w = W.cavity(n)
        G = eth.problem(w)
        _, _, sv = G.solve(tol=1e-8, precision="fp64")
        u, p, st = G.solve(tol=1e-8, precision="fp64", mq_mode="cheb")
        G.close()
        assert st["status"] == 0, st
        its.append((n, sv["iters_total"], st["iters_total"]))
        if n == 16:
            g = fem.Grid(n)
            s = problem.System(g, w["nu"])
            b = s.rhs(w["f_nodal"], w["ubc"])
            xd, _ = direct.solve(s, b)
            x = s.canonical(np.concatenate([u.cpu().numpy(), p.cpu().numpy()]))
            assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)
    print("MINRES iterations (n, V-cycle M_Q, M_cheb):", its)
    assert its[-1][2] > its[0][2]                        # P_2 degrades under refinement
    assert its[-1][1] <= its[0][1] + 6                   # the default block does not

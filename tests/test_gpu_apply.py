"""Parity of every eth_apply operator with the oracle's assembled CSR matrices.

Grids span one tile (n <= 30), several tiles and ragged tails (the CUDA tile
owns 31 x 7 elements).  Bound per entry: |y - y_ref| <= tol * (|K| |x|)_i,
tol = 1e-13 for FP64 element arithmetic and 5e-5 for FP32 (sum
factorisation takes a few hundred FP32 rounding steps per output).
"""
import numpy as np
import pytest
import scipy.sparse as sp

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


def _oracle_ops(s):
    g = s.g
    Mv = sp.block_diag([s.Mv, s.Mv]).tocsr()
    return {"K": s.K, "KT": s.K.T.tocsr(), "A": s.Anu, "F": s.F, "B": s.BI, "BT": s.BI.T.tocsr(),
            "MQ": s.MQ, "MV": Mv, "K1": s.K1}


def _check(y, M, x, tol):
    ref = M @ x
    bound = abs(M) @ abs(x) + 1e-300
    err = np.abs(y - ref)
    assert np.all(err <= tol * bound + 1e-14 * np.abs(ref).max()), (err / bound).max()


@pytest.mark.parametrize("n", [2, 4, 16, 62, 70, 126])
@pytest.mark.parametrize("kind", ["stokes", "oseen"])
def test_apply_parity(eth, n, kind):
    w = W.oseen_cavity(n, nu=0.01, seed=1) if kind == "oseen" else W.mms(n, seed=0, nu=0.7)
    g = fem.Grid(n)
    s = problem.System(g, w["nu"], w["wind"])
    G = eth.problem(w)
    rng = np.random.default_rng(n)
    for op, M in _oracle_ops(s).items():
        x = rng.standard_normal(M.shape[1])
        xt = torch.as_tensor(x, device="cuda")
        for fp32, tol in ((False, 1e-13), (True, 5e-5)):
            y = G.apply(op, xt, fp32=fp32).cpu().numpy()
            _check(y, M, x, tol)
    b = G.rhs().cpu().numpy()
    bref = s.rhs(w["f_nodal"], w["ubc"])
    assert np.abs(b - bref).max() <= 1e-13 * np.abs(bref).max()
    G.close()


def test_apply_domain_anisotropic(eth):
    n = 40
    dom = (0.0, 2.0, -1.0, 0.5)
    g = fem.Grid(n, *dom)
    rng = np.random.default_rng(3)
    wind = rng.standard_normal(g.nu)
    s = problem.System(g, 0.3, wind)
    G = eth.Grid(n, "oseen", domain=dom)
    G.set_coefficients(0.3, torch.as_tensor(wind, device="cuda"))
    for op in ("K", "KT", "MQ", "MV"):
        M = _oracle_ops(s)[op]
        x = rng.standard_normal(M.shape[1])
        y = G.apply(op, torch.as_tensor(x, device="cuda")).cpu().numpy()
        _check(y, M, x, 1e-13)
    G.close()

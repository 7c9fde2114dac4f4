"""Picard iteration for steady Navier-Stokes on the GPU (eth_picard: a sequence of
two-stage Oseen solves whose wind is the previous velocity) against the oracle's
Picard iteration with direct solves: the iterates and the nonlinear residual of
every step."""
import numpy as np
import pytest

from oracle import fem, picard
from paper_2303_10233_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eth():
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_10233_gb300 import eth as E
    return E


@pytest.mark.parametrize("n,nu,precision", [(16, 1 / 50, "fp64"), (32, 1 / 20, "mixed")])
def test_picard_matches_oracle(eth, n, nu, precision):
    steps = 5
    w = W.cavity(n, nu=nu)
    g = fem.Grid(n)
    xs, res = picard.picard(g, nu, w["f_nodal"], w["ubc"], steps)
    G = eth.Grid(n, "oseen")
    G.set_coefficients(nu, torch.zeros(2 * g.nv, dtype=torch.float64, device="cuda"))
    f = torch.as_tensor(w["f_nodal"], device="cuda")
    ub = torch.as_tensor(w["ubc"], device="cuda")
    u, p, nlres, stats = G.picard(f, ub, steps, tol=1e-11, precision=precision, restart_max=160, maxit=4000)
    G.close()
    assert all(s["status"] == 0 for s in stats), stats
    x = np.concatenate([u.cpu().numpy(), p.cpu().numpy()])
    assert np.linalg.norm(x - xs[-1]) <= 1e-7 * np.linalg.norm(xs[-1])
    for a, b in zip(nlres, res):
        assert abs(a - b) <= 1e-4 * b + 1e-9, (nlres, res)
    assert nlres[-1] < nlres[0]

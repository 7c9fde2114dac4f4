"""The GPU's Q1 PCD Schur block (Sec. 3.1, Eq. discrete-commutator1x) against the
oracle's, element by element.

eth_apply_pcd applies M_S^{-1} r = Ap^+ F1 Q1^{-1} r with chosen inner step
counts; with many Chebyshev steps for Q1^{-1} and many V-cycle-preconditioned CG
steps for Ap^+ it is the exact block, which must equal oracle.krylov.PCD1's
sparse-direct schur_inv (FP64: 1e-9; FP32 inner arithmetic: 1e-4).  The adjoint
form (F1^T, used by the adjoint Oseen solve) is compared with
Ap^+ F1^T Q1^{-1} from the same oracle pieces.  The solver's own setting (10
Chebyshev steps, 2 CG steps) is checked to stay a fair approximation of it.
"""
import numpy as np
import pytest

from oracle import fem, krylov, problem
from paper_2303_10233_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eth():
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_10233_gb300 import eth as E
    return E


def _mean_free(v):
    return v - v.mean()


@pytest.mark.parametrize("n,nu", [(16, 1 / 50), (64, 1 / 100)])
def test_pcd_block_matches_oracle(eth, n, nu):
    w = W.oseen_cavity(n, nu=nu, seed=1)
    g = fem.Grid(n)
    s = problem.System(g, w["nu"], w["wind"])
    pcd = krylov.PCD1(s)
    G = eth.problem(w)
    rng = np.random.default_rng(7 + n)
    for k in range(2):
        r = rng.standard_normal(g.n1)
        ref = _mean_free(pcd.schur_inv(r))
        rt = torch.as_tensor(r, device=G.device)
        z64 = G.apply_pcd(rt, cheb_steps=80, ap_its=60).cpu().numpy()
        assert abs(z64.mean()) <= 1e-10 * np.abs(z64).max()
        err = np.abs(z64 - ref).max() / np.abs(ref).max()
        assert err <= 1e-9, (n, k, err)
        z32 = G.apply_pcd(rt, cheb_steps=40, ap_its=40, fp32=True).cpu().numpy()
        e32 = np.abs(z32 - ref).max() / np.abs(ref).max()
        assert e32 <= 1e-4, (n, k, e32)
        # the adjoint block: Ap^+ F1^T Q1^{-1}
        refa = _mean_free(pcd.Apsolve(pcd.F1.T @ pcd.Q1solve(r)))
        za = G.apply_pcd(rt, cheb_steps=80, ap_its=60, adjoint=True).cpu().numpy()
        ea = np.abs(za - refa).max() / np.abs(refa).max()
        assert ea <= 1e-9, (n, k, ea)
    # the solver's inexact setting (10 Chebyshev steps, 2 CG steps) stays close to the block
    r = rng.standard_normal(g.n1)
    ref = _mean_free(pcd.schur_inv(r))
    zs = G.apply_pcd(torch.as_tensor(r, device=G.device), cheb_steps=10, ap_its=2).cpu().numpy()
    assert np.linalg.norm(zs - ref) <= 0.5 * np.linalg.norm(ref)
    with pytest.raises(eth.EthError):
        G.apply_pcd(torch.as_tensor(r, device=G.device), cheb_steps=10, ap_its=0)
    G.close()


def test_pcd_rejects_stokes_grid(eth):
    G = eth.problem(W.cavity(8))
    with pytest.raises(eth.EthError):
        G.apply_pcd(torch.zeros(G.n1, dtype=torch.float64, device=G.device))
    G.close()

"""Adjoint solves and gradients on the GPU against the oracle's exact (direct)
adjoint, the symmetric-Stokes identity, and central finite differences of
the GPU forward solve through torch.autograd."""
import numpy as np
import pytest

from oracle import adjoint, direct, fem, problem
from paper_2303_10233_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_10233_gb300 import autograd, eth
    return eth, autograd


TIGHT = dict(tol=1e-11, precision="fp64", mg_min_n=4, maxit=4000)


@pytest.mark.parametrize("n", [8, 16])
def test_oseen_gradients_match_dense_adjoint(E, n):
    eth, _ = E
    w = W.diff(n, nu=1 / 200)
    g = fem.Grid(n)
    s = problem.System(g, w["nu"], w["wind"])
    J, gf_ref, gnu_ref, lam_ref = adjoint.gradients(s, w["f_nodal"], w["ubc"], w["u_target"])
    G = eth.problem(w)
    u, p, st = G.solve(**TIGHT)
    assert st["status"] == 0
    ut = torch.as_tensor(w["u_target"], device="cuda")
    ru = 2.0 * (u - ut)
    rp = torch.zeros(G.n1 + G.n0, dtype=torch.float64, device="cuda")
    lu, lp, sa = G.solve_adjoint(ru, rp, **TIGHT)
    assert sa["status"] == 0, sa
    gf, gnu = G.adjoint_gradients(lu, u)
    gf = gf.cpu().numpy()
    assert np.linalg.norm(gf - gf_ref) <= 1e-7 * np.linalg.norm(gf_ref)
    assert abs(gnu - gnu_ref) <= 1e-7 * abs(gnu_ref)
    # the adjoint velocity itself (interior nodes; boundary rows are identity rows)
    I = np.concatenate([~g.bnd, ~g.bnd])
    lr = lam_ref[: g.nu]
    assert np.linalg.norm(lu.cpu().numpy()[I] - lr[I]) <= 1e-7 * np.linalg.norm(lr[I])
    G.close()


def test_stokes_adjoint_is_forward_operator(E):
    eth, _ = E
    w = W.mms(16, seed=0)
    G = eth.problem(w)
    b = G.rhs()
    nu2 = 2 * G.nv
    lu, lp, sa = G.solve_adjoint(b[:nu2].contiguous(), b[nu2:].contiguous(), **TIGHT)
    u, p, st = G.solve(**TIGHT)
    assert torch.linalg.norm(lu - u) <= 1e-8 * torch.linalg.norm(u)
    G.close()


def test_autograd_matches_finite_differences(E):
    eth, ag = E
    n = 8
    w = W.diff(n, nu=1 / 200)
    G = eth.Grid(n, "oseen")
    wind = torch.as_tensor(w["wind"], device="cuda")
    ubc = torch.as_tensor(w["ubc"], device="cuda")
    ut = torch.as_tensor(w["u_target"], device="cuda")
    f = torch.as_tensor(w["f_nodal"], device="cuda").clone().requires_grad_(True)
    nu = torch.tensor(w["nu"], dtype=torch.float64, device="cuda", requires_grad=True)
    u, p = ag.solve(f, nu, G, ubc, wind, **TIGHT)
    J = ((u - ut) ** 2).sum()
    J.backward()

    def Jof(fv, nuv):
        uu, _ = ag.solve(fv, nuv, G, ubc, wind, **TIGHT)
        return float(((uu - ut) ** 2).sum())

    rng = np.random.default_rng(11)
    eps = 1e-4
    with torch.no_grad():
        for _ in range(3):
            d = torch.as_tensor(rng.standard_normal(f.numel()), device="cuda")
            d /= torch.linalg.norm(d)
            fd = (Jof(f + eps * d, nu) - Jof(f - eps * d, nu)) / (2 * eps)
            an = float(f.grad @ d)
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (fd, an)
        h = 1e-4 * float(nu)
        fd = (Jof(f, nu + h) - Jof(f, nu - h)) / (2 * h)
        assert abs(fd - float(nu.grad)) <= 1e-4 * abs(fd), (fd, float(nu.grad))
    G.close()

"""The masked multigrid of the step (reading R34), pinned on the oracle: the velocity
space of the coarse masked grid (h = 2/m) is a subspace of the fine one (h = 1/m) with the
same Dirichlet and outflow roles, so the rediscretised coarse operator equals the Galerkin
product P^T A_f P over the free nodes, P the Q2 interpolation (the quadratic Lagrange basis
of the coarse element evaluated at the fine nodes, t = 0, 1/4, 1/2, 3/4)."""
import numpy as np
import pytest

from oracle import step


def _lagrange(t):
    return np.array([2.0 * (t - 0.5) * (t - 1.0), -4.0 * t * (t - 1.0), 2.0 * t * (t - 0.5)])


def _interp_1d(nf_lattice, nc_lattice):
    """Fine lattice index i -> coarse lattice weights (coarse element of side 4 fine steps)."""
    P = np.zeros((nf_lattice, nc_lattice))
    for i in range(nf_lattice):
        E, r = divmod(i, 4)
        if r == 0:
            P[i, 2 * E] = 1.0
        elif r == 2:
            P[i, 2 * E + 1] = 1.0
        else:
            P[i, 2 * E: 2 * E + 3] = _lagrange(r / 4.0)
    return P


@pytest.mark.parametrize("m", [2, 4])
def test_rediscretised_coarse_operator_is_galerkin(m):
    gf, gc = step.step_grid(m), step.step_grid(m // 2)
    sf, sc = step.StepSystem(gf, 1.0 / 50.0), step.StepSystem(gc, 1.0 / 50.0)
    Px = _interp_1d(gf.Nx, gc.Nx)
    Py = _interp_1d(gf.Ny, gc.Ny)
    P = np.kron(Py, Px)                      # lattice index j * Nx + i, x fastest
    ff, fc = ~gf.fixed, ~gc.fixed
    Af = sf.Anu.toarray()[: gf.nv, : gf.nv][np.ix_(ff, ff)]
    Ac = sc.Anu.toarray()[: gc.nv, : gc.nv][np.ix_(fc, fc)]
    Pfc = P[np.ix_(ff, fc)]
    G = Pfc.T @ Af @ Pfc
    assert np.abs(G - Ac).max() <= 1e-12 * np.abs(Ac).max()
    # every free fine node's interpolant only involves coarse nodes of an active element
    assert np.abs(P[np.ix_(ff, ~gc.q2_active)]).max() == 0.0

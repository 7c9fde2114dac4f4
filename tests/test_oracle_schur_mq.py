"""Reading R17 pinned on the oracle: the Schur complement S = Qk - R^T Q0^{-1} R of the
two-field pressure mass M_Q (Sec. 2.3) and the Q1 Laplacian K1 share their null vector
(the constant) and satisfy h^2/24 K1 <= S <= h^2/12 K1, element by element and hence for
the assembled matrices, so a Q1-Laplacian V-cycle scaled by 16/h^2 approximates S^+ within
a factor two whatever the grid."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import fem


@pytest.mark.parametrize("n", [4, 8])
def test_schur_of_pressure_mass_between_scaled_laplacians(n):
    g = fem.Grid(n)
    MQ, Qk, R, Q0 = fem.pressure_mass(g)
    S = (Qk - R.T @ sp_inv_diag(Q0) @ R).toarray()
    K1 = fem.q1_stiffness(g).toarray()
    h2 = g.hx * g.hy
    one = np.ones(g.n1)
    assert np.abs(S @ one).max() <= 1e-13 * np.abs(S).max()
    assert np.abs(K1 @ one).max() <= 1e-13 * np.abs(K1).max()
    # pencil on the complement of the constant
    W = sla.null_space(one[None, :])
    ev = sla.eigh(W.T @ S @ W, W.T @ K1 @ W, eigvals_only=True)
    assert ev.min() >= h2 / 24.0 * (1 - 1e-10) and ev.max() <= h2 / 12.0 * (1 + 1e-10), (ev.min() / h2, ev.max() / h2)


def test_element_eigenvalues():
    g = fem.Grid(1, 0.0, 1.0, 0.0, 1.0)
    MQ, Qk, R, Q0 = fem.pressure_mass(g)
    S = (Qk - R.T @ sp_inv_diag(Q0) @ R).toarray()
    h2 = g.hx * g.hy
    ev = np.sort(np.linalg.eigvalsh(S)) / h2
    assert np.allclose(ev, [0.0, 1.0 / 36.0, 1.0 / 12.0, 1.0 / 12.0], atol=1e-14)
    evk = np.sort(np.linalg.eigvalsh(fem.q1_stiffness(g).toarray()))
    assert np.allclose(evk, [0.0, 2.0 / 3.0, 1.0, 1.0], atol=1e-14)


def sp_inv_diag(D):
    return sp.diags(1.0 / D.diagonal())

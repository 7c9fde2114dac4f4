"""The preconditioner of the step's Ap solves (reading R33), pinned on the oracle: the
PCD matrix Ap = B1 Md^{-1} B1^T over the free velocity columns (Sec. 3.1) and the Q1
Laplacian of the active elements plus a unit shift on the outflow column are spectrally
equivalent with a constant that does not grow under refinement, so a fixed number of
CG steps preconditioned by the latter's V-cycle is a mesh-independent approximation of
Ap^{-1}.  Without the shift the Laplacian is singular on the constants while Ap is not."""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import fem, step


def _pencil(m):
    g = step.step_grid(m)
    s = step.StepSystem(g, 1.0 / 50.0)
    md = s.Mv.diagonal()
    inv = np.where(md > 0.0, 1.0 / np.where(md > 0.0, md, 1.0), 0.0)
    Ap = (s.B1I @ sp.diags(np.concatenate([inv, inv])) @ s.B1I.T).toarray()
    act = g.q1_active
    Ap = Ap[np.ix_(act, act)]
    K1 = fem.q1_stiffness(g).toarray()[np.ix_(act, act)]
    col = (np.arange(g.n1) % (g.nx + 1))[act]
    D = np.diag((col == g.nx).astype(float))
    return Ap, K1, D


def test_ap_spectrally_equivalent_to_shifted_laplacian():
    ratios = []
    for m in (1, 2, 4):
        Ap, K1, D = _pencil(m)
        ev = sla.eigh(Ap, K1 + D, eigvals_only=True)
        assert ev.min() > 0.25 and ev.max() < 10.0, (m, ev.min(), ev.max())
        ratios.append(ev.max() / ev.min())
    assert max(ratios) <= 25.0 and ratios[-1] <= 1.05 * ratios[0], ratios


def test_unshifted_laplacian_singular_but_ap_not():
    Ap, K1, D = _pencil(2)
    one = np.ones(K1.shape[0])
    assert np.abs(K1 @ one).max() <= 1e-12 * np.abs(K1).max()
    assert np.linalg.norm(Ap @ one) >= 1e-3 * np.linalg.norm(Ap, 2) * np.linalg.norm(one)

"""The Stokes step of the inflow-outflow Picard iteration and the PCD Schur block
(Sec. 3, Test problem 3; Sec. 3.1, Eq. discrete-commutator1x): why the first Picard
step needs the Stokes limit of the commutator.

* With no wind the Robin term vanishes and F1 = nu K1 annihilates the constants on the
  active Q1 nodes, so M_S^{-1} = Ap^{-1} F1 Q1^{-1} maps Q1 * 1 to zero: it is singular.
* The Schur complement of the outflow problem, B1 F^{-1} B1^T, is not singular: the
  constant pressure is not in ker B1^T once the outflow velocities are free.
* The Stokes limit F1 = nu Ap (the commutator's own requirement for F = nu A) gives
  M_S^{-1} = nu Q1^{-1}, nonsingular, and the two-stage method with it reaches the
  direct solution.
"""
import numpy as np

from oracle import krylov, step
from paper_2303_10233_gb300 import workloads as W


class _StokesLimitPCD1(step.StepPCD1):
    """StepPCD1 with M_S^{-1} = nu Q1^{-1} (the commutator with F1 = nu Ap)."""

    def schur_inv(self, rp):
        return self.sys.nu * self.Q1solve(rp)


def _stokes(m):
    w = W.step(m)
    g = step.step_grid(m)
    return w, g, step.StepSystem(g, w["nu"])


def test_literal_pcd_is_singular_for_stokes():
    w, g, s = _stokes(2)
    pcd = step.StepPCD1(s)
    one = g.q1_active.astype(float)
    f1_one = (pcd.F1 @ one)[g.q1_active]
    assert np.abs(f1_one).max() <= 1e-13 * np.abs(pcd.F1).max()
    q1_one = (s.Qk + s.pin1) @ one
    assert np.abs(pcd.schur_inv(q1_one)[g.q1_active]).max() <= 1e-12


def test_outflow_schur_complement_is_nonsingular():
    w, g, s = _stokes(1)
    act = g.q1_active
    B1 = s.B1I.toarray()[act]
    S = B1 @ np.linalg.solve(s.F.toarray(), B1.T)
    sv = np.linalg.svd(S, compute_uv=False)
    assert sv[-1] >= 1e-6 * sv[0]
    # and it does not annihilate the constant
    one = np.ones(act.sum())
    assert np.linalg.norm(S @ one) >= 1e-3 * np.linalg.norm(S, 2) * np.linalg.norm(one)


def test_stokes_limit_two_stage_reaches_direct_solution():
    w, g, s = _stokes(2)
    b = s.rhs(w["ubc"])
    xd = s.solve(b)
    x, info = krylov.two_stage(s, b, eta=1e-10, pcd_cls=_StokesLimitPCD1, m1_cls=step.StepM1, maxit=400)
    k = s.k
    p = x[g.nu:] - (k @ x[g.nu:]) / (k @ k) * k
    x = np.concatenate([x[: g.nu], p])
    assert np.linalg.norm(b - s.K @ x) <= 1e-10 * 1.01 * np.linalg.norm(b)
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)
    assert info["its1"] <= 40, info["its1"]

"""Krylov solvers and block preconditioners in FP64 (test infrastructure only).

* ``minres``      -- preconditioned MINRES, Algorithm 1 of the paper (Lanczos
                     three-term recurrence with Givens rotations), steps taken
                     in the paper's order and notation.
* ``P1``          -- the block-diagonal preconditioner blkdiag(F, (1/nu) M_Q)
                     with exact solves (Sec. 2.4, "P_1"); the M_Q solve is the
                     augmented (Lagrange-multiplier) system of Sec. 2.2, which
                     returns z orthogonal to k.
* ``gmres``       -- right-preconditioned restarted GMRES; the least-squares
                     problem of each cycle is solved with ``numpy.linalg.lstsq``
                     (the plain definition: minimum residual over the Krylov
                     space).
* ``M1``          -- block-triangular [F B^T; 0 -(1/nu) M_Q] (Eq. nse-precon-ref).
* ``PCD1``        -- block-triangular [F B1^T; 0 -M_S] with the Q1 PCD Schur
                     approximation M_S^{-1} = Ap^{-1} F1 Q1^{-1}
                     (Eq. discrete-commutator1x, Ap = B1 Md^{-1} B1^T, Md the
                     diagonal of the velocity mass matrix).
* ``two_stage``   -- the two-stage PCD method of Sec. 3.1 (Step I on the
                     reduced system to c*eta, Step II on the full system with
                     M_1 from [u1*, q1*, 0] to eta), returning the Prop. 2
                     quantities at the switch.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem
from .direct import bordered_solve


# ---------------------------------------------------------------------------
# Algorithm 1: preconditioned MINRES
# ---------------------------------------------------------------------------
def minres(K, Pinv, b, x0, tol=1e-8, maxit=1000, true_tol=None):
    """Preconditioned MINRES (Algorithm 1).

    K: callable x -> K x (symmetric); Pinv: callable r -> z solving P z = r
    (P symmetric positive semi-definite).  Stops when |eta_j| / eta_1 < tol,
    i.e. the P^{-1}-norm of the residual is reduced by ``tol`` (Sec. 2.4), or,
    when ``true_tol`` is given, additionally requires the Euclidean residual
    ||b - K x|| <= true_tol * ||b|| (checked when the eta test first passes).
    Returns (x, info) with info["its"], info["eta"] (history of |eta|) and the
    coefficients of the preconditioned Lanczos process the recurrence runs on:
    info["delta"] = [delta_1 .. delta_k] (diagonal of T_k) and info["gamma"] =
    [gamma_1 .. gamma_{k+1}] (gamma_2 .. gamma_k off the diagonal of T_k,
    gamma_{k+1} the entry below it in T_{k+1,k}).
    """
    x = np.array(x0, dtype=np.float64, copy=True)
    v_old = np.zeros_like(x)                    # v^(j-1), starts as v^(0) = 0
    w_old = np.zeros_like(x)                    # w^(j-1), starts as w^(0) = 0
    w = np.zeros_like(x)                        # w^(j),   starts as w^(1) = 0
    gamma_old = 0.0                             # gamma_{j-1}, gamma_0 = 0
    v = b - K(x)                                # v^(1)
    z = Pinv(v)                                 # P z^(1) = v^(1)
    gamma = np.sqrt(np.dot(z, v))               # gamma_1
    eta = gamma
    s_old = s = 0.0                             # s_0, s_1
    c_old = c = 1.0                             # c_0, c_1
    hist = [abs(eta)]
    deltas, gammas = [], [gamma]
    eta1 = abs(eta)
    bnorm = np.linalg.norm(b)
    its = 0
    if eta1 == 0.0:
        return x, {"its": 0, "eta": hist, "delta": deltas, "gamma": gammas}
    for j in range(1, maxit + 1):
        z = z / gamma
        Kz = K(z)
        delta = np.dot(Kz, z)
        v_new = Kz - (delta / gamma) * v
        if gamma_old != 0.0:
            v_new -= (gamma / gamma_old) * v_old
        z_new = Pinv(v_new)
        gamma_new = np.sqrt(np.dot(z_new, v_new))
        deltas.append(delta)
        gammas.append(gamma_new)
        a0 = c * delta - c_old * s * gamma
        a1 = np.sqrt(a0 * a0 + gamma_new * gamma_new)
        a2 = s * delta + c_old * c * gamma
        a3 = s_old * gamma
        c_new = a0 / a1
        s_new = gamma_new / a1
        w_new = (z - a3 * w_old - a2 * w) / a1
        x = x + (c_new * eta) * w_new
        eta = -s_new * eta
        # advance the recurrence: index j+1 becomes j
        v_old, v = v, v_new
        z = z_new
        w_old, w = w, w_new
        gamma_old, gamma = gamma, gamma_new
        c_old, c = c, c_new
        s_old, s = s, s_new
        its = j
        hist.append(abs(eta))
        if abs(eta) / eta1 < tol:
            if true_tol is None or np.linalg.norm(b - K(x)) <= true_tol * bnorm:
                break
        if gamma == 0.0:
            break
    return x, {"its": its, "eta": hist, "delta": deltas, "gamma": gammas}


# ---------------------------------------------------------------------------
# exact block solvers
# ---------------------------------------------------------------------------
class _LU:
    def __init__(self, M):
        self.lu = spla.splu(sp.csc_matrix(M), permc_spec="COLAMD")

    def __call__(self, r):
        return self.lu.solve(r)


class MQSolve:
    """Augmented solve [M_Q k; k^T 0][z; lambda] = [r; 0] (Sec. 2.2): z solves
    M_Q z = r (r consistent) and k^T z = 0 (Euclidean)."""

    def __init__(self, sys):
        self.k = sys.k
        aug = sp.bmat([[sys.MQ, sp.csr_matrix(self.k[:, None])],
                       [sp.csr_matrix(self.k[None, :]), None]])
        self.lu = _LU(aug)

    def __call__(self, r):
        return self.lu(np.concatenate([r, [0.0]]))[:-1]


class NullSolve:
    """Solve a symmetric singular M z = r - (mean) with z orthogonal to 1."""

    def __init__(self, M):
        nn = M.shape[0]
        one = np.ones(nn)
        aug = sp.bmat([[M, sp.csr_matrix(one[:, None])], [sp.csr_matrix(one[None, :]), None]])
        self.lu = _LU(aug)

    def __call__(self, r):
        r = r - r.mean()
        return self.lu(np.concatenate([r, [0.0]]))[:-1]


class P1:
    """blkdiag(F_velocity, (1/nu) M_Q) with exact solves (Sec. 2.4, P_1).

    F_velocity is the Stokes velocity block nu*A with identity boundary rows.
    The pressure part returns nu * M_Q^+ r with z orthogonal to k.
    """

    def __init__(self, sys):
        self.sys = sys
        self.Asolve = _LU(sys.Anu)
        self.MQ = MQSolve(sys)

    def __call__(self, r):
        nu_ = self.sys.g.nu
        return np.concatenate([self.Asolve(r[:nu_]), self.sys.nu * self.MQ(r[nu_:])])


class PIdeal:
    """blkdiag(A, B A^{-1} B^T) with the pressure block pseudo-inverted on the
    complement of span{e1, e0} (Sec. 2: P_ideal).  Dense: tiny grids only."""

    def __init__(self, sys):
        self.sys = sys
        self.Asolve = _LU(sys.Anu)
        BI = sys.BI.toarray()
        Ainv_Bt = np.column_stack([self.Asolve(BI[i]) for i in range(BI.shape[0])])
        S = BI @ Ainv_Bt
        self.Spinv = np.linalg.pinv(S, rcond=1e-10, hermitian=True)

    def __call__(self, r):
        nu_ = self.sys.g.nu
        return np.concatenate([self.Asolve(r[:nu_]), self.Spinv @ r[nu_:]])


# ---------------------------------------------------------------------------
# GMRES (right preconditioning)
# ---------------------------------------------------------------------------
def gmres(K, Minv, b, x0, tol_abs, restart=50, maxit=2000):
    """Restarted right-preconditioned GMRES(m) on K x = b.

    Builds the Arnoldi basis V of K M^{-1} by modified Gram-Schmidt, keeps
    Z = M^{-1} V (flexible storage, identical to right preconditioning for a
    fixed M), and minimises ||beta e_1 - H y|| by least squares.  Stops when
    the Euclidean residual norm (Eq. residual-norm) is <= tol_abs.
    Returns (x, info) with info["its"] and info["res"] (residual history).
    """
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - K(x)
    beta = np.linalg.norm(r)
    hist = [beta]
    its = 0
    while beta > tol_abs and its < maxit:
        m = restart
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        y = None
        for j in range(m):
            Z.append(Minv(V[j]))
            wv = K(Z[j])
            for i in range(j + 1):
                H[i, j] = np.dot(wv, V[i])
                wv = wv - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(wv)
            rhs = np.zeros(j + 2); rhs[0] = beta
            y, *_ = np.linalg.lstsq(H[: j + 2, : j + 1], rhs, rcond=None)
            res = np.linalg.norm(rhs - H[: j + 2, : j + 1] @ y)
            its += 1
            hist.append(res)
            if res <= tol_abs or its >= maxit or H[j + 1, j] == 0.0:
                break
            V.append(wv / H[j + 1, j])
        for i, yi in enumerate(y):
            x = x + yi * Z[i]
        r = b - K(x)
        beta = np.linalg.norm(r)
        hist[-1] = beta
    return x, {"its": its, "res": hist}


class M1:
    """[F B^T; 0 -(1/nu) M_Q]^{-1} (Eq. nse-precon-ref), exact blocks:
    z_p = -nu M_Q^+ r_p (z_p orthogonal to k), z_u = F^{-1}(r_u - B^T z_p)."""

    def __init__(self, sys):
        self.sys = sys
        self.Fsolve = _LU(sys.F)
        self.MQ = MQSolve(sys)

    def __call__(self, r):
        s = self.sys
        nu_ = s.g.nu
        zp = -s.nu * self.MQ(r[nu_:])
        zu = self.Fsolve(r[:nu_] - s.BI.T @ zp)
        return np.concatenate([zu, zp])


class PCD1:
    """[F B1^T; 0 -M_S]^{-1} on the reduced system (Step I of Sec. 3.1).

    M_S^{-1} r = Ap^{-1} F1 Q1^{-1} r  (Eq. discrete-commutator1x), with
    Q1 the Q1 mass, F1 = nu*K1 + N1(w) and Ap = B1 Md^{-1} B1^T over interior
    velocity columns (Md = diag of the velocity mass matrix); Ap is singular
    with the constants, so its solve projects them out.
    """

    def __init__(self, sys):
        self.sys = sys
        g = sys.g
        self.Fsolve = _LU(sys.F)
        self.Q1solve = _LU(sys.Qk)
        K1 = fem.q1_stiffness(g)
        self.F1 = sys.nu * K1
        if sys.wind is not None:
            self.F1 = self.F1 + fem.q1_convection(g, sys.wind)
        self.F1 = self.F1.tocsr()
        md = sys.Mv.diagonal()
        Mdinv = sp.diags(np.concatenate([1.0 / md, 1.0 / md]))
        self.Ap = (sys.B1I @ Mdinv @ sys.B1I.T).tocsr()
        self.Apsolve = NullSolve(self.Ap)

    def schur_inv(self, rp):
        return self.Apsolve(self.F1 @ self.Q1solve(rp))

    def __call__(self, r):
        s = self.sys
        nu_ = s.g.nu
        zp = -self.schur_inv(r[nu_:])
        zu = self.Fsolve(r[:nu_] - s.B1I.T @ zp)
        return np.concatenate([zu, zp])


def two_stage(sys, b, eta=1e-6, c=10.0, restart=50, maxit=2000, x0=None, pcd_cls=None, m1_cls=None):
    """Two-stage PCD solve of Sec. 3.1.

    Step I: GMRES + PCD1 on the reduced system [F B1^T; B1 0][u; q1] = [f; g1]
    until its residual is <= c*eta*||b_red||.  Step II: GMRES + M1 on the full
    system from [u1*, q1*, 0] until ||b - K x|| <= eta*||b||.
    ``x0`` defaults to the lifted boundary data (interior zero).  ``pcd_cls`` and
    ``m1_cls`` replace the Step I and Step II preconditioner classes (default PCD1
    and M1, for the enclosed square; other domains bring their own).
    Returns (x, info) with the iteration counts and the Prop. 2 quantities
    (||z*||^2 and the bound c^2 eta^2 ||b_red||^2 + ||r0*||^2, where r0* is the
    P0 block of the residual at the switch; it equals B0 u1* when g0 = 0).
    """
    g = sys.g
    nu_, n1 = g.nu, g.n1
    if x0 is None:
        x0 = np.concatenate([sys.DB @ b[:nu_], np.zeros(g.np_)])
    bred = b[: nu_ + n1]
    Kred = lambda v: sys.K1 @ v
    pcd = (pcd_cls or PCD1)(sys)
    nb_red = np.linalg.norm(bred)
    x1, info1 = gmres(Kred, pcd, bred, x0[: nu_ + n1], c * eta * nb_red, restart, maxit)
    xs = np.concatenate([x1, np.zeros(g.n0)])
    zs = b - sys.K @ xs
    z2 = float(np.dot(zs, zs))
    r0 = zs[nu_ + n1:]
    bound = (c * eta * nb_red) ** 2 + float(np.dot(r0, r0))
    m1 = (m1_cls or M1)(sys)
    x, info2 = gmres(lambda v: sys.K @ v, m1, b, xs, eta * np.linalg.norm(b), restart, maxit)
    return x, {"its1": info1["its"], "its2": info2["its"], "res1": info1["res"],
               "res2": info2["res"], "z_star_sq": z2, "prop2_bound": bound,
               "B0u1_sq": float(np.linalg.norm(sys.B0I @ x1[:nu_]) ** 2)}

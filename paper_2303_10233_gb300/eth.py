"""Thin ctypes binding of the C ABI in ``include/eth.h`` (argument marshalling only).

Every numerical step runs in the CUDA library ``_lib/libeth.so``; this module
only converts torch tensors to device pointers and option dicts to the
``eth_opts`` struct.  Importing it fails loudly when the library is missing:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libeth.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "eth.h")

STOKES, OSEEN = 0, 1
OPS = {"K": 0, "KT": 1, "A": 2, "F": 3, "B": 4, "BT": 5, "MQ": 6, "MV": 7, "K1": 8, "K1T": 9}
STATUS = {0: "ok", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCONV", 5: "EBREAKDOWN",
          6: "EINCONSISTENT", 7: "ETIMEOUT", 8: "ENAN"}
# statuses that still come with a meaningful result (returned, status in the stats):
# tolerance not reached, and a right-hand side whose null-space component was removed
SOFT = (0, 4, 6)


class EthError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("restart", ctypes.c_int),
                ("c_stage", ctypes.c_double), ("precision", ctypes.c_int), ("mg_pre", ctypes.c_int),
                ("mg_post", ctypes.c_int), ("mg_min_n", ctypes.c_int), ("mq_mode", ctypes.c_int),
                ("a_exact", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("refine_inner_tol", ctypes.c_double), ("graph", ctypes.c_int), ("verbose", ctypes.c_int),
                ("autotune", ctypes.c_int), ("restart_max", ctypes.c_int), ("mg_omega", ctypes.c_double),
                ("oseen_prec", ctypes.c_int), ("lsc_cg", ctypes.c_int), ("mq_cheb_steps", ctypes.c_int),
                ("mq_cheb_a", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("iters_stage1", ctypes.c_int), ("iters_stage2", ctypes.c_int),
                ("refine_passes", ctypes.c_int), ("iters_total", ctypes.c_int),
                ("relres_true", ctypes.c_double), ("relres0", ctypes.c_double),
                ("prop2_lhs", ctypes.c_double), ("prop2_bound", ctypes.c_double),
                ("seconds", ctypes.c_double), ("alg_bytes", ctypes.c_double),
                ("status", ctypes.c_int), ("kernel_launches", ctypes.c_int),
                ("escalations", ctypes.c_int), ("tile_rows", ctypes.c_int),
                ("tile_persistent", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path=LIB_PATH):
    """Loads libeth.so (build it with ``paper_2303_10233_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    pi = ctypes.POINTER(ctypes.c_int)
    sig = {
        "eth_sizes": (i, [i, pi, pi, pi]),
        "eth_status_string": (ctypes.c_char_p, [i]),
        "eth_last_error": (ctypes.c_char_p, []),
        "eth_default_opts": (None, [ctypes.POINTER(Opts)]),
        "eth_grid_create": (i, [i, d, d, d, d, i, vp, ctypes.POINTER(vp)]),
        "eth_grid_destroy": (None, [vp]),
        "eth_grid_set_tile": (i, [vp, i, i]),
        "eth_set_coefficients": (i, [vp, d, vp]),
        "eth_set_rhs": (i, [vp, vp, vp]),
        "eth_get_rhs": (i, [vp, vp]),
        "eth_solve": (i, [vp, ctypes.POINTER(Opts), vp, vp, ctypes.POINTER(Stats)]),
        "eth_solve_host": (i, [vp, ctypes.POINTER(Opts), vp, vp, vp, vp, ctypes.POINTER(Stats)]),
        "eth_solve_adjoint": (i, [vp, ctypes.POINTER(Opts), vp, vp, vp, vp, ctypes.POINTER(Stats)]),
        "eth_picard": (i, [vp, ctypes.POINTER(Opts), vp, vp, i, vp, vp, ctypes.POINTER(d), ctypes.POINTER(Stats)]),
        "eth_apply": (i, [vp, i, i, vp, vp]),
        "eth_lanczos": (i, [vp, i, vp, vp, pi]),
        "eth_est_infsup": (i, [vp, vp, vp, i, vp]),
        "eth_adjoint_gradients": (i, [vp, vp, vp, vp, ctypes.POINTER(d)]),
        "eth_apply_k_dot_static": (i, [i, d, d, d, d, d, i, vp, vp, vp, vp]),
        "eth_apply_pcd": (i, [vp, i, i, i, i, vp, vp]),
        "eth_apply_mqcheb": (i, [vp, i, i, d, d, vp, vp]),
        "eth_mask_roles": (i, [i, i, vp, i, vp, vp, vp]),
        "eth_mgrid_create": (i, [i, i, d, d, d, vp, i, vp, ctypes.POINTER(vp)]),
        "eth_mgrid_destroy": (None, [vp]),
        "eth_mgrid_sizes": (i, [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
        "eth_mgrid_roles": (i, [vp, vp, vp, vp, pi, pi]),
        "eth_mgrid_set_coefficients": (i, [vp, d, vp]),
        "eth_mgrid_apply": (i, [vp, i, vp, vp]),
        "eth_mgrid_rhs": (i, [vp, vp, vp]),
        "eth_mgrid_solve": (i, [vp, ctypes.POINTER(Opts), vp, vp, ctypes.POINTER(Stats)]),
        "eth_mgrid_picard": (i, [vp, ctypes.POINTER(Opts), vp, i, vp, vp, ctypes.POINTER(d), ctypes.POINTER(Stats)]),
        "eth_batch_create": (i, [i, ctypes.POINTER(vp), ctypes.POINTER(vp)]),
        "eth_batch_solve": (i, [vp, ctypes.POINTER(Opts), ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(Stats)]),
        "eth_batch_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def header_functions(path=HEADER):
    """Names of the functions declared in include/eth.h."""
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eth_[a-z_0-9]+)\s*\(", src)))


def _check(st):
    if st != 0:
        raise EthError(st, load().eth_last_error().decode())


def sizes(n):
    nv, n1, n0 = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    nt = load().eth_sizes(n, ctypes.byref(nv), ctypes.byref(n1), ctypes.byref(n0))
    return nv.value, n1.value, n0.value, nt


def make_opts(**kw):
    o = Opts()
    load().eth_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(f"unknown option {k}")
        if k == "precision" and isinstance(v, str):
            v = {"fp64": 0, "mixed": 1}[v]
        if k == "oseen_prec" and isinstance(v, str):
            v = {"pcd": 0, "lsc": 1}[v]
        if k == "mq_mode" and isinstance(v, str):
            v = {"vcycle": 0, "exact": 1, "cheb": 2}[v]
        setattr(o, k, v)
    return o


def _ptr(t, numel=None, device=None):
    """Device pointer of a contiguous CUDA float64 tensor; with ``numel`` its
    length and with ``device`` its device are checked first (the C ABI takes raw
    pointers and cannot check either)."""
    import torch
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA float64 tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    if device is not None and t.device != device:
        raise ValueError(f"tensor on {t.device}, the grid lives on {device}")
    return ctypes.c_void_p(t.data_ptr())


class Grid:
    """Handle of one n x n Q2--Q1* problem (wraps eth_grid)."""

    def __init__(self, n, kind="stokes", domain=(-1.0, 1.0, -1.0, 1.0), stream=None, device=None):
        import torch
        L = load()
        self.n = int(n)
        self.kind = OSEEN if kind in ("oseen", OSEEN) else STOKES
        self.nv, self.n1, self.n0, self.nt = sizes(self.n)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        if self.stream.device != self.device:
            raise ValueError(f"stream of {self.stream.device} for a grid on {self.device}")
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):   # the handle belongs to the device current at creation
            _check(L.eth_grid_create(self.n, *map(float, domain), self.kind,
                                     ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h

    def _p(self, t, numel):
        return _ptr(t, numel, self.device)

    def close(self):
        if getattr(self, "h", None):
            load().eth_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _zeros(self, m):
        import torch
        return torch.zeros(m, dtype=torch.float64, device=self.device)

    def set_coefficients(self, nu, wind=None):
        self._wind = wind
        _check(load().eth_set_coefficients(self.h, float(nu), self._p(wind, 2 * self.nv)))

    def set_tile(self, rows, persistent=0):
        """Pins the fused K apply's form: tiles of 32 x rows elements (rows in {4, 8, 16}); persistent=1:
        the persistent pipelined form (rows = 8); persistent=2: the warp-strip form with `rows` element
        rows per warp (4, 8, 16, 32); rows = 0 re-enables tuning."""
        _check(load().eth_grid_set_tile(self.h, int(rows), int(persistent)))

    def set_rhs(self, f_nodal, ubc):
        _check(load().eth_set_rhs(self.h, self._p(f_nodal, 2 * self.nv), self._p(ubc, 2 * self.nv)))

    def rhs(self):
        b = self._zeros(self.nt)
        _check(load().eth_get_rhs(self.h, self._p(b, self.nt)))
        return b

    def _op_sizes(self, op):
        u2, pp, u1 = 2 * self.nv, self.n1 + self.n0, 2 * self.nv + self.n1
        return {"K": (self.nt, self.nt), "KT": (self.nt, self.nt), "A": (u2, u2), "F": (u2, u2), "MV": (u2, u2),
                "B": (u2, pp), "BT": (pp, u2), "MQ": (pp, pp), "K1": (u1, u1), "K1T": (u1, u1)}[op]

    def apply(self, op, x, fp32=False):
        nin, nout = self._op_sizes(op)
        y = self._zeros(nout)
        _check(load().eth_apply(self.h, OPS[op], int(bool(fp32)), self._p(x, nin), self._p(y, nout)))
        return y

    def apply_pcd(self, rp, cheb_steps=10, ap_its=2, adjoint=False, fp32=False):
        """M_S^{-1} rp = Ap^+ F1 Q1^{-1} rp (the Q1 PCD Schur block of Step I) with the given
        inner step counts; returns the mean-free result (N_1)."""
        zp = self._zeros(self.n1)
        _check(load().eth_apply_pcd(self.h, int(bool(adjoint)), int(bool(fp32)), int(cheb_steps), int(ap_its),
                                    self._p(rp, self.n1), self._p(zp, self.n1)))
        return zp

    def apply_mqcheb(self, r, steps=20, a=0.0, b=0.0, fp32=False):
        """Chebyshev-SGS approximation of M_Q^+ r (the M_cheb block of P_2), k projected out."""
        m = self.n1 + self.n0
        z = self._zeros(m)
        _check(load().eth_apply_mqcheb(self.h, int(bool(fp32)), int(steps), float(a), float(b), self._p(r, m),
                                       self._p(z, m)))
        return z

    def solve(self, u=None, p=None, **opts):
        u = self._zeros(2 * self.nv) if u is None else u
        p = self._zeros(self.n1 + self.n0) if p is None else p
        o = make_opts(**opts)
        st = Stats()
        rc = load().eth_solve(self.h, ctypes.byref(o), self._p(u, 2 * self.nv), self._p(p, self.n1 + self.n0),
                              ctypes.byref(st))
        if rc not in SOFT:
            _check(rc)
        return u, p, st.as_dict()

    def solve_host(self, f_nodal, ubc, **opts):
        f = np.ascontiguousarray(f_nodal, dtype=np.float64)
        ub = np.ascontiguousarray(ubc, dtype=np.float64)
        if f.size != 2 * self.nv or ub.size != 2 * self.nv:
            raise ValueError(f"expected host arrays of {2 * self.nv} elements")
        u = np.zeros(2 * self.nv); p = np.zeros(self.n1 + self.n0)
        o = make_opts(**opts)
        st = Stats()
        c = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        rc = load().eth_solve_host(self.h, ctypes.byref(o), c(f), c(ub), c(u), c(p), ctypes.byref(st))
        if rc not in SOFT:
            _check(rc)
        return u, p, st.as_dict()

    def solve_host_pinned(self, f_pinned, ubc_pinned, u_pinned, p_pinned, **opts):
        """eth_solve_host with caller-owned (pinned) host tensors; returns stats."""
        for t, m in ((f_pinned, 2 * self.nv), (ubc_pinned, 2 * self.nv), (u_pinned, 2 * self.nv),
                     (p_pinned, self.n1 + self.n0)):
            if t.is_cuda or t.dtype != torch_float64() or not t.is_contiguous() or t.numel() != m:
                raise ValueError(f"expected a contiguous host float64 tensor of {m} elements")
        o = make_opts(**opts)
        st = Stats()
        c = lambda t: ctypes.c_void_p(t.data_ptr())
        rc = load().eth_solve_host(self.h, ctypes.byref(o), c(f_pinned), c(ubc_pinned), c(u_pinned),
                                   c(p_pinned), ctypes.byref(st))
        if rc not in SOFT:
            _check(rc)
        return st.as_dict()

    def solve_adjoint(self, ru, rp, **opts):
        lu = self._zeros(2 * self.nv); lp = self._zeros(self.n1 + self.n0)
        o = make_opts(**opts)
        st = Stats()
        nu2, npp = 2 * self.nv, self.n1 + self.n0
        rc = load().eth_solve_adjoint(self.h, ctypes.byref(o), self._p(ru, nu2), self._p(rp, npp), self._p(lu, nu2),
                                      self._p(lp, npp), ctypes.byref(st))
        if rc not in SOFT:
            _check(rc)
        return lu, lp, st.as_dict()


    def picard(self, f_nodal, ubc, steps, **opts):
        """Picard iteration for steady Navier-Stokes (Oseen grid; zero wind first).
        Returns (u, p, nonlinear residual per step, stats per step)."""
        u = self._zeros(2 * self.nv); p = self._zeros(self.n1 + self.n0)
        o = make_opts(**opts)
        res = (ctypes.c_double * steps)()
        st = (Stats * steps)()
        nu2 = 2 * self.nv
        rc = load().eth_picard(self.h, ctypes.byref(o), self._p(f_nodal, nu2), self._p(ubc, nu2), int(steps),
                               self._p(u, nu2), self._p(p, self.n1 + self.n0), res, st)
        if rc not in SOFT:
            _check(rc)
        return u, p, list(res), [s_.as_dict() for s_ in st]

    def lanczos(self):
        """(delta, gamma) of the first MINRES run of the last Stokes solve: delta[j-1] =
        delta_j, gamma[j-1] = gamma_{j+1} (FP64 device tensors)."""
        import torch
        k = ctypes.c_int()
        _check(load().eth_lanczos(self.h, 0, None, None, ctypes.byref(k)))
        d = torch.empty(k.value, dtype=torch.float64, device=self.device)
        gm = torch.empty(k.value, dtype=torch.float64, device=self.device)
        _check(load().eth_lanczos(self.h, k.value, self._p(d, k.value), self._p(gm, k.value), ctypes.byref(k)))
        return d, gm

    def est_infsup(self, delta=None, gamma=None):
        """EST-MINRES estimates of gamma^2 after each MINRES iteration (NaN where none)."""
        if delta is None:
            delta, gamma = self.lanczos()
        k = delta.numel()
        est = self._zeros(k)
        _check(load().eth_est_infsup(self.h, self._p(delta, k), self._p(gamma, k), int(k), self._p(est, k)))
        return est

    def adjoint_gradients(self, lu, u):
        """(grad_f, grad_nu) of J = ||u - u_t||^2 from the adjoint velocity lu."""
        gf = self._zeros(2 * self.nv)
        gn = ctypes.c_double()
        nu2 = 2 * self.nv
        _check(load().eth_adjoint_gradients(self.h, self._p(lu, nu2), self._p(u, nu2), self._p(gf, nu2),
                                            ctypes.byref(gn)))
        return gf, gn.value


def apply_k_dot_static(n, nu, x, y, dot, fp32=False, domain=(-1.0, 1.0, -1.0, 1.0), stream=None):
    """y = K x and dot = <K x, x> for a Stokes grid, through the allocation-free entry point."""
    import torch
    nt = sizes(int(n))[3]
    dev = x.device
    if dot.numel() < 1:
        raise ValueError("dot needs one element")
    px, py, pd = _ptr(x, nt, dev), _ptr(y, nt, dev), _ptr(dot, None, dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    if st.device != dev:
        raise ValueError(f"stream of {st.device} for tensors on {dev}")
    with torch.cuda.device(dev):   # the scratch address is looked up on the current device
        _check(load().eth_apply_k_dot_static(int(n), *map(float, domain), float(nu), int(bool(fp32)), px, py, pd,
                                             ctypes.c_void_p(st.cuda_stream)))


class Batch:
    """Concurrent solves of independent instances (wraps eth_batch)."""

    def __init__(self, grids):
        self.grids = list(grids)
        arr = (ctypes.c_void_p * len(self.grids))(*[g.h.value for g in self.grids])
        h = ctypes.c_void_p()
        _check(load().eth_batch_create(len(self.grids), arr, ctypes.byref(h)))
        self.h = h

    def solve(self, **opts):
        """Solves every instance; returns (velocities, pressures, stats per instance, status)."""
        us = [g._zeros(2 * g.nv) for g in self.grids]
        ps = [g._zeros(g.n1 + g.n0) for g in self.grids]
        ua = (ctypes.c_void_p * len(us))(*[t.data_ptr() for t in us])
        pa = (ctypes.c_void_p * len(ps))(*[t.data_ptr() for t in ps])
        st = (Stats * len(us))()
        o = make_opts(**opts)
        rc = load().eth_batch_solve(self.h, ctypes.byref(o), ua, pa, st)
        return us, ps, [s.as_dict() for s in st], rc

    def close(self):
        if getattr(self, "h", None):
            load().eth_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mask_roles(nx, ny, active, outflow=True):
    """Host-side node roles of a masked grid: (fixed, dirichlet) over the Q2 lattice and the
    active Q1 nodes, as boolean numpy arrays (no device needed)."""
    act = np.ascontiguousarray(np.asarray(active, dtype=bool).reshape(int(ny), int(nx)).astype(np.uint8))
    nv, n1 = (2 * nx + 1) * (2 * ny + 1), (nx + 1) * (ny + 1)
    fx = np.zeros(nv, dtype=np.uint8); dr = np.zeros(nv, dtype=np.uint8); qa = np.zeros(n1, dtype=np.uint8)
    c = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(load().eth_mask_roles(int(nx), int(ny), c(act), int(bool(outflow)), c(fx), c(dr), c(qa)))
    return fx.astype(bool), dr.astype(bool), qa.astype(bool)


class MGrid:
    """Handle of a masked uniform grid (wraps eth_mgrid): the active squares of an
    nx x ny box of square elements of side h from (x0, y0); ``outflow`` makes the
    box's right edge a natural outflow boundary (Sec. 3, Test problem 3)."""

    def __init__(self, nx, ny, h, x0, y0, active, outflow=True, stream=None, device=None):
        import torch
        L = load()
        act = np.ascontiguousarray(np.asarray(active, dtype=bool).reshape(int(ny), int(nx)).astype(np.uint8))
        self.nx, self.ny, self.h = int(nx), int(ny), float(h)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        if self.stream.device != self.device:
            raise ValueError(f"stream of {self.stream.device} for a grid on {self.device}")
        hnd = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(L.eth_mgrid_create(self.nx, self.ny, self.h, float(x0), float(y0),
                                      act.ctypes.data_as(ctypes.c_void_p), int(bool(outflow)),
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(hnd)))
        self.h_ = hnd
        q = [ctypes.c_longlong() for _ in range(4)]
        _check(L.eth_mgrid_sizes(self.h_, *[ctypes.byref(v) for v in q]))
        self.nv, self.n1, self.n0, self.nt = (v.value for v in q)

    def close(self):
        if getattr(self, "h_", None):
            load().eth_mgrid_destroy(self.h_)
            self.h_ = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _p(self, t, numel):
        return _ptr(t, numel, self.device)

    def _zeros(self, m):
        import torch
        return torch.zeros(m, dtype=torch.float64, device=self.device)

    def roles(self):
        """Host arrays (fixed velocity nodes, Dirichlet nodes, active Q1 nodes), the number of
        multigrid levels and the free nodes of the coarsest level."""
        fx = np.zeros(self.nv, dtype=np.uint8); dr = np.zeros(self.nv, dtype=np.uint8)
        qa = np.zeros(self.n1, dtype=np.uint8)
        lv, cf = ctypes.c_int(), ctypes.c_int()
        c = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(load().eth_mgrid_roles(self.h_, c(fx), c(dr), c(qa), ctypes.byref(lv), ctypes.byref(cf)))
        return fx.astype(bool), dr.astype(bool), qa.astype(bool), lv.value, cf.value

    def set_coefficients(self, nu, wind=None):
        self._wind = wind
        _check(load().eth_mgrid_set_coefficients(self.h_, float(nu), self._p(wind, 2 * self.nv)))

    def _op_sizes(self, op):
        u2, pp, u1 = 2 * self.nv, self.n1 + self.n0, 2 * self.nv + self.n1
        return {"K": (self.nt, self.nt), "K1": (u1, u1), "A": (u2, u2), "F": (u2, u2), "B": (u2, pp),
                "BT": (pp, u2), "MQ": (pp, pp)}[op]

    def apply(self, op, x):
        nin, nout = self._op_sizes(op)
        y = self._zeros(nout)
        _check(load().eth_mgrid_apply(self.h_, OPS[op], self._p(x, nin), self._p(y, nout)))
        return y

    def rhs(self, ubc):
        b = self._zeros(self.nt)
        _check(load().eth_mgrid_rhs(self.h_, self._p(ubc, 2 * self.nv), self._p(b, self.nt)))
        return b

    def solve(self, b, **opts):
        x = self._zeros(self.nt)
        o = make_opts(**opts)
        st = Stats()
        rc = load().eth_mgrid_solve(self.h_, ctypes.byref(o), self._p(b, self.nt), self._p(x, self.nt), ctypes.byref(st))
        if rc not in SOFT:
            _check(rc)
        return x, st.as_dict()

    def picard(self, ubc, steps, keep_all=False, **opts):
        """Picard iteration from the Stokes solution; returns (last iterate, every iterate or None,
        nonlinear residual per step, stats per step)."""
        import torch
        x = self._zeros(self.nt)
        xs = torch.zeros(steps * self.nt, dtype=torch.float64, device=self.device) if keep_all else None
        o = make_opts(**opts)
        res = (ctypes.c_double * steps)()
        st = (Stats * steps)()
        rc = load().eth_mgrid_picard(self.h_, ctypes.byref(o), self._p(ubc, 2 * self.nv), int(steps),
                                     self._p(x, self.nt), self._p(xs, steps * self.nt), res, st)
        if rc not in SOFT:
            _check(rc)
        return x, (xs.view(steps, self.nt) if keep_all else None), list(res), [s_.as_dict() for s_ in st]


def torch_float64():
    import torch
    return torch.float64


def problem(w, device=None):
    """Grid with coefficients and right-hand side from a workloads dict."""
    import torch
    g = Grid(w["n"], "oseen" if w.get("wind") is not None else "stokes", device=device)
    dev = g.device
    wind = None if w.get("wind") is None else torch.as_tensor(w["wind"], dtype=torch.float64, device=dev)
    g.set_coefficients(w["nu"], wind)
    g.set_rhs(torch.as_tensor(w["f_nodal"], dtype=torch.float64, device=dev),
              torch.as_tensor(w["ubc"], dtype=torch.float64, device=dev))
    return g

#!/usr/bin/env python
"""Benchmark of the enriched Taylor--Hood Stokes solve on GB300.

Workload: Stokes on a 256 x 256 uniform Q2--Q1* grid of [-1,1]^2 with the
seeded manufactured solution (six sine stream-function modes, seed 0),
MINRES with the block-diagonal preconditioner (one GMG V(1,1) on A, M_Q^+ with
k projected out), FP32 applies and FP64 Krylov recurrences with FP64
iterative refinement, to a 1e-6 relative true residual.

One step = one full solve to tolerance with the inputs resident in HBM.
value = MDoF.iter/s = N_t * MINRES iterations / solve time / 1e6 (summed
over ranks; ranks run independent replicas, no collective in the data path).
The L2 cache (126 MB) is flushed between steps by writing a 512 MB buffer,
outside the per-step CUDA-event timing.

``--impl reference`` times the FP64 CPU oracle (SciPy, exact-block MINRES)
on a bounded number of iterations of the same workload.  The default run also
reports the oracle's whole solve to tolerance (cpu_baseline), the Oseen 512^2
two-stage solve (oseen512), the uneven 64-instance batch (batch64) and the
roofline of the K apply (roofline).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the oracle (CPU baseline / reference arm) may use every host core for its dense
# BLAS work (set before numpy is imported; the GPU path uses no CPU BLAS); its sparse
# products and SuperLU solves run on one core whatever this setting
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, str(os.cpu_count() or 1))

N_GRID = 256
SEED = 0
TOL = 1e-6
METRIC = "MDoF.iter/s, Stokes 256^2 MINRES+GMG to 1e-6 rel. residual"
UNIT = "MDoF.iter/s"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0])); smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# oracle (CPU) sample: exact-block MINRES iterations on the same workload
# ---------------------------------------------------------------------------
def host_info():
    """Host cores and the CPU model line of lscpu (recorded beside the CPU figures)."""
    info = {"os_cpu_count": os.cpu_count(), "blas_threads": os.environ.get("OPENBLAS_NUM_THREADS")}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            k, _, v = ln.partition(":")
            if k.strip() in ("Model name", "Architecture", "CPU(s)", "Thread(s) per core", "Socket(s)"):
                info[k.strip()] = v.strip()
    except Exception:
        pass
    return info


def oracle_to_tolerance(n, tol):
    """The oracle's time to tolerance on the bench workload: Algorithm 1 MINRES with the
    exact P_1 blocks (SuperLU factorisations, timed separately) from the lifted zero
    guess until the true relative residual is <= tol."""
    import numpy as np
    from oracle import fem, krylov, problem
    from paper_2303_10233_gb300 import workloads as W
    w = W.mms(n, seed=SEED)
    g = fem.Grid(n)
    s = problem.System(g, w["nu"], w["wind"])
    b = s.rhs(w["f_nodal"], w["ubc"])
    t = time.perf_counter()
    P = krylov.P1(s)
    tfac = time.perf_counter() - t
    x0 = np.concatenate([s.DB @ b[: g.nu], np.zeros(g.np_)])
    t = time.perf_counter()
    x, info = krylov.minres(lambda v: s.K @ v, P, b, x0, tol=tol, maxit=400, true_tol=tol)
    dt = time.perf_counter() - t
    res = float(np.linalg.norm(b - s.K @ x) / np.linalg.norm(b))
    return info["its"], dt, tfac, res


def oracle_sample(n, iters, setup=None):
    import numpy as np
    from oracle import fem, krylov, problem
    from paper_2303_10233_gb300 import workloads as W
    if setup is None:
        w = W.mms(n, seed=SEED)
        g = fem.Grid(n)
        s = problem.System(g, w["nu"], w["wind"])
        b = s.rhs(w["f_nodal"], w["ubc"])
        t = time.perf_counter()
        P = krylov.P1(s)
        tfac = time.perf_counter() - t
        setup = (g, s, b, P, tfac)
    g, s, b, P, tfac = setup
    x0 = np.concatenate([s.DB @ b[: g.nu], np.zeros(g.np_)])
    t = time.perf_counter()
    x, info = krylov.minres(lambda v: s.K @ v, P, b, x0, tol=1e-30, maxit=iters)
    dt = time.perf_counter() - t
    return info["its"], dt, setup


def _config(nt, ws):
    """The workload both arms run (the reference arm times the oracle on the same one)."""
    return {"workload": "stokes_mms_256", "n": N_GRID, "N_t": nt, "tol": TOL, "precision": "mixed",
            "preconditioner": "blkdiag(GMG V(1,1) Jacobi, M_Q^+ via Q1 V-cycle)",
            "l2": "512 MB buffer written between steps (outside per-step events)",
            "parallelism": f"replicas x{ws}"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2303_10233_gb300 import workloads as W
    nt = W.sizes(N_GRID)[4]
    its, dt, setup = oracle_sample(N_GRID, 2)          # includes the factorisation of the exact blocks
    per_it = dt / max(its, 1)
    budget = 150.0 / max(args.steps + args.warmup, 1)
    m = max(2, min(40, int(budget / max(per_it, 1e-3))))
    for _ in range(args.warmup):
        oracle_sample(N_GRID, m, setup)
    vals, times = [], []
    for _ in range(args.steps):
        its, dt, _ = oracle_sample(N_GRID, m, setup)
        vals.append(nt * its / dt / 1e6)
        times.append(dt)
    value = nt * m * len(times) / sum(times) / 1e6
    sample = (f"{m} MINRES iterations (Algorithm 1, exact P_1 blocks by SuperLU, factorised once in "
              f"{setup[4]:.1f} s, not timed) per step on the 256^2 MMS system, N_t={nt}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(nt, ws),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "host": host_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def aggregate(dist, tot_s, its, device):
    """Whole-job figures of the replicas: the slowest rank's timed seconds (max over
    ranks) and the iterations of all ranks (sum); identity without a process group."""
    if not dist:
        return tot_s, its
    import torch
    tt = torch.tensor([tot_s, its], dtype=torch.float64, device=device)
    mx = tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = tt.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_10233_gb300 import eth, workloads as W

    w = W.mms(N_GRID, seed=SEED)
    G = eth.problem(w, device=local)
    nt = G.nt
    opts = dict(tol=TOL, precision="mixed")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        G.solve(**opts)
    torch.cuda.synchronize()

    clk = Clocks(local)
    clk.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        e0, e1 = evs[k]
        e0.record()
        _, _, st = G.solve(**opts)
        e1.record()
        stats.append(st)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    step_ms = [a.elapsed_time(b) for a, b in evs]
    its = sum(s["iters_total"] for s in stats)
    tot_s = sum(step_ms) / 1e3
    tot_max, its_all = aggregate(dist, tot_s, its, "cuda")
    value = nt * its_all / tot_max / 1e6
    launches = sum(s["kernel_launches"] for s in stats)

    # ---- plain FP64 GPU form (same solve, FP64 applies and FP64 multigrid)
    G.solve(tol=TOL, precision="fp64")
    f64_ms = []
    f64_its = 0
    for k in range(min(5, args.steps)):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, _, st = G.solve(tol=TOL, precision="fp64")
        e1.record()
        torch.cuda.synchronize()
        f64_ms.append(e0.elapsed_time(e1))
        f64_its += st["iters_total"]

    # ---- end to end through the C ABI with pinned host buffers
    nu2 = 2 * G.nv
    fh = torch.from_numpy(np.ascontiguousarray(w["f_nodal"])).pin_memory()
    uh = torch.from_numpy(np.ascontiguousarray(w["ubc"])).pin_memory()
    uo = torch.empty(nu2, dtype=torch.float64).pin_memory()
    po = torch.empty(G.n1 + G.n0, dtype=torch.float64).pin_memory()
    G.solve_host_pinned(fh, uh, uo, po, **opts)
    torch.cuda.synchronize()
    e2e_its = 0
    e2e_t = 0.0
    for k in range(min(10, args.steps)):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = G.solve_host_pinned(fh, uh, uo, po, **opts)
        e1.record()
        torch.cuda.synchronize()
        e2e_t += e0.elapsed_time(e1) / 1e3
        e2e_its += st["iters_total"]
    e2e_value = nt * e2e_its / e2e_t / 1e6 * ws
    h2d = 2 * nu2 * 8
    d2h = nt * 8

    # ---- Oseen 512^2 (two-stage PCD GMRES, nu = 1/100): time to tolerance, mixed and FP64
    oseen = oseen_line(torch, eth, W, local)
    # ---- the uneven 64-instance batch, concurrent mixed vs plain FP64 one at a time
    batch = batch_line(torch, eth, W, local) if not args.no_batch else None
    # ---- the flow over a step (masked grid, natural outflow), five Picard steps at h = 1/32
    stepl = step_line(torch, eth, W, local, cpu=(ws == 1 and not args.no_cpu and rank == 0))

    # ---- roofline of the dominant kernel, timed live on the launching stream
    roof = roofline(G, torch, eth)
    clocks = clk.stop()

    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu:
        its_c, dt_c, tfac, res_c = oracle_to_tolerance(N_GRID, TOL)
        cpu = {"value": nt * its_c / dt_c / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
               "time_to_tol_s": dt_c, "factorisation_s": tfac, "iters": its_c, "relres": res_c,
               "host": host_info(),
               "sample": f"the whole 256^2 MMS solve: {its_c} exact-block MINRES iterations (Algorithm 1, P_1 by "
                         f"SuperLU) to relative residual {res_c:.1e} in {dt_c:.1f} s, factorisation {tfac:.1f} s "
                         f"not included; SciPy sparse products and SuperLU solves use one core (BLAS threads = "
                         f"host cores)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(step_ms), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 applies / f64 Krylov", "data": "synthetic",
        "config": _config(nt, ws),
        "time_to_tol_ms": statistics.median(step_ms),
        "iters_per_solve": its / max(len(stats), 1),
        "relres": max(s["relres_true"] for s in stats),
        "fp64_plain": {"ms": statistics.median(f64_ms) if f64_ms else None,
                       "iters_per_solve": f64_its / max(len(f64_ms), 1),
                       "speedup_mixed_vs_fp64": (statistics.median(f64_ms) / statistics.median(step_ms)) if f64_ms else None},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roof,
        "oseen512": oseen,
        "batch64": batch,
        "step": stepl,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "wall_s": t_wall,
    }
    print(json.dumps(line), flush=True)
    G.close()
    if dist:
        dist.destroy_process_group()


def _kernel_hash():
    """Hash of the sources of the roofline kernel, the warp-strip fused K apply (its
    header, the element helpers of the tile header and the conversions of common.cuh)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("q2strip.cuh", "q2tile.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2303_10233_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(rows):
    """DRAM bytes per launch of the roofline kernel from the committed ncu summary,
    or None when the kernel sources changed since that capture or it was taken with
    another number of element rows per warp."""
    path = os.path.join(ROOT, "profiles", "kapply_strip_stokes_1024_fp32.txt")
    try:
        kv = dict(line.split("=", 1) for line in open(path).read().split("\n") if "=" in line)
        if kv.get("kernel_source_hash", "").strip() != _kernel_hash():
            return None
        if int(kv.get("rows", "0")) != rows:
            return None
        return float(kv["dram_bytes_read"]) + float(kv["dram_bytes_write"])
    except Exception:
        return None


def oseen_line(torch, eth, W, dev, steps=3):
    """The Oseen workload on 512^2 (seeded wind, nu = 1/100, lid-driven cavity): median
    CUDA-event time to a 1e-6 true residual of the mixed-precision two-stage PCD solve
    (GMRES(50), adaptive restart to 160) and of the plain FP64 form, iterations of both
    stages, and N_t x iterations / time."""
    w = W.oseen_cavity(512, nu=0.01, seed=1)
    O = eth.problem(w, device=dev)
    opts = dict(tol=TOL, restart_max=160, maxit=4000)
    out = {"workload": "oseen_cavity_512_nu0.01", "N_t": O.nt}
    for prec in ("mixed", "fp64"):
        O.solve(precision=prec, **opts)
        ms, sts = [], []
        for _ in range(steps if prec == "mixed" else 2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, _, st = O.solve(precision=prec, **opts)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            sts.append(st)
        its = sts[-1]["iters_total"]
        t = statistics.median(ms)
        out[prec] = {"ms": t, "iters": [sts[-1]["iters_stage1"], sts[-1]["iters_stage2"]],
                     "relres": max(x["relres_true"] for x in sts), "status": sts[-1]["status"],
                     "mdof_iter_s": O.nt * its / (t / 1e3) / 1e6}
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms"] / out["mixed"]["ms"]
    O.close()
    return out


def batch_line(torch, eth, W, dev):
    """The seeded uneven batch (64 Stokes / Oseen instances, n in {32, 64, 128, 256},
    nu log-uniform in [1e-3, 1e-1]): wall time of one concurrent mixed-precision batch
    solve to 1e-6 (Oseen instances with the LSC preconditioner M_3), after a warm-up
    solve that also runs the autotuners, against the plain FP64 form solved one
    instance at a time; N_t x iterations summed over the instances / wall time."""
    insts = W.batch(seed=2)
    grids = [eth.problem(w, device=dev) for w in insts]
    opts = dict(tol=TOL, oseen_prec="lsc", restart=150, maxit=4000)
    B = eth.Batch(grids)
    B.solve(**opts)
    torch.cuda.synchronize()
    t = time.perf_counter()
    _, _, sts, rc = B.solve(**opts)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t
    B.close()
    work = sum(G.nt * st["iters_total"] for G, st in zip(grids, sts))
    t = time.perf_counter()
    its64 = 0
    for G in grids:
        _, _, st = G.solve(precision="fp64", graph=0, **opts)
        its64 += st["iters_total"]
    torch.cuda.synchronize()
    wall64 = time.perf_counter() - t
    out = {"workload": "batch64_seed2", "sum_N_t": sum(G.nt for G in grids), "wall_s": wall, "status": rc,
           "converged": sum(1 for st in sts if st["status"] == 0), "iters": sum(st["iters_total"] for st in sts),
           "mdof_iter_s": work / wall / 1e6, "fp64_one_at_a_time_s": wall64,
           "speedup_mixed_batched_vs_fp64": wall64 / wall}
    for G in grids:
        G.close()
    return out


def step_line(torch, eth, W, dev, m=32, cpu=True):
    """The flow over a step (Sec. 3, Test problem 3) on the masked grid with h = 1/m
    (m = 32: 11 m^2 = 11264 active squares, the paper's intermediate grid), nu = 1/50:
    CUDA-event time of five Picard steps from the Stokes solution, each solved by the
    two-stage PCD method to a 1e-6 true residual, after a warm-up run that captures
    the Arnoldi-step graphs; iterations of both stages per step, nonlinear residuals,
    N_t x iterations / time.  With cpu: the oracle's exact-block two-stage method on
    the fifth (Oseen) system at h = 1/16, timed on the host (factorisations included)."""
    w = W.step(m)
    G = eth.MGrid(w["nx"], w["ny"], w["h"], w["x0"], w["y0"], w["active"], outflow=True, device=dev)
    G.set_coefficients(w["nu"])
    ub = torch.as_tensor(w["ubc"], dtype=torch.float64, device=G.device)
    G.picard(ub, 5, tol=TOL)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, _, res, sts = G.picard(ub, 5, tol=TOL)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    its = sum(st["iters_total"] for st in sts)
    out = {"workload": f"step_h1_{m}_nu0.02_picard5", "N_t": G.nt, "active_elements": int(w["active"].sum()),
           "ms": ms, "iters": [[st["iters_stage1"], st["iters_stage2"]] for st in sts],
           "relres": max(st["relres_true"] for st in sts), "status": [st["status"] for st in sts],
           "nonlinear_residuals": res, "last_solve_ms": sts[-1]["seconds"] * 1e3,
           "mdof_iter_s": G.nt * its / (ms / 1e3) / 1e6,
           "gpu_launches": sum(st["kernel_launches"] for st in sts)}
    G.close()
    if cpu:
        from oracle import step as ostep
        mc = 16
        wc = W.step(mc)
        g = ostep.step_grid(mc)
        xs, _ = ostep.picard(g, wc["nu"], wc["ubc"], 4)
        s = ostep.StepSystem(g, wc["nu"], xs[-1][: g.nu])
        b = s.rhs(wc["ubc"])
        t = time.perf_counter()
        _, info = ostep.two_stage(s, b, eta=TOL)
        dt = time.perf_counter() - t
        out["oracle_h1_16"] = {"N_t": g.nt, "s": dt, "iters": [info["its1"], info["its2"]],
                               "mdof_iter_s": g.nt * (info["its1"] + info["its2"]) / dt / 1e6,
                               "sample": "the fifth Picard system at h = 1/16 by the oracle's two-stage method with "
                                         "exact (SuperLU) blocks, factorisations included"}
    return out


def _time_apply(torch, eth, H, fp32, reps=40):
    """CUDA-event time (s) of one eth_apply(K) on H's stream, two input/output pairs
    alternating (their 336 MB at 1024^2 exceed the L2)."""
    xs = [torch.randn(H.nt, dtype=torch.float64, device=H.device) for _ in range(2)]
    ys = [torch.empty_like(xs[0]) for _ in range(2)]
    L = eth.load()
    for k in range(4):
        L.eth_apply(H.h, eth.OPS["K"], fp32, eth._ptr(xs[k % 2]), eth._ptr(ys[k % 2]))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(H.stream):
        e0.record()
        for k in range(reps):
            L.eth_apply(H.h, eth.OPS["K"], fp32, eth._ptr(xs[k % 2]), eth._ptr(ys[k % 2]))
        e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps / 1e3


ROOF_ROWS = (4, 6, 8)   # warp-strip shapes timed; the fastest is the roofline kernel


def roofline(G, torch, eth):
    """Fused K apply (warp-strip kernel k_q2s, FP32 element arithmetic, FP64 in/out) on
    the 1024^2 grid of the same workload family, timed live for each element-row count
    per warp in ROOF_ROWS; the fastest is reported.  Algorithmic bytes = 16 B x N_t per
    launch (FP64 in + out).  The shared-memory tile kernel of the same operator is
    timed beside it, and the Oseen operator (its FP32 wind read as well: + 8 B x N_v) on
    the 512^2 grid of the Oseen workload."""
    from paper_2303_10233_gb300 import workloads as W
    peak, src = _peaks()
    H = eth.problem(W.mms(1024, seed=SEED), device=G.device.index)
    times = {}
    for rows in ROOF_ROWS:
        H.set_tile(rows, 2)
        times[rows] = _time_apply(torch, eth, H, 1)
    H.set_tile(8, 0)
    t_tile = _time_apply(torch, eth, H, 1)
    rows = min(times, key=times.get)
    t = times[rows]
    bytes_ = 16.0 * H.nt
    ach = bytes_ / t / 1e9
    H.close()
    O = eth.problem(W.oseen_cavity(512, nu=0.01, seed=1), device=G.device.index)
    osn = {}
    for r in ROOF_ROWS:
        O.set_tile(r, 2)
        osn[f"strip{r}"] = _time_apply(torch, eth, O, 1)
    O.set_tile(8, 0)
    osn["tile32x8"] = _time_apply(torch, eth, O, 1)
    best = min(osn, key=osn.get)
    ob = 16.0 * O.nt + 8.0 * O.nv
    O.close()
    return {"kernel": f"k_q2s warp-strip fused K apply, {rows} element rows per warp (FP32 element math, "
                      f"FP64 I/O), Stokes n=1024", "bound": "hbm",
            "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_source": f"{src} (burst copy)", "traffic": _profiled_traffic(rows),
            "alg_bytes_per_launch": bytes_, "us_per_launch": t * 1e6,
            "us_by_rows": {str(r): round(v * 1e6, 2) for r, v in times.items()},
            "tile_kernel_us": t_tile * 1e6, "tile_kernel_frac": bytes_ / t_tile / 1e9 / peak,
            "oseen512": {"best": best, "us": osn[best] * 1e6, "alg_bytes_per_launch": ob,
                         "achieved_gbs": ob / osn[best] / 1e9, "frac": ob / osn[best] / 1e9 / peak,
                         "us_by_kernel": {k: round(v * 1e6, 2) for k, v in osn.items()}}}


def profile_apply(n, kind, rows):
    """Five K applies (FP32 element arithmetic) on an n x n grid for ncu captures: the
    warp-strip kernel with `rows` element rows per warp, or the 32 x 8 tile kernel (rows 0)."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_10233_gb300 import eth, workloads as W
    w = W.oseen_cavity(n, nu=0.01, seed=1) if kind == "oseen" else W.mms(n, seed=SEED)
    G = eth.problem(w)
    G.set_tile(rows, 2) if rows else G.set_tile(8, 0)
    x = torch.randn(G.nt, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    for _ in range(5):
        eth.load().eth_apply(G.h, eth.OPS["K"], 1, eth._ptr(x), eth._ptr(y))
    torch.cuda.synchronize()
    print(f"profile_apply n={n} kind={kind} rows={rows} N_t={G.nt} done")
    G.close()


def profile_solve(n, kind):
    """Two default solves of the n x n workload (Stokes MMS or Oseen cavity, nu = 1/100)
    for an ncu launch list of the solver (the second solve is the one to read).  The
    Stokes solves replay their MINRES graph from the host (graph = 2): the same kernels as
    the device-side loop, whose conditional-node body ncu does not list launch by launch."""
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_10233_gb300 import eth, workloads as W
    w = W.oseen_cavity(n, nu=0.01, seed=1) if kind == "oseen" else W.mms(n, seed=SEED)
    G = eth.problem(w)
    for _ in range(2):
        _, _, st = G.solve(tol=TOL, graph=2 if kind == "stokes" else 1)
    print(f"profile_solve n={n} kind={kind} its={st['iters_stage1']}+{st['iters_stage2']} "
          f"ms={st['seconds'] * 1e3:.1f} launches={st['kernel_launches']}")
    G.close()


def profile_step(m):
    """Two Picard steps (Stokes, then Oseen) on the step with h = 1/m, stream launches,
    for an ncu launch list of the masked-grid solver (the Oseen solve's launches follow
    the Stokes solve's)."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_10233_gb300 import eth, workloads as W
    w = W.step(m)
    G = eth.MGrid(w["nx"], w["ny"], w["h"], w["x0"], w["y0"], w["active"], outflow=True)
    G.set_coefficients(w["nu"])
    _, _, res, sts = G.picard(torch.as_tensor(w["ubc"], device="cuda"), 2, tol=TOL, graph=0)
    print(f"profile_step m={m} its={[(s_['iters_stage1'], s_['iters_stage2']) for s_ in sts]} "
          f"launches={[s_['kernel_launches'] for s_ in sts]}")
    G.close()


def est_table(nmax):
    """EST-MINRES inf-sup estimates on the lid-driven cavity for n = 16, 32, .., nmax
    (one JSON line per grid): MINRES iterations and the final gamma^2 estimate with
    the exact blocks of P_1 (FP64, inner CG to 1e-12) and with the default
    multigrid approximations (mixed precision, first refinement pass), the solve
    time and the CUDA-event time of the estimate kernel (all iterations' estimates)."""
    import __graft_entry__ as ge
    ge.build()
    import torch
    from paper_2303_10233_gb300 import eth, workloads as W
    n = 16
    while n <= nmax:
        w = W.cavity(n)
        row = {"n": n}
        for tag, opts in (("p1", dict(precision="fp64", a_exact=1, mq_mode=1, inner_tol=1e-12)),
                          ("mg", dict(precision="mixed"))):
            G = eth.problem(w)
            _, _, st = G.solve(tol=1e-8, **opts)
            d, gm = G.lanczos()
            est = G.est_infsup(d, gm)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(G.stream):
                e0.record()
                for _ in range(20):
                    G.est_infsup(d, gm)
                e1.record()
            e1.synchronize()
            row[tag] = {"its": st["iters_total"], "lanczos_steps": int(d.numel()),
                        "gamma2_est": float(est[-1].item()), "solve_ms": round(st["seconds"] * 1e3, 2),
                        "est_us": round(e0.elapsed_time(e1) / 20 * 1e3, 1)}
            G.close()
        print(json.dumps(row))
        n *= 2


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-instance batch measurement")
    ap.add_argument("--profile-apply", type=int, default=0, metavar="N",
                    help="only run the fused K apply (FP32 math) 5 times on an N x N grid (for ncu captures)")
    ap.add_argument("--profile-kind", default="stokes", choices=["stokes", "oseen"])
    ap.add_argument("--profile-rows", type=int, default=4,
                    help="element rows per warp of the strip kernel in --profile-apply (0: the tile kernel)")
    ap.add_argument("--profile-solve", type=int, default=0, metavar="N",
                    help="only run two default solves on an N x N grid of --profile-kind (for ncu launch lists)")
    ap.add_argument("--profile-step", type=int, default=0, metavar="M",
                    help="two Picard steps of the step problem at h = 1/M for an ncu launch list")
    ap.add_argument("--est", type=int, default=0, metavar="N",
                    help="only print EST-MINRES inf-sup estimates on cavity grids 16 .. N")
    args = ap.parse_args()
    if args.est:
        est_table(args.est)
        return
    if args.profile_apply:
        profile_apply(args.profile_apply, args.profile_kind, args.profile_rows)
        return
    if args.profile_solve:
        profile_solve(args.profile_solve, args.profile_kind)
        return
    if args.profile_step:
        profile_step(args.profile_step)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

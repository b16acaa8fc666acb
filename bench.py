"""Benchmark: HDG trace solves/s to a relative residual of 1e-8 on one GB300.

Workload (flat periodic square, 256 x 256 x 2 = 131,072 triangles): side
5.12e6 m, g = 9.81, H = 1e3 m, f = 1e-4 1/s, acoustic Courant number
c tau / h = 8, DG degree p = 3 (local blocks 30, trace blocks 12), right-hand
sides = seeded zero-mean unit-RMS Gaussian random fields with a k^-3 power
spectrum (synthetic data shaped like the paper's flat-domain workload).

A step = one solve: condensed right-hand side (step 1), (F)GMRES with the
two-level V-cycle to a true relative residual of 1e-8 (step 2), recovery of
(u, h) (step 3).  ``value`` is the mixed-precision solver (FP32 inner solves,
FP64 iterative refinement); the plain FP64 solver on the same GPU is reported
beside it (``plain_fp64``), as is the CPU oracle on a bounded sample
(``cpu_baseline``).  ``--impl reference`` times the CPU oracle alone.

Multi-GPU: replicas only (independent solves per rank, no collective on the
data path); launched by torchrun, rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HDG trace solves/s to rel.res 1e-8: mixed/learned vs plain FP64 MG, same GB300"
SIDE, NGRID, G, DEPTH, F0 = 5.12e6, 256, 9.81, 1.0e3, 1.0e-4
SAMPLE_N = 64            # oracle sample: 64 x 64 x 2 = 8,192 triangles of the same workload
RADIUS, OMEGA = 6.371e6, 7.292e-5
SPHERE_R, SAMPLE_R = 6, 4   # sphere workload: r = 6 (81,920 triangles); oracle sample r = 4 (5,120)
# P1 hierarchies: flat down to the 4 x 4 periodic grid (16 vertices), sphere
# down to r - 5 (at least r = 1, 42 vertices).  Ending them at about a thousand
# vertices (solved exactly by the multi-CTA dense product) leaves the oracle's
# iteration counts unchanged, but measured 1 % slower on the mixed-precision
# flat workload and costs an 18 ms larger inverse at every condensation.
FLAT_COARSEST, SPHERE_COARSEST_DEPTH = 4, 5


def flat_hierarchy(n: int):
    import hdg_inputs as I
    return I.periodic_square_hierarchy(n, side=SIDE * n / NGRID, n_coarsest=FLAT_COARSEST)


def sphere_hierarchy(r: int):
    import hdg_inputs as I
    return I.sphere_hierarchy(r, RADIUS, r_coarsest=max(r - SPHERE_COARSEST_DEPTH, 1))


def workload(n: int, p: int, courant: float, seed: int):
    import hdg_inputs as I
    mesh = flat_hierarchy(n)
    c = math.sqrt(G * DEPTH)
    tau = courant * mesh.h / c
    f = I.coriolis_flat(mesh, F0)
    ru, rh = I.gaussian_field_rhs(mesh, p, seed, grid=max(4 * n, 128), kmax=n / 2)
    return mesh, tau, f, ru, rh


def workload_name(n, p, courant):
    return (f"flat periodic {n}x{n}x2 ({2 * n * n:,} triangles), HDG p={p}, acoustic Courant {courant:g}, "
            f"g={G}, H={DEPTH:g} m, f={F0:g}, k^-3 Gaussian RHS")


def sphere_workload(r: int, p: int, courant: float, seed: int):
    """Icosahedral sphere refined r times (20 * 4^r flat triangles), radius
    6.371e6 m, f = 2 Omega sin(latitude) (P1), g = 9.81, H drawn from
    U[5e3, 1e4] m by the seed, tau = Courant * h_r / c; right-hand sides are
    random spherical-harmonic fields up to degree 64 with l^-3 variance."""
    import numpy as np
    import hdg_inputs as I
    mesh = sphere_hierarchy(r)
    H = float(np.random.default_rng(seed).uniform(5e3, 1e4))
    tau = courant * mesh.h / math.sqrt(G * H)
    f = I.coriolis_sphere(mesh, OMEGA)
    ru, rh = I.spherical_harmonic_rhs(mesh, p, seed, lmax=64)
    return mesh, tau, f, ru, rh, H


def workload_label(kind: str, p: int, courant: float, seed: int) -> str:
    """Name of the full workload (without generating its right-hand sides)."""
    if kind == "sphere":
        import numpy as np
        import hdg_inputs as I
        mesh = sphere_hierarchy(SPHERE_R)
        H = float(np.random.default_rng(seed).uniform(5e3, 1e4))
        tau = courant * mesh.h / math.sqrt(G * H)
        fmax = float(np.abs(I.coriolis_sphere(mesh, OMEGA)).max())
        return (f"icosahedral sphere r={SPHERE_R} ({mesh.n_cells:,} triangles), radius 6.371e6 m, HDG p={p}, "
                f"acoustic Courant {courant:g}, g={G}, H={H:.0f} m, f=2 Omega sin(lat) (max |f| tau = "
                f"{fmax * tau:.2f}), spherical-harmonic RHS to degree 64")
    return workload_name(NGRID, p, courant)


def make_workload(kind: str, full: bool, p: int, courant: float, seed: int) -> dict:
    """The benchmark workload (full = True) or the oracle's bounded sample of it."""
    if kind == "sphere":
        r = SPHERE_R if full else SAMPLE_R
        mesh, tau, f, ru, rh, H = sphere_workload(r, p, courant, seed)
        return dict(mesh=mesh, tau=tau, f=f, ru=ru, rh=rh, g=G, H=H)
    n = NGRID if full else SAMPLE_N
    mesh, tau, f, ru, rh = workload(n, p, courant, seed)
    return dict(mesh=mesh, tau=tau, f=f, ru=ru, rh=rh, g=G, H=DEPTH)


# ---------------------------------------------------------------- algorithmic bytes per launch
def trace_bytes(cat: str, NF: int, pp: int, s_width: int | None = None) -> float:
    """Minimum bytes a facet-row kernel must move: the operator values (5 blocks
    of (p+1)^2 per facet), the neighbour ids, the inverted facet blocks where
    used, and each trace vector it touches read or written once.  s_width
    overrides the bytes per operator value (2 for the BF16 preconditioner copy)."""
    w = 8 if cat.endswith("64") else 4
    S = 5 * pp * pp * (s_width or w) + 16
    vec = pp * w
    base = cat[:-2]
    if base == "apply":
        per = S + 2 * vec
    elif base == "residual":
        per = S + 3 * vec
    elif base == "smooth":
        per = S + pp * pp * w + 3 * vec
    elif base == "smooth_first":
        per = pp * pp * w + 2 * vec
    else:
        raise KeyError(cat)
    return float(NF) * per


# ---------------------------------------------------------------- clocks
CLOCK_QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi sampling every 50 ms.  Started before the warm-up: a cold
    nvidia-smi start costs CPU time that would otherwise fall into the timed
    region; wait_ready() holds until it has run for 1.5 s.  Each sample carries
    nvidia-smi's own timestamp; stop(t0, t1) keeps those inside the timed window."""

    def __init__(self, gpu_index: int, path: str = ""):
        self.proc = None
        self.fh = None
        self.t_start = time.time()
        # the raw samples go to path when given (--clocks-csv), else to a temporary file
        self.tmp = not path
        if self.tmp:
            import tempfile
            fd, path = tempfile.mkstemp(prefix=f"clocks_{os.getpid()}_", suffix=".csv")
            os.close(fd)
        self.path = path
        try:
            if os.path.dirname(self.path):
                os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={CLOCK_QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def wait_ready(self, seconds: float = 1.5) -> None:
        if self.proc is not None:
            time.sleep(max(0.0, self.t_start + seconds - time.time()))

    def stop(self, t0: float = None, t1: float = None) -> dict:
        if self.proc is None:
            if getattr(self, "fh", None) is not None:
                self.fh.close()
            if self.tmp and os.path.exists(self.path):
                os.remove(self.path)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        import datetime
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        with open(self.path) as fh:
            lines = fh.readlines()
        if self.tmp:
            os.remove(self.path)
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        if t0 is not None and t1 is not None:
            inside = [r for r in rows if t0 - 0.06 <= r[0] <= t1 + 0.06]
            rows = inside or rows
        sm, smax, reasons = [], [], set()
        for _, a, b, flags in rows:
            sm.append(a)
            smax.append(b)
            for nm, v in zip(names, flags):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
def host_threads() -> dict:
    """Host cores and the thread settings the oracle process runs with."""
    try:
        avail = len(os.sched_getaffinity(0))
    except AttributeError:
        avail = os.cpu_count()
    return {"nproc": avail, "cpu_count": os.cpu_count(),
            **{k: os.environ.get(k, "unset") for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}}


def oracle_run(p: int, courant: float, warmup: int, steps: int, seed: int = 0, kind: str = "flat",
               full: bool = True, direct: bool = False) -> dict:
    """Time the oracle (plain FP64 FGMRES + V-cycle, as it stands) on the
    benchmark workload (full = True) or its small sample: set-up (cell
    operators, trace operator, preconditioner) once and untimed, then `warmup`
    untimed and `steps` timed solves, each one condensed right-hand side,
    FGMRES(30) to 1e-8 and recovery.  direct = True also times SciPy's sparse
    LU of the trace operator (factor and solve), the analogue of the paper's
    direct-solver comparison."""
    import numpy as np
    from oracle.hdg import HDGProblem
    from oracle.solver import TwoLevelPreconditioner, gmres
    t_all = time.perf_counter()
    wl = make_workload(kind, full, p, courant, seed)
    mesh, tau, f, ru, rh = wl["mesh"], wl["tau"], wl["f"], wl["ru"], wl["rh"]
    t0 = time.perf_counter()
    prob = HDGProblem(mesh, p, tau=tau, g=wl["g"], H=wl["H"], f_vertex=f)
    S = prob.trace_operator()
    pc = TwoLevelPreconditioner(prob, mesh, S, coarse="gmg")
    setup_s = time.perf_counter() - t0
    times, iters, res = [], [], []
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        gvec = prob.condensed_rhs(ru, rh)
        lam, info = gmres(lambda v: S @ v, gvec, pc, restart=30, rtol=1e-8)
        prob.recover(lam, ru, rh)
        if k >= warmup:
            times.append(time.perf_counter() - t0)
            iters.append(info["iters"])
            res.append(float(info["true_rel_res"]))
    out = {"sec_per_solve": float(np.median(times)), "sec_total": float(np.sum(times)), "times": times,
           "iters": iters, "true_rel_res": res, "n_cells": mesh.n_cells, "setup_s": setup_s, **host_threads()}
    if direct:
        import scipy.sparse.linalg as spla
        gvec = prob.condensed_rhs(ru, rh)
        t0 = time.perf_counter()
        lu = spla.splu(S.tocsc())
        t1 = time.perf_counter()
        x = lu.solve(gvec)
        t2 = time.perf_counter()
        out["direct"] = {"factor_s": t1 - t0, "solve_s": t2 - t1, "lu_nnz": int(lu.L.nnz + lu.U.nnz),
                         "true_rel_res": float(np.linalg.norm(gvec - S @ x) / np.linalg.norm(gvec))}
    out["wall_s"] = time.perf_counter() - t_all
    return out


def oracle_command(p: int, courant: float, warmup: int, steps: int, kind: str = "flat", direct: bool = False):
    """The oracle runs in a process of its own, single-threaded (SciPy's sparse
    products are single-threaded anyway; BLAS pinned to one thread)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-run", "--p", str(p), "--courant", str(courant),
           "--warmup", str(warmup), "--steps", str(steps), "--workload", kind] + (["--cpu-direct"] if direct else [])
    return cmd, env


def oracle_start(p, courant, warmup, steps, kind="flat", direct=False):
    """Start the oracle process now (before any CUDA call); collect it with oracle_wait."""
    import tempfile
    cmd, env = oracle_command(p, courant, warmup, steps, kind, direct)
    out = tempfile.TemporaryFile(mode="w+")
    err = tempfile.TemporaryFile(mode="w+")
    return subprocess.Popen(cmd, stdout=out, stderr=err, env=env, text=True), out, err


def oracle_wait(handle, timeout=3600) -> dict:
    proc, out, err = handle
    rc = proc.wait(timeout=timeout)
    out.seek(0)
    err.seek(0)
    if rc != 0:
        raise RuntimeError(f"oracle run failed: {err.read()[-2000:]}")
    return json.loads(out.read().strip().splitlines()[-1])


def oracle_sample_text(r: dict, kind: str, name: str) -> str:
    return (f"the full workload ({name}): {len(r['times'])} timed solve(s) after {r['setup_s']:.0f} s of untimed "
            f"set-up, each one condensed RHS, FGMRES(30) + V-cycle to 1e-8 and recovery (median per solve); "
            f"single-threaded NumPy/SciPy oracle, as it stands")


def cpu_baseline_entry(r: dict, kind: str, name: str) -> dict:
    val = 1.0 / r["sec_per_solve"]
    entry = {"value": val, "unit": "solves/s", "cores": 1, "kind": "oracle",
             "sample": oracle_sample_text(r, kind, name), "sec_per_solve": r["sec_per_solve"],
             "iters": r["iters"], "setup_s": r["setup_s"], "wall_s": r["wall_s"],
             "host": {k: r[k] for k in ("nproc", "cpu_count", "OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                        "MKL_NUM_THREADS")}}
    if "direct" in r:
        entry["direct_splu"] = r["direct"]
    return entry


# ---------------------------------------------------------------- replicas
def max_over_ranks(dist, x: float, device) -> float:
    """Largest x over the ranks of the process group (x itself without one).
    The replicas share nothing on the data path; only their timings meet here."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, steps: int, ms_max: float) -> float:
    """Whole-job solves/s: every rank solves `steps` problems; the slowest rank's time counts."""
    return world * steps / (ms_max * 1e-3)


# ---------------------------------------------------------------- GPU arms
def gpu_arm(args, rank: int, world: int):
    import numpy as np
    import torch
    from paper_2004_09389_gb300 import HDGSolver, HDG_FP64, HDG_MIXED_FP32, HDG_MIXED_BF16, HDG_MIXED_FGMRES64, build
    build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    wl = make_workload(args.workload, True, args.p, args.courant, args.seed + rank)
    mesh, tau, f, ru, rh, g_, H_ = wl["mesh"], wl["tau"], wl["f"], wl["ru"], wl["rh"], wl["g"], wl["H"]
    ru_d = torch.from_numpy(ru).to(dev)
    rh_d = torch.from_numpy(rh).to(dev)
    out = {}
    arms = [(a, p) for a, p in (("mixed", HDG_MIXED_FP32), ("mixed_bf16", HDG_MIXED_BF16),
                                ("fgmres64", HDG_MIXED_FGMRES64), ("fp64", HDG_FP64))
            if a in args.arms.split(",")]
    for arm, prec in arms:
        s = HDGSolver(mesh, args.p, tau, g_, H_, f_vertex=f, rtol=args.rtol, precision=prec,
                      inner_rtol=args.inner_rtol, restart=args.restart, reorth=args.reorth)
        NF, pp = s.n_facets, args.p + 1
        tuned = s.autotune() if args.autotune else None
        # condensation (step 0, once per operator), timed warm and apart from the solves
        torch.cuda.synchronize()
        t_c = time.perf_counter()
        s.condense()
        torch.cuda.synchronize()
        condense_ms = (time.perf_counter() - t_c) * 1e3
        lam_d = torch.empty((NF, pp), dtype=torch.float64, device=dev)
        u_d = torch.empty((s.n_cells, 2, s.n_p), dtype=torch.float64, device=dev)
        h_d = torch.empty((s.n_cells, s.n_p), dtype=torch.float64, device=dev)
        infos = []

        # the recovery of this solve: lambda from the handle (NULL); a two-float handle
        # also takes what its step 1 kept of the right-hand side (NULL r_u, r_h)
        rec_r = (None, None) if prec in (HDG_MIXED_FP32, HDG_MIXED_BF16) else (ru_d, rh_d)

        def step():
            infos.append(s.solve_dev(ru_d, rh_d, lam_d))
            s.recover_dev(rec_r[0], rec_r[1], None, u_d, h_d)

        clocks = ClockSampler(dev.index, args.clocks_csv) if arm == "mixed" else None
        for _ in range(args.warmup):
            step()
        infos.clear()
        s.profile_enable(timing=False)          # launch counters only
        stream = s.stream                        # the handle's stream: every kernel of the solve runs on it
        if clocks:
            clocks.wait_ready()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_wall0 = time.time()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        t_wall1 = time.time()
        barrier()
        ms = e0.elapsed_time(e1)
        clk = clocks.stop(t_wall0, t_wall1) if clocks else None
        launches = sum(n for _, n in s.profile_read().values())
        ms = max_over_ranks(dist, ms, dev)
        # second pass with per-kernel event timing for the roofline (caches as the
        # solve leaves them), third pass with L2 evicted before every timed launch
        # (operands from DRAM: the HBM figure)
        nprof = max(1, min(args.steps, 3))
        s.profile_enable(timing=True)
        for _ in range(nprof):
            step()
        prof = s.profile_read()
        s.profile_enable(timing=True, cold=True)
        for _ in range(nprof):
            step()
        prof_cold = s.profile_read()
        s.profile_enable(timing=False)           # per-kernel events off again for the end-to-end pass
        # end to end through the host-pointer C-ABI calls (pinned host buffers)
        ru_h = torch.from_numpy(ru).pin_memory()
        rh_h = torch.from_numpy(rh).pin_memory()
        lam_h = torch.empty((NF, pp), dtype=torch.float64).pin_memory()
        u_h = torch.empty((s.n_cells, 2, s.n_p), dtype=torch.float64).pin_memory()
        hh_h = torch.empty((s.n_cells, s.n_p), dtype=torch.float64).pin_memory()
        import ctypes as C
        from paper_2004_09389_gb300 import _lib
        info = _lib.hdg_solve_info()

        def host_step():
            # steps 1-3 through the one-call host entry point (hdg_solve_recover)
            _lib.check(s.h, s.lib.hdg_solve_recover(s.h, ru_h.data_ptr(), rh_h.data_ptr(), lam_h.data_ptr(),
                                                    u_h.data_ptr(), hh_h.data_ptr(), C.byref(info)))

        for _ in range(args.warmup):
            host_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_step()
        barrier()
        e2e_s = time.perf_counter() - t0
        e2e_s = max_over_ranks(dist, e2e_s, dev)
        h2d = ru.nbytes + rh.nbytes
        d2h = lam_h.numel() * 8 + u_h.numel() * 8 + hh_h.numel() * 8
        levels = [mesh] + list(mesh.levels)
        nK, m = 3 * s.n_p, 3 * pp
        out[arm] = dict(ms=ms, infos=infos, clocks=clk, launches=launches, prof=prof, prof_cold=prof_cold,
                        e2e_s=e2e_s, levels_nv=[lv.n_vertices for lv in levels],
                        condense_ms=condense_ms, n_p=s.n_p, prof_steps=nprof, tuned=tuned,
                        h2d=h2d, d2h=d2h, NF=NF, pp=pp, n_cells=s.n_cells,
                        keep_z=prec in (HDG_MIXED_FP32, HDG_MIXED_BF16),
                        coarse=(f"P1 geometric V-cycle over {len(levels)} levels, {levels[0].n_vertices:,} -> "
                                f"{levels[-1].n_vertices} vertices (dense coarsest solve)"),
                        data_gb=(8.0 * s.n_cells * (nK * nK + 2 * nK * m) + 8.0 * NF * 5 * pp * pp) / 1e9)
        s.close()
        torch.cuda.empty_cache()
    # the FMA rates, measured after every timed region (seconds of FP64 work)
    from paper_2004_09389_gb300 import _lib as hdglib
    fma = {"fp64_tflops": hdglib.fma_rate(8), "fp32_tflops": hdglib.fma_rate(4),
           "how": "hdg_fma_rate: 8 independent FMA chains per thread, 8 x 256 threads per SM, CUDA events, best of 3"}
    if dist is not None:
        dist.destroy_process_group()
    return out, fma


def step13_bytes(arm: dict):
    """Algorithmic bytes of one condensed right-hand side (cell and gather
    kernels together) and of one recovery.  Two-float handles keep z_K = R_M r_K
    in step 1: its cell kernel reads R_M, r and the cell geometry (9 float pairs)
    and writes z and the cell rows; the recovery reads X_B, z and lambda and
    writes u, h.  FP64 handles read W_K, r in step 1 and R_M, X_B, r, lambda in
    step 3."""
    N, nK, m = arm["n_cells"], 3 * arm["n_p"], 3 * arm["pp"]
    if arm.get("keep_z"):
        return 8.0 * N * (nK * nK + 2 * nK + m) + 72.0 * N, 8.0 * N * (nK * m + 2 * nK + m)
    return 8.0 * N * (m * nK + nK + m), 8.0 * N * (nK * nK + nK * m + 3 * nK + m)


def whole_solve(arm: dict, peaks: dict, steps: int) -> dict:
    """Algorithmic bytes of one solve's facet-row kernels, condensed right-hand
    side and recovery (launch counts from the library's accounting) over the
    whole solve time; the P1 V-cycle and the Krylov vectors are not counted, so
    the fraction is a lower bound."""
    prof, NF, pp, N = arm["prof"], arm["NF"], arm["pp"], arm["n_cells"]
    nK, m = 3 * arm["n_p"], 3 * pp
    ps = arm["prof_steps"]
    total = 0.0
    for cat, (_, n) in prof.items():
        if n and cat.startswith(("apply", "residual", "smooth")):
            total += trace_bytes(cat, NF, pp) * n / ps
    # step 1 (two launches per call) and step 3
    rhs_b, rec_b = step13_bytes(arm)
    total += rhs_b * (prof["rhs"][1] / 2) / ps
    total += rec_b * prof["recover"][1] / ps
    ms = arm["ms"] / steps
    achieved = total / (ms * 1e-3) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    return {"bytes_per_solve": total, "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "counted": "facet-row kernels, condensed RHS, recovery (P1 V-cycle and Krylov vectors not counted)"}


def fp64_fmas_per_facet(cat: str, pp: int) -> int:
    """FMAs per facet of an FP64 facet-row kernel (operator blocks, inverse block)."""
    base = cat[:-2]
    return {"apply": 5 * pp * pp, "residual": 5 * pp * pp, "smooth": 6 * pp * pp, "smooth_first": pp * pp}[base]


def p1_cycle_bytes(levels_nv: list, w: int, width: int = 8) -> float:
    """Algorithmic bytes of one P1 V-cycle (2 + 2 Jacobi sweeps per level): each
    sweep reads the padded ELL values and columns, the inverse diagonal, b and x
    and writes x; the residual reads the operator, b and x and writes r; the
    transfers read and write each level's vector once; the coarsest level reads
    its dense FP64 inverse."""
    total = 0.0
    for nv in levels_nv[:-1]:
        sweep = nv * (width * (4 + w) + 4 * w)
        total += 4 * sweep + nv * (width * (4 + w) + 3 * w) + 4 * nv * w
    nc = levels_nv[-1]
    return total + 8.0 * nc * nc + 16.0 * nc


def _kernel_entry(name, prof, cold, cat, bytes_per_launch, peak, total_w, note=None):
    ms_w, n_w = prof[cat]
    ms_c, n_c = cold[cat]
    if not n_w:
        return None
    e = {"kernel": name, "share_of_kernel_time": ms_w / total_w if total_w else None,
         "launches": n_w, "avg_us_warm": ms_w * 1e3 / n_w, "avg_us_cold": ms_c * 1e3 / max(n_c, 1)}
    if bytes_per_launch:
        e.update({"algorithmic_bytes_per_launch": bytes_per_launch,
                  "achieved_cold": bytes_per_launch * n_c / (ms_c * 1e-3) / 1e9 if ms_c > 0 else None,
                  "achieved_warm": bytes_per_launch * n_w / (ms_w * 1e-3) / 1e9 if ms_w > 0 else None})
        e["frac_cold"] = e["achieved_cold"] / peak if e["achieved_cold"] else None
    if note:
        e["note"] = note
    return e


def roofline(arm: dict, peaks: dict, fma: dict | None = None, bf16_pre: bool = False) -> dict:
    """Roofline of the facet-row kernel with the largest share of the solve's
    kernel time: algorithmic bytes per launch x launches over its CUDA-event
    time with L2 evicted before every launch (cold: operands from DRAM), against
    the measured HBM copy bandwidth; the same in the running solve (warm) as a
    second figure.  FP64 facet-row kernels also get their FP64-pipe fraction
    against the measured FMA rate.  `others` lists the remaining kernel
    families with their shares."""
    prof, cold, NF, pp = arm["prof"], arm["prof_cold"], arm["NF"], arm["pp"]
    cats = [c for c in prof if c.startswith(("apply", "residual", "smooth")) and prof[c][1]]
    total = sum(ms for ms, _ in prof.values())
    best = max(cats, key=lambda c: prof[c][0])
    bf16_op = bf16_pre and best.startswith("smooth") and best.endswith("32") and not best.startswith("smooth_first")
    per_launch = trace_bytes(best, NF, pp, 2 if bf16_op else None)
    ms_c, n_c = cold[best]
    ms_w, n_w = prof[best]
    achieved = per_launch * n_c / (ms_c * 1e-3) / 1e9 if ms_c > 0 else 0.0
    warm = per_launch * n_w / (ms_w * 1e-3) / 1e9 if ms_w > 0 else 0.0
    peak = peaks.get("hbm_gbs", 6800.0)
    traffic = stored_traffic(best, pp - 1, "bf16" if bf16_op else ("fp64" if best.endswith("64") else "fp32"))
    family_ms = sum(prof[c][0] for c in cats)
    out = {"bound": "hbm", "kernel": best, "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "traffic": traffic, "algorithmic_bytes_per_launch": per_launch,
           "launches": n_c, "avg_us": ms_c * 1e3 / max(n_c, 1),
           "timing": "CUDA events on the handle's stream; L2 evicted (3 x L2 read) before every launch",
           "warm": {"achieved": warm, "frac": warm / peak, "avg_us": ms_w * 1e3 / max(n_w, 1),
                    "timing": "CUDA events in the running solve (part of the operator L2-resident)"},
           "share_of_kernel_time": ms_w / total if total else None,
           "facet_row_family_share": family_ms / total if total else None,
           "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"}
    if best.endswith("64") and fma:
        fl = 2.0 * fp64_fmas_per_facet(best, pp) * NF * n_c / (ms_c * 1e-3) / 1e12
        out["fp64_pipe"] = {"achieved_tflops": fl, "peak_tflops": fma["fp64_tflops"],
                            "frac": fl / fma["fp64_tflops"], "peak_source": "hdg_fma_rate (of measured)"}
    # the other kernel families of the solve
    N, nK, m = arm["n_cells"], 3 * arm["n_p"], 3 * pp
    w32 = 4 if (prof["smooth32"][1] or prof["smooth_first32"][1]) else 8
    ncyc = max(prof["smooth_first32"][1] + prof["smooth_first64"][1], 1)
    others = [
        _kernel_entry("P1 V-cycle (all P1 kernels)", prof, cold, "p1",
                      p1_cycle_bytes(arm["levels_nv"], w32) * ncyc / max(prof["p1"][1], 1), peak, total,
                      "levels up to 32,768 vertices are L2-resident in the running solve: latency-bound"),
        _kernel_entry("recover", prof, cold, "recover", step13_bytes(arm)[1], peak, total),
        _kernel_entry("condensed RHS (cell + gather kernels)", prof, cold, "rhs", step13_bytes(arm)[0] / 2, peak,
                      total),
        _kernel_entry("Krylov (Gram-Schmidt update with norm and Givens, dots, scalings)", prof, cold, "krylov",
                      None, peak, total, "reductions of (j+1) values per iteration: latency of the grid-wide sum"),
        _kernel_entry("restriction / prolongation", prof, cold, "transfer", None, peak, total),
    ]
    out["others"] = [e for e in others if e]
    return out


def condense_rate(arm: dict, fma: dict) -> dict:
    """FP64 flop rate of the condensation against the measured FP64 FMA rate.
    Per cell: Gauss-Jordan elimination of [A_K | B_K | Mass_K] (n_K x (2 n_K + m),
    sum over pivots k of n_K (2 n_K + m - k - 1) FMAs), then S_K = Mt_K + C_K X_B
    (m^2 n_K) and W_K = C_K R_M (m n_K^2)."""
    nK, m, N = 3 * arm["n_p"], 3 * arm["pp"], arm["n_cells"]
    lda = 2 * nK + m
    fmas = sum(nK * (lda - k - 1) for k in range(nK)) + m * m * nK + m * nK * nK
    tf = 2.0 * fmas * N / (arm["condense_ms"] * 1e-3) / 1e12
    return {"flops_per_cell": 2 * fmas, "achieved_tflops": tf, "peak_tflops": fma["fp64_tflops"],
            "frac": tf / fma["fp64_tflops"], "timing": "host wall clock around hdg_condense (one call, synchronised)",
            "note": "includes the facet-row assembly, the P1 operators and the dense coarsest inverse"}


def stored_traffic(cat: str, p: int, op: str):
    """DRAM bytes per launch from an ncu capture (profiles/traffic.json), keyed by
    kernel category, degree and operator type; None unless it was taken on the
    current source of the facet-row kernels."""
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(tpath):
        return None
    ent = json.load(open(tpath)).get(f"{cat}_{op}_p{p}")
    if ent and ent.get("source_sha") == source_sha():
        return ent["bytes_per_launch"]
    return None


def source_sha() -> str:
    """Hash of the facet-row kernels' source (the smoother's code and its launch
    bounds live in k_trace.cu); stored DRAM traffic is used only while it matches."""
    import hashlib
    hsh = hashlib.sha256()
    for name in ("k_trace.cu",):
        hsh.update(open(os.path.join(ROOT, "paper_2004_09389_gb300", "csrc", name), "rb").read())
    return hsh.hexdigest()[:16]


def batch_workload(n_problems: int, seed: int):
    """Uneven independent problems: flat n in {32, 64, 128, 256}, sphere r in
    {3, 4, 5, 6}, p in {1, 2, 3}, tau = tau0 * 2^U[0, 2] (acoustic Courant
    4..16).  On the coarse spheres at large Courant numbers max |f| tau
    reaches about 10: there the damped block-Jacobi sweep amplifies the
    rotation-dominated modes, so those problems (max |f| tau > 1.5) use the
    Chebyshev smoother (smoother = 1).  Flat right-hand sides are k^-3 Gaussian
    fields; sphere ones random spherical-harmonic fields up to degree 64 with
    l^-3 variance.  Meshes and fields are cached per (mesh, p)."""
    import numpy as np
    import hdg_inputs as I
    rng = np.random.default_rng(seed)
    meshes, fields, out = {}, {}, []
    radius, omega = 6.371e6, 7.292e-5
    for k in range(n_problems):
        kind = ("flat", "sphere")[k % 2]
        size = int(rng.choice([32, 64, 128, 256])) if kind == "flat" else int(rng.integers(3, 7))
        p = int(rng.integers(1, 4))
        key = (kind, size)
        if key not in meshes:
            if kind == "flat":
                meshes[key] = flat_hierarchy(size)
            else:
                meshes[key] = sphere_hierarchy(size)
        mesh = meshes[key]
        if (key, p) not in fields:
            if kind == "flat":
                fields[(key, p)] = I.gaussian_field_rhs(mesh, p, seed + k, grid=max(4 * size, 128), kmax=size / 2)
            else:
                fields[(key, p)] = I.spherical_harmonic_rhs(mesh, p, seed + k, lmax=64)
        ru, rh = fields[(key, p)]
        if kind == "flat":
            g, H = G, DEPTH
            f = I.coriolis_flat(mesh, F0)
        else:
            g, H = 9.81, float(rng.uniform(5e3, 1e4))
            f = I.coriolis_sphere(mesh, omega)
        c = math.sqrt(g * H)
        courant = 4.0 * 2.0 ** rng.uniform(0, 2)
        tau = courant * mesh.h / c
        fmax = float(np.max(np.abs(f)))
        out.append(dict(mesh=mesh, p=p, tau=tau, g=g, H=H, f=f, ru=ru, rh=rh, kind=kind, size=size,
                        ftau=fmax * tau, smoother=1 if fmax * tau > 1.5 else 0))
    return out


def sequence_main(args):
    """Learned sweep over a sequence of solves: icosahedral sphere r = 7 (327,680
    triangles), p = 2, Courant 8, f = 2 Omega sin(lat), H drawn by the seed; a
    50-step sequence r^(s+1) = 0.98 r^(s) + 0.2 xi^(s) (normalised), each xi a
    seeded random combination of a pool of 12 spherical-harmonic fields up to
    degree 32 (generated once).  The network (hidden 64, inference on the tensor
    cores) is trained on the r = 5 sphere (same p, physics and Courant number) on
    residuals that plain solves of spherical-harmonic right-hand sides produce,
    and its parameters are copied to the r = 7 handle; the sequence is timed
    with the learned sweep off and on (mixed precision both times), every step
    one solve + recovery."""
    import numpy as np
    import torch
    import hdg_inputs as I
    from paper_2004_09389_gb300 import HDGSolver, HDG_MIXED_FP32, build
    build.build()
    dev = torch.device("cuda", 0)
    r, p, steps = 7, 2, 50
    mesh = sphere_hierarchy(r)
    H = float(np.random.default_rng(args.seed).uniform(5e3, 1e4))
    tau = args.courant * mesh.h / math.sqrt(G * H)
    f = I.coriolis_sphere(mesh, OMEGA)
    t0 = time.perf_counter()
    pool = [I.spherical_harmonic_rhs(mesh, p, args.seed + 100 + k, lmax=32) for k in range(12)]
    t_gen = time.perf_counter() - t0
    PU = np.stack([a for a, _ in pool])
    PH = np.stack([b for _, b in pool])
    rng = np.random.default_rng(args.seed + 7)

    def combo():
        c = rng.standard_normal(len(pool))
        u, h = np.tensordot(c, PU, 1), np.tensordot(c, PH, 1)
        nrm = math.sqrt((np.sum(u * u) + np.sum(h * h)) / (u.size + h.size))
        return u / nrm, h / nrm

    # training on the r = 5 sphere (same p, physics and Courant number): the
    # network sees RMS-normalised facet patches, so its parameters carry over
    rt = 5
    mesh_t = sphere_hierarchy(rt)
    tau_t = args.courant * mesh_t.h / math.sqrt(G * H)
    st = HDGSolver(mesh_t, p, tau_t, G, H, f_vertex=I.coriolis_sphere(mesh_t, OMEGA), precision=HDG_MIXED_FP32,
                   rtol=args.rtol)
    npar = st.learned_init(hidden=64, capacity=256, seed=args.seed)
    n_stored = 0
    for k in range(8):
        u_t, h_t = I.spherical_harmonic_rhs(mesh_t, p, args.seed + 500 + k, lmax=32)
        n_stored = st.learned_collect_dev(torch.from_numpy(u_t).to(dev), torch.from_numpy(h_t).to(dev))
    t0 = time.perf_counter()
    l0, l1 = st.learned_train(steps=400, batch=8, lr=2e-3)
    t_train = time.perf_counter() - t0
    theta = st.learned_params()
    st.close()
    s = HDGSolver(mesh, p, tau, G, H, f_vertex=f, precision=HDG_MIXED_FP32, rtol=args.rtol)
    s.learned_init(hidden=64, capacity=1, seed=args.seed)
    s.set_learned_params(theta)
    # the sequence, resident on the device
    u, h = combo()
    seq = []
    for k in range(steps):
        seq.append((torch.from_numpy(u).to(dev), torch.from_numpy(h).to(dev)))
        xu, xh = combo()
        u, h = 0.98 * u + 0.2 * xu, 0.98 * h + 0.2 * xh
        nrm = math.sqrt((np.sum(u * u) + np.sum(h * h)) / (u.size + h.size))
        u, h = u / nrm, h / nrm
    lam = torch.empty((s.n_facets, p + 1), dtype=torch.float64, device=dev)
    uo = torch.empty((s.n_cells, 2, s.n_p), dtype=torch.float64, device=dev)
    ho = torch.empty((s.n_cells, s.n_p), dtype=torch.float64, device=dev)

    def run(on):
        s.learned_enable(on, tensor_cores=True)
        for k in range(3):                                   # warm-up (graph capture)
            s.solve_dev(*seq[k], lam)
        torch.cuda.synchronize()
        infos = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        for ru_d, rh_d in seq:
            infos.append(s.solve_dev(ru_d, rh_d, lam))
            s.recover_dev(ru_d, rh_d, lam, uo, ho)
        e1.record(s.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        return {"value": steps / (ms * 1e-3), "unit": "solves/s", "ms_per_step": ms / steps,
                "iters": [i["iters"] for i in infos], "fallbacks": int(sum(i["fallback_used"] for i in infos)),
                "max_true_rel_res": max(i["true_rel_res"] for i in infos)}

    plain = run(False)
    learned = run(True)
    line = {"metric": METRIC + " (learned sequence)", "value": learned["value"], "unit": "solves/s",
            "n_gpus": 1, "steps": steps, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": (f"icosahedral sphere r={r} ({mesh.n_cells:,} triangles), HDG p={p}, Courant "
                                    f"{args.courant:g}, H={H:.0f} m, 50-step sequence r <- 0.98 r + 0.2 xi over a "
                                    f"pool of 12 spherical-harmonic fields to degree 32"),
                       "network": f"facet patch, hidden 64, {npar} parameters, tcgen05 inference (BF16 x BF16 -> FP32)",
                       "training": {"mesh": f"icosahedral sphere r={rt}", "residuals": n_stored, "plain_solves": 8,
                                    "steps": 400, "batch": 8,
                                    "loss_first": l0, "loss_last": l1, "seconds": t_train},
                       "field_generation_s": t_gen},
            "learned": learned, "plain_mixed": plain,
            "learned_vs_plain": learned["value"] / plain["value"]}
    s.close()
    print(json.dumps(line))


def imex_main(args):
    """IMEX time loop on the device (Sec. 3.3, ARS2(2,3,2) of Sec. 5.1 by default;
    Coriolis explicit, gravity waves implicit): icosahedral sphere r = 6 (81,920
    triangles), p = 3, radius 6.371e6 m, f = 2 Omega sin(latitude), H drawn from
    U[5e3, 1e4] m by the seed, dt = Courant * h_r / c with acoustic Courant 8;
    initial state = random spherical-harmonic fields to degree 64 (the solve's
    right-hand-side generator).  One condensation for the scheme's a_ii dt
    (outside the loop), then `warmup` untimed and `steps` timed steps, each
    all stage solves, recoveries and explicit stage terms; mixed precision and
    FP64 solves."""
    import numpy as np
    import torch
    import hdg_inputs as I
    from paper_2004_09389_gb300 import HDGSolver, HDG_FP64, HDG_MIXED_FP32, build
    build.build()
    dev = torch.device("cuda", 0)
    r, p = SPHERE_R, args.p
    mesh = sphere_hierarchy(r)
    H = float(np.random.default_rng(args.seed).uniform(5e3, 1e4))
    dt = args.courant * mesh.h / math.sqrt(G * H)
    f = I.coriolis_sphere(mesh, OMEGA)
    u0, h0 = I.spherical_harmonic_rhs(mesh, p, args.seed, lmax=64)
    out = {}
    for arm, prec in (("mixed", HDG_MIXED_FP32), ("fp64", HDG_FP64)):
        s = HDGSolver(mesh, p, dt, G, H, f_vertex=None, rtol=args.rtol, precision=prec, condense=False)
        s.imex_init(f)
        ud = torch.from_numpy(u0).to(dev)
        hd = torch.from_numpy(h0).to(dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.imex_step_dev(args.imex_scheme, dt, ud, hd)          # the first step condenses for a_ii dt
        torch.cuda.synchronize()
        first_ms = (time.perf_counter() - t0) * 1e3
        for _ in range(max(args.warmup - 1, 0)):
            s.imex_step_dev(args.imex_scheme, dt, ud, hd)
        infos = []
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        for _ in range(args.steps):
            infos.append(s.imex_step_dev(args.imex_scheme, dt, ud, hd))
        e1.record(s.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        hsum = float(hd.sum().item())
        out[arm] = {"value": args.steps / (ms * 1e-3), "unit": "steps/s", "ms_per_step": ms / args.steps,
                    "iters_per_step": [i["iters"] for i in infos],
                    "max_true_rel_res": max(i["true_rel_res"] for i in infos),
                    "first_step_ms_with_condensation": first_ms, "sum_h": hsum}
        s.close()
    line = {"metric": "IMEX steps/s (ARS2-type step: stage solves to rel.res 1e-8, recoveries, explicit Coriolis)",
            "value": out["mixed"]["value"], "unit": "steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": (f"icosahedral sphere r={r} ({mesh.n_cells:,} triangles), HDG p={p}, scheme "
                                    f"{args.imex_scheme}, acoustic Courant {args.courant:g} per step (dt = "
                                    f"{dt:.0f} s), H={H:.0f} m, f=2 Omega sin(lat) (max |f| dt = "
                                    f"{float(np.abs(f).max()) * dt:.2f}), spherical-harmonic initial state")},
            "mixed": out["mixed"], "plain_fp64": out["fp64"],
            "speedup_vs_plain_fp64": out["mixed"]["value"] / out["fp64"]["value"]}
    print(json.dumps(line))


def lf_main(args):
    """Lax-Friedrichs solver (vector trace, RT0 coarse space; flat meshes, FP64):
    the benchmark's flat 256 x 256 x 2 workload (side 5.12e6 m, g = 9.81,
    H = 1e3 m, f = 1e-4, k^-3 Gaussian RHS) at p = 1 and 2 with a shorter time
    step (acoustic Courant 2: the Lax-Friedrichs two-level method needs many
    more iterations than the upwind one at Courant 8); solves/s to rel.res 1e-8
    (condensed RHS + FGMRES + recovery), the upwind FP64 solver on the same
    workload beside it."""
    import torch
    from paper_2004_09389_gb300 import HDGSolver, HDG_FP64, build
    build.build()
    out = {}
    for p in (1, 2):
        wl = make_workload("flat", True, p, args.courant, args.seed)
        ru_d, rh_d = torch.from_numpy(wl["ru"]).cuda(), torch.from_numpy(wl["rh"]).cuda()
        row = {}
        for name, flux in (("lax_friedrichs", 1), ("upwind", 0)):
            s = HDGSolver(wl["mesh"], p, wl["tau"], wl["g"], wl["H"], f_vertex=wl["f"], rtol=args.rtol,
                          precision=HDG_FP64, flux=flux, max_iter=3000, restart=args.restart)
            tb = s.n_trace // s.n_facets
            lam = torch.empty((s.n_facets, tb), dtype=torch.float64, device="cuda")
            u = torch.empty((s.n_cells, 2, s.n_p), dtype=torch.float64, device="cuda")
            h = torch.empty((s.n_cells, s.n_p), dtype=torch.float64, device="cuda")
            for _ in range(args.warmup):
                s.solve_dev(ru_d, rh_d, lam)
                s.recover_dev(ru_d, rh_d, lam, u, h)
            torch.cuda.synchronize()
            infos = []
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s.stream)
            for _ in range(args.steps):
                infos.append(s.solve_dev(ru_d, rh_d, lam))
                s.recover_dev(ru_d, rh_d, lam, u, h)
            e1.record(s.stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            row[name] = {"value": args.steps / (ms * 1e-3), "unit": "solves/s", "ms_per_step": ms / args.steps,
                         "iters": infos[-1]["iters"], "true_rel_res": infos[-1]["true_rel_res"],
                         "trace_dofs": s.n_trace}
            s.close()
        out[f"p{p}"] = row
    line = {"metric": "HDG trace solves/s to rel.res 1e-8, Lax-Friedrichs vector trace with RT0 coarse space (FP64)",
            "value": out["p1"]["lax_friedrichs"]["value"], "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": workload_name(NGRID, 1, args.courant) + "; also p=2",
                       "precond": "2+2 block-Jacobi on 2(p+1) facet blocks, RT0 grad-div coarse problem by 20 "
                                  "Chebyshev steps"},
            **out}
    print(json.dumps(line))


def batch_main(args):
    """The uneven batch two ways: merged (one host thread; the launches of all
    problems merged into multi-problem kernels, one CUDA graph per wave; the
    headline value) and threaded (hdg_solve_batch_dev: one stream per problem,
    per-problem step graphs, a pool of host threads); then the same solves one
    after another for the per-solve latency."""
    import numpy as np
    import torch
    from paper_2004_09389_gb300 import HDGSolver, HDG_MIXED_FP32, MergedBatch, build, solve_batch_dev
    build.build()
    probs = batch_workload(args.batch, args.seed)
    # (solves only, no recovery: step 1 keeps nothing for one, keep_rhs = 0)
    solvers = [HDGSolver(x["mesh"], x["p"], x["tau"], x["g"], x["H"], f_vertex=x["f"], rtol=args.rtol,
                         precision=HDG_MIXED_FP32, restart=args.restart, smoother=x["smoother"], max_iter=2000,
                         keep_rhs=0)
               for x in probs]
    tuned = [s.autotune() for s in solvers] if args.autotune else None
    ru = [torch.from_numpy(x["ru"]).cuda() for x in probs]
    rh = [torch.from_numpy(x["rh"]).cuda() for x in probs]
    lam = [torch.zeros((s.n_facets, s.p + 1), dtype=torch.float64, device="cuda") for s in solvers]
    n = len(solvers)

    def timed(run):
        torch.cuda.synchronize()
        for _ in range(args.warmup):
            run()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            out = run()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / args.steps, out

    batch = MergedBatch(solvers)
    t_merged, infos = timed(lambda: batch.solve_dev(ru, rh, lam))
    st = batch.stats()
    batch.close()
    t_threaded, infos_t = timed(lambda: solve_batch_dev(solvers, ru, rh, lam))
    # the same solves one after another, for the per-solve latency
    lat = []
    for s, a, b, l in zip(solvers, ru, rh, lam):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s.solve_dev(a, b, l)
        torch.cuda.synchronize()
        lat.append(time.perf_counter() - t1)
    line = {"metric": "batched HDG trace solves/s to rel.res 1e-8 (uneven problems, mixed precision)",
            "value": n / t_merged, "unit": "solves/s", "n_problems": n, "steps": args.steps, "warmup": args.warmup,
            "ms_per_batch": t_merged * 1e3, "host_threads": 1,
            "merged": {"waves_per_batch": st["waves"] / (args.steps + args.warmup),
                       "launches_per_wave": st["launches"] / max(st["waves"], 1),
                       "problem_launches_per_wave": st["records"] / max(st["waves"], 1),
                       "graph_replays": st["replays"], "graph_builds": st["builds"],
                       "groups": os.environ.get("HDG_BATCH_GROUPS", "4"),
                       "host_ms_per_batch": {k[8:]: st[k] / 1e6 / (args.steps + args.warmup)
                                             for k in ("host_ns_fibers", "host_ns_launch", "host_ns_wait")}},
            "threaded_solves_per_s": n / t_threaded, "threaded_ms_per_batch": t_threaded * 1e3,
            "sequential_solves_per_s": n / sum(lat),
            "latency_ms": {"median": float(np.median(lat)) * 1e3, "max": float(np.max(lat)) * 1e3},
            "iters": [i["iters"] for i in infos], "max_true_rel_res": max(i["true_rel_res"] for i in infos),
            "same_iters_threaded": [i["iters"] for i in infos] == [i["iters"] for i in infos_t],
            "cells": [s.n_cells for s in solvers], "p": [s.p for s in solvers],
            "autotune": tuned, "data": "synthetic",
            "max_ftau": max(x["ftau"] for x in probs), "chebyshev_problems": sum(x["smoother"] for x in probs),
            "config": {"workload": "64 problems: flat n in {32,64,128,256}, sphere r in {3..6} (spherical-harmonic "
                                   "RHS to degree 64), p in {1,2,3}, acoustic Courant 4..16; Chebyshev smoother where "
                                   "max|f| tau > 1.5; FP32 inner + FP64 refinement"}}
    print(json.dumps(line))
    for s in solvers:
        s.close()


def profile_condense_main(args):
    """Set-up and condensation of one mixed-precision handle of the flat
    n x n x 2 workload (p = 3) between cudaProfilerStart/Stop, for ncu."""
    import torch
    from paper_2004_09389_gb300 import HDGSolver, HDG_MIXED_FP32, build
    build.build()
    n = args.profile_condense
    mesh, tau, f, ru, rh = workload(n, args.p, args.courant, args.seed)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    s = HDGSolver(mesh, args.p, tau, G, DEPTH, f_vertex=f, rtol=args.rtol, precision=HDG_MIXED_FP32)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"profile_condense": f"flat {n}x{n}x2 p={args.p}", "cells": s.n_cells}))
    s.close()


def profile_batch_main(args):
    """One merged batched solve of the uneven batch (after two warm-up solves)
    between cudaProfilerStart/Stop, for an ncu launch list."""
    import torch
    from paper_2004_09389_gb300 import HDGSolver, HDG_MIXED_FP32, MergedBatch, build
    build.build()
    probs = batch_workload(args.batch or 64, args.seed)
    # (solves only, no recovery: step 1 keeps nothing for one, keep_rhs = 0)
    solvers = [HDGSolver(x["mesh"], x["p"], x["tau"], x["g"], x["H"], f_vertex=x["f"], rtol=args.rtol,
                         precision=HDG_MIXED_FP32, restart=args.restart, smoother=x["smoother"], max_iter=2000,
                         keep_rhs=0)
               for x in probs]
    ru = [torch.from_numpy(x["ru"]).cuda() for x in probs]
    rh = [torch.from_numpy(x["rh"]).cuda() for x in probs]
    lam = [torch.zeros((s.n_facets, s.p + 1), dtype=torch.float64, device="cuda") for s in solvers]
    b = MergedBatch(solvers)
    for _ in range(2):
        b.solve_dev(ru, rh, lam)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    infos = b.solve_dev(ru, rh, lam)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    st = b.stats()
    print(json.dumps({"profile_batch": len(solvers), "iters": sum(i["iters"] for i in infos), **st}))
    b.close()
    for s in solvers:
        s.close()


def profile_solve_main(args):
    """One warm solve + recovery inside cudaProfilerStart/Stop: the launch list of a
    solve as it runs in the timed loop (caches warm from the previous solves)."""
    import torch
    from paper_2004_09389_gb300 import HDGSolver, HDG_FP64, HDG_MIXED_FP32, HDG_MIXED_BF16, HDG_MIXED_FGMRES64, build
    build.build()
    prec = {"mixed": HDG_MIXED_FP32, "mixed_bf16": HDG_MIXED_BF16, "fgmres64": HDG_MIXED_FGMRES64,
            "fp64": HDG_FP64}[args.profile_solve]
    wl = make_workload(args.workload, True, args.p, args.courant, args.seed)
    s = HDGSolver(wl["mesh"], args.p, wl["tau"], wl["g"], wl["H"], f_vertex=wl["f"], rtol=args.rtol, precision=prec,
                  inner_rtol=args.inner_rtol, restart=args.restart, reorth=args.reorth)
    ru_d, rh_d = torch.from_numpy(wl["ru"]).cuda(), torch.from_numpy(wl["rh"]).cuda()
    # the recovery as the timed step runs it (two-float handles: NULL right-hand sides)
    rec_r = (None, None) if prec in (HDG_MIXED_FP32, HDG_MIXED_BF16) else (ru_d, rh_d)
    lam = torch.empty((s.n_facets, args.p + 1), dtype=torch.float64, device="cuda")
    u = torch.empty((s.n_cells, 2, s.n_p), dtype=torch.float64, device="cuda")
    h = torch.empty((s.n_cells, s.n_p), dtype=torch.float64, device="cuda")
    for _ in range(max(args.warmup, 1)):
        s.solve_dev(ru_d, rh_d, lam)
        s.recover_dev(*rec_r, None, u, h)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    info = s.solve_dev(ru_d, rh_d, lam)
    s.recover_dev(*rec_r, None, u, h)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"profile_solve": args.profile_solve, "workload": workload_label(args.workload, args.p,
                                                                                       args.courant, args.seed),
                      "iters": info["iters"], "true_rel_res": info["true_rel_res"]}))
    s.close()


def profile_learned_main(args):
    """The learned facet-patch sweep inside one FP32 preconditioner application on
    the benchmark workload: off, FP32 network on the CUDA cores, network on the
    tensor cores (hidden 64, parameters 0.3 N(0, 1) from seed 1), 50 applications
    each timed by CUDA events on the handle's stream; then one application with
    each network between profiler start and stop (for ncu --profile-from-start off)."""
    import numpy as np
    import torch
    from paper_2004_09389_gb300 import HDGSolver, HDG_MIXED_FP32, build
    build.build()
    wl = make_workload("flat", True, args.p, args.courant, args.seed)
    s = HDGSolver(wl["mesh"], args.p, wl["tau"], wl["g"], wl["H"], f_vertex=wl["f"], precision=HDG_MIXED_FP32)
    npar = s.learned_init(hidden=64, capacity=4)
    s.set_learned_params((0.3 * np.random.default_rng(1).standard_normal(npar)).astype(np.float32))
    v = torch.randn(s.n_facets * (args.p + 1), device="cuda")
    z = torch.empty_like(v)
    out = {}
    for name, tc in (("off", None), ("fp32", False), ("tensor_cores", True)):
        if tc is None:
            s.learned_enable(False)
        else:
            s.learned_enable(True, tensor_cores=tc)
        for _ in range(3):
            s.precond_apply32_dev(v, z)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        for _ in range(50):
            s.precond_apply32_dev(v, z)
        e1.record(s.stream)
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) / 50 * 1e3
    torch.cuda.profiler.start()
    for tc in (False, True):
        s.learned_enable(True, tensor_cores=tc)
        s.precond_apply32_dev(v, z)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    s.close()
    print(json.dumps({"profile_learned": "precond application us", **{k: round(t, 1) for k, t in out.items()}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--p", type=int, default=3)
    ap.add_argument("--imex-scheme", dest="imex_scheme", default="ARS2", choices=["theta", "ARS2", "SSP2", "ARS3"])
    ap.add_argument("--workload", default="flat", choices=["flat", "sphere", "sequence", "imex", "lf"],
                    help="flat: periodic 256x256x2 square (the headline); sphere: icosahedral sphere r=6; "
                         "sequence: learned sweep over a 50-step sequence on the r=7 sphere")
    ap.add_argument("--courant", type=float, default=8.0)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--inner-rtol", dest="inner_rtol", type=float, default=1e-4)
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--reorth", type=int, default=0, choices=[0, 1],
                    help="Arnoldi orthogonalisation: 0 one classical Gram-Schmidt pass, 1 two passes")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--oracle-steps", type=int, default=2,
                    help="timed oracle solves for cpu_baseline (full workload, after one untimed set-up)")
    ap.add_argument("--cpu-direct", dest="cpu_direct", action="store_true",
                    help="also time SciPy's sparse LU of the trace operator in the oracle process")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--arms", default="mixed,mixed_bf16,fgmres64,fp64",
                    help="solver arms to run (profiling runs may pick one)")
    ap.add_argument("--oracle-run", dest="oracle_run", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--batch", type=int, default=0, help="run the batched-solve benchmark with this many problems")
    ap.add_argument("--autotune", action="store_true", help="autotune launch shapes per handle (off by default: on the 256x256x2 workload the defaults measured faster)")
    ap.add_argument("--clocks-csv", dest="clocks_csv", default="",
                    help="keep the raw nvidia-smi clock samples of the timed region in this CSV file")
    ap.add_argument("--profile-learned", dest="profile_learned", action="store_true",
                    help="time one FP32 preconditioner application with the learned sweep off, on the CUDA cores "
                         "and on the tensor cores (hidden 64, random parameters), then run one of each between "
                         "profiler start and stop; prints the times, no bench line")
    ap.add_argument("--profile-condense", dest="profile_condense", type=int, default=0,
                    help="set up one mixed handle of the flat NxNx2 workload between cudaProfilerStart/Stop")
    ap.add_argument("--profile-batch", dest="profile_batch", action="store_true",
                    help="one merged batched solve of the --batch workload between cudaProfilerStart/Stop")
    ap.add_argument("--profile-solve", dest="profile_solve", default="",
                    choices=["", "mixed", "mixed_bf16", "fgmres64", "fp64"],
                    help="warm up, then run one solve and recovery of this arm between profiler start and stop "
                         "(for ncu --profile-from-start off); prints the iteration count, no bench line")
    args = ap.parse_args()
    if args.profile_solve:
        profile_solve_main(args)
        return
    if args.profile_condense:
        profile_condense_main(args)
        return
    if args.profile_batch:
        profile_batch_main(args)
        return
    if args.profile_learned:
        profile_learned_main(args)
        return
    if args.batch:
        batch_main(args)
        return
    if args.workload == "sequence":
        sequence_main(args)
        return
    if args.workload == "imex":
        imex_main(args)
        return
    if args.workload == "lf":
        lf_main(args)
        return

    if args.oracle_run:
        print(json.dumps(oracle_run(args.p, args.courant, args.warmup, args.steps, kind=args.workload,
                                    direct=args.cpu_direct)))
        return

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    name = workload_label(args.workload, args.p, args.courant, args.seed)

    if args.impl == "reference":
        if rank != 0:
            return
        t0 = time.perf_counter()
        cmd, env = oracle_command(args.p, args.courant, args.warmup, args.steps, args.workload, args.cpu_direct)
        res = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=3600)
        if res.returncode != 0:
            raise RuntimeError(f"oracle run failed: {res.stderr[-2000:]}")
        r = json.loads(res.stdout.strip().splitlines()[-1])
        val = args.steps / r["sec_total"]
        cb = cpu_baseline_entry(r, args.workload, name)
        cb["value"] = val
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * r["sec_total"] / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": name, "rtol": args.rtol},
                "cpu_baseline": cb,
                "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "iters": r["iters"], "wall_s": time.perf_counter() - t0}
        print(json.dumps(line))
        return

    res, fma = gpu_arm(args, rank, world)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle runs in a process of its own (exec'd, so it inherits no CUDA
        # state) after the GPU arms: run beside them, it cost them a few per cent
        cpu = cpu_baseline_entry(oracle_wait(oracle_start(args.p, args.courant, 0, args.oracle_steps, args.workload,
                                                          args.cpu_direct)), args.workload, name)
    if rank != 0:
        return
    if set(res) != {"mixed", "mixed_bf16", "fgmres64", "fp64"}:
        # partial run (profiling): a short summary, not a bench line
        print(json.dumps({k: {"ms_per_step": v["ms"] / args.steps, "iters": [i["iters"] for i in v["infos"]]}
                          for k, v in res.items()}))
        return
    peaks = {}
    ppath = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(ppath):
        peaks = json.load(open(ppath))
    mx, fp, mb, fg = res["mixed"], res["fp64"], res["mixed_bf16"], res["fgmres64"]
    K = args.steps
    value = replica_value(world, K, mx["ms"])
    fp_value = replica_value(world, K, fp["ms"])
    it_mx = [i["iters"] for i in mx["infos"]]
    it_fp = [i["iters"] for i in fp["infos"]]
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": mx["ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 inner + f32x2 (two-float, ~48-bit) refinement, RHS and recovery", "data": "synthetic",
        "config": {"workload": name, "n_cells": mx["n_cells"], "n_trace_dofs": mx["NF"] * mx["pp"],
                   "rtol": args.rtol, "inner_rtol": args.inner_rtol, "restart": args.restart,
                   "smoother": "2+2 block-Jacobi omega=2/3", "coarse": mx["coarse"],
                   "orthogonalisation": "CGS2" if args.reorth else "CGS (one pass)",
                   "l2": (f"inputs larger than L2 (per-cell matrices and trace operator {mx['data_gb']:.2f} GB "
                          f"resident in HBM, L2 129 MB), no flush"),
                   "parallelism": f"replicas x{world}"},
        "iters": it_mx, "true_rel_res": [i["true_rel_res"] for i in mx["infos"]],
        "plain_fp64": {"value": fp_value, "unit": "solves/s", "ms_per_step": fp["ms"] / K, "iters": it_fp,
                       "true_rel_res": [i["true_rel_res"] for i in fp["infos"]],
                       "roofline": roofline(fp, peaks, fma)},
        "mixed_bf16_smoother": {"value": world * K / (mb["ms"] * 1e-3), "unit": "solves/s",
                                "ms_per_step": mb["ms"] / K, "iters": [i["iters"] for i in mb["infos"]],
                                "true_rel_res": [i["true_rel_res"] for i in mb["infos"]],
                                "roofline": roofline(mb, peaks, fma, bf16_pre=True)},
        "fp64_fgmres_fp32_preconditioner": {
            "value": world * K / (fg["ms"] * 1e-3), "unit": "solves/s", "ms_per_step": fg["ms"] / K,
            "iters": [i["iters"] for i in fg["infos"]], "true_rel_res": [i["true_rel_res"] for i in fg["infos"]],
            "e2e": {"value": world * K / fg["e2e_s"], "unit": "solves/s"},
            "precision": "FP64 FGMRES, orthogonalisation, residual, RHS, recovery; FP32 V-cycle, FP64 coarsest solve"},
        "speedup_vs_plain_fp64": value / fp_value,
        "roofline": roofline(mx, peaks, fma),
        "whole_solve": whole_solve(mx, peaks, K),
        "condense_ms": {"mixed": mx["condense_ms"], "fp64": fp["condense_ms"]},
        "condense_fp64_pipe": condense_rate(fp, fma),
        "measured_fma": fma,
        "kernel_ms": {k: v[0] for k, v in mx["prof"].items() if v[1]},
        "gpu_launches": mx["launches"],
        "clocks": mx["clocks"],
        "e2e": {"value": world * K / mx["e2e_s"], "unit": "solves/s", "h2d_bytes_per_step": mx["h2d"],
                "d2h_bytes_per_step": mx["d2h"]},
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()

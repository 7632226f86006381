"""Benchmark: implicit JFNK steps on the 3D stratified convective box.

Workload: problem 4 of `workloads` -- 256^3 cells, walls in z, gravity along
-z, superadiabatic polytrope (index 1.4, density contrast 20), conduction
chi = K0 T^3, seeded velocity noise (rms Mach 1e-3), CFL_hydro = 200,
Crank-Nicolson, sound + conduction physics-based preconditioner, Newton
tolerance 1e-8, GMRES(30) with eta = 1e-4.  A "step" is one implicit time
step (all Newton iterations, each with its GMRES solve: preconditioner
applies, Jacobian-free products, Gram-Schmidt).  The state (670 MB per FP64
vector) is far larger than L2, so no flush is needed between steps.

Arms: the default arm times the CUDA library in mixed precision (FP32 Krylov
basis and preconditioner, FP64 residual) -- `value` -- and the plain FP64
path beside it.  `--impl reference` times the CPU oracle (the only reference
implementation of the paper's method here) on the host cores.

Multi-GPU: the method as built runs on one GPU; with torchrun each rank runs
an independent replica (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "implicit steps/s & Jv Gcell/s at 256³: FP32-Krylov vs FP64 plain, Newton tol 1e-8"
UNIT = "implicit steps/s"
NEWTON_TOL = 1e-8
ETA = 1e-4

# FP64 work per cell of one residual evaluation inside Jv, per kernel (3D,
# internal energy, gravity, conduction, FP32 Krylov vectors), measured with
# the ncu thread-instruction counters of a 128^3 capture (profiles/
# jv_kernels_128cubed.md), divided by the cell count:
#   FP64_INST_PER_CELL       DADD + DMUL + DFMA on the FP64 pipe
#   FP64_PIPE_INST_PER_CELL  every instruction the FP64 pipe executed
#                            (with the reciprocal approximation, ...)
#   INT_PIPE_OPS_PER_CELL    the correctly rounded FP64 products the flux
#                            kernels form on the integer pipes (emu64.cuh),
#                            counted from the source
#   FP64_FLOPS_PER_CELL      dadd + dmul + 2 dfma + the integer-pipe products
# KERNEL_COUNTS_HASH is kernel_source_hash() of the sources those counts were
# measured on (renewed without a new capture only after changes outside the
# five kernels, such as the once-per-Newton k_scaling).
KERNEL_COUNTS_HASH = "0fd12461f02c86f1"
FP64_INST_PER_CELL = {"perturb": 10.0, "eos": 6.0, "face_fluxes": 42.0, "mom_fluxes": 54.0, "assemble": 56.0}
FP64_PIPE_INST_PER_CELL = {"perturb": 10.0, "eos": 6.0, "face_fluxes": 42.0, "mom_fluxes": 54.0, "assemble": 56.0}
INT_PIPE_OPS_PER_CELL = {"perturb": 0.0, "eos": 0.0, "face_fluxes": 24.0, "mom_fluxes": 36.0, "assemble": 7.0}
FP64_FLOPS_PER_CELL = {"perturb": 15.0, "eos": 6.0, "face_fluxes": 84.0, "mom_fluxes": 108.0, "assemble": 95.0}
# DRAM bytes per cell per launch from the same capture (dram__bytes_read +
# dram__bytes_write); at 128^3 part of the reads hit the 129 MB L2, so these
# are lower bounds for 256^3 (where the algorithmic bytes below apply).
DRAM_BYTES_PER_CELL_128 = {"perturb": 112.3, "eos": 17.0, "face_fluxes": 87.0, "mom_fluxes": 99.7,
                           "assemble": 306.4}
JV_KERNELS = ["perturb", "eos", "face_fluxes", "mom_fluxes", "assemble"]
# Algorithmic HBM bytes per cell of one launch of each Jv kernel (3D, FP64
# state, FP32 Krylov vectors; each array the kernel must touch read or
# written once).
HBM_BYTES_PER_CELL = {"perturb": 5 * (8 + 4 + 8) + 3 * 8, "eos": 2 * 8 + 3 * 8, "face_fluxes": 5 * 8 + 3 * 8 + 6 * 8,
                      "mom_fluxes": 3 * 8 + 3 * 8 + 9 * 8, "assemble": 5 * 8 + 8 + 6 * 8 + 9 * 8 + 5 * 8 * 3 + 5 * 4}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "src": "measured"}
    return {"hbm_gbs": 6800.0, "src": "fallback"}


# FP64 peak of GB300 from its unit counts and clock, used only when the
# probe below cannot run: ncu reports a sustained peak of 2 FP64 thread
# instructions per cycle per SM; 152 SMs at the 2070 MHz maximum SM clock give
# 0.629 T instructions/s, 1.26 TFLOP/s with an FMA counted as two flops.
FP64_PEAK_TFLOPS = 1.258
FP64_PEAK_TINST = 0.629


def kernel_source_hash() -> str:
    """Hash of the sources of the Jv kernels whose ncu instruction counts are
    recorded above; the roofline object flags the counts as stale when the
    sources no longer match the hash they were measured at."""
    import hashlib
    h = hashlib.sha256()
    for f in ("residual.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1512_03662_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def fp64_probe(device, stream, reps=5):
    """Measured FP64 issue rate of this GPU: a grid of 8 resident 256-thread
    blocks per SM, each thread running eight independent DFMA chains
    (libfp64probe.so), timed with CUDA events on `stream`; returns the best
    of `reps` launches in T instructions/s (a DFMA is one instruction and two
    flops) with the clocks sampled meanwhile."""
    import ctypes
    import torch
    from paper_1512_03662_gb300 import build as B
    lib = ctypes.CDLL(B.PROBE_LIB)
    lib.fp64_probe_launch.restype = ctypes.c_int
    lib.fp64_probe_launch.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p]
    lib.fp64_probe_fma_per_thread.restype = ctypes.c_longlong
    lib.fp64_probe_fma_per_thread.argtypes = [ctypes.c_int]
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    blocks, iters = sms * 8, 16384
    out = torch.empty(blocks * 256, dtype=torch.float64, device=device)
    ptr, sp = ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream)
    for _ in range(2):
        if lib.fp64_probe_launch(ptr, blocks, iters, 0.999, sp) != 0:
            raise RuntimeError("FP64 probe launch failed")
    clocks = ClockSampler(device.index or 0)
    clocks.start()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            lib.fp64_probe_launch(ptr, blocks, iters, 0.999, sp)
            e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    if not bool(torch.isfinite(out).all()):
        raise RuntimeError("FP64 probe produced non-finite values")
    inst = blocks * 256 * lib.fp64_probe_fma_per_thread(iters)
    best = min(times)
    return {"tinst_s": inst / (best / 1e3) / 1e12, "tflops": 2 * inst / (best / 1e3) / 1e12,
            "ms_best": best, "ms_median": statistics.median(times), "launches": reps, "sms": sms,
            "dfma_per_launch": inst, "clocks": clk}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_workload(n):
    import workloads as W
    wl = W.config(4, n=(n, n, n))
    # same physical time step at any resolution: CFL scales with n
    wl.cfl_hydro = 200.0 * n / 256.0
    return wl


# Solver options of the benchmark: one V(1,1) cycle per preconditioner
# apply (the library default is two V(2,2) cycles).  On this workload one
# cycle needs no more GMRES iterations than two (14.7 vs 15.0 per Newton
# iteration) and the apply costs 40 % less; one pre- and one post-smoothing
# sweep instead of two need 1.7 % more GMRES iterations per step over five
# steps and make the apply 2.05 instead of 2.70 ms (0.526 vs 0.513 steps/s
# over steps 4-8).  At much longer time steps than the workload's (problem
# 2 at 32^2 and CFL 100) one cycle is not enough, hence the library
# default.  Command-line options override these.
OPT_OVERRIDES = {"mg_cycles": 1, "mg_nu1": 1, "mg_nu2": 1}
# the options given on the command line alone (the studies otherwise use the
# library defaults)
CLI_OPTS = {}
# lambda of the extra arm of the benchmark line.  At lambda = 1e-7 (Sect.
# 5.1.1) the first-order truncation error of the Jacobian-free quotient
# limits the late Newton iterations of this workload (about 1e-2 of the
# linear residual: see tests/test_oracle_newton_convergence.py).  Eq.
# pert_old makes delta grow with ||R^-1 X||, i.e. with the square root of
# the number of unknowns, so the perturbation the paper tuned at 64^3 is
# reached at 256^3 with lambda = 1e-7 (64/256)^(3/2) = 1.25e-8; the arm
# reports the step rate with that lambda beside the headline.
LAM_ARM = 1.25e-8


def run_arm(jf, wl, precision, steps, warmup, device, stream, profile):
    import torch
    o = jf.default_options(theta=wl.theta, precond=wl.precond, precision=precision, **OPT_OVERRIDES)
    S = jf.Solver.from_workload(wl, o, device=device, stream=stream)
    X0 = torch.as_tensor(wl.X0, dtype=torch.float64, device=device)
    X = X0.clone()
    dt = S.dt_from_cfl(X, wl.cfl_hydro)
    for _ in range(warmup):
        st = S.step(X, dt, NEWTON_TOL, ETA)
    S.set_profiling(profile)
    stats = []
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(steps):
            stats.append(S.step(X, dt, NEWTON_TOL, ETA))
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    S.set_profiling(False)
    return S, X0, dt, ms, stats, X


def e2e_arm(jf, wl, precision, steps, warmup, device, stream, S=None):
    """Same metric through the public API with HOST buffers: every step copies
    the state from pinned host memory to the device, steps, and copies the
    new state back.  The same warm-up steps as the device arm come first, so
    both time the same steps of the run.  S: the solver to step (the device
    arm's, as a user keeps one solver for a run), else a new one."""
    import torch
    if S is None:
        o = jf.default_options(theta=wl.theta, precond=wl.precond, precision=precision, **OPT_OVERRIDES)
        S = jf.Solver.from_workload(wl, o, device=device, stream=stream)
    host = torch.as_tensor(wl.X0, dtype=torch.float64).pin_memory()
    X = torch.empty_like(host, device=device)
    with torch.cuda.stream(stream):
        X.copy_(host, non_blocking=True)
    dt = S.dt_from_cfl(X, wl.cfl_hydro)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            X.copy_(host, non_blocking=True)
            S.step(X, dt, NEWTON_TOL, ETA)
            host.copy_(X, non_blocking=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stats = []
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(steps):
            X.copy_(host, non_blocking=True)
            stats.append(S.step(X, dt, NEWTON_TOL, ETA))
            host.copy_(X, non_blocking=True)
        e1.record(stream)
    torch.cuda.synchronize()
    nbytes = host.numel() * 8
    return e0.elapsed_time(e1), nbytes, stats


def convergence(stats) -> dict:
    """Counts over the timed steps: steps that met the Newton tolerance,
    steps stopped at newton_max, and linear solves stopped at gmres_max_it."""
    return {"steps_converged": sum(1 for s in stats if s["converged"]),
            "steps_timed": len(stats),
            "newton_capped": sum(1 for s in stats if not s["converged"]),
            "gmres_capped": sum(1 - c for s in stats for c in s["gmres_converged"]),
            "linear_solves": sum(s["newton_iterations"] for s in stats)}


def oracle_sample(n_small=32, steps=1, with_stats=False):
    """The CPU oracle as it stands: implicit steps of the same construction at
    n_small^3 with the same physical dt and solver settings; returns (s per
    step, threads) and, with with_stats, the Newton and GMRES counts."""
    import torch
    from oracle import discretization as D
    from oracle import jfnk as J
    wl = make_workload(n_small)
    P = D.Problem.from_workload(wl)
    dt = D.cfl_dt(P, wl.X0, wl.cfl_hydro)
    X = torch.as_tensor(wl.X0)
    t0 = time.perf_counter()
    st = None
    for _ in range(steps):
        X, st = J.newton_step(P, X, dt, J.Options(precond=wl.precond, newton_tol=NEWTON_TOL, eta=ETA,
                                                   **OPT_OVERRIDES))
    sec = (time.perf_counter() - t0) / steps
    if with_stats:
        return sec, torch.get_num_threads(), {"newton_iterations": st.newton_iterations,
                                              "gmres_iterations": list(st.gmres_iterations),
                                              "converged": bool(st.converged)}
    return sec, torch.get_num_threads()


def cpu_info() -> dict:
    """Host CPU: logical core count and model name (lscpu, else /proc/cpuinfo)."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    return {"logical_cores": os.cpu_count(), "model": model, "machine": platform.machine()}


def oracle_kernels(wl, threads: int, reps: int) -> dict:
    """The oracle's residual F(X; X^n) (two evaluations of R_U, as
    jfnk_residual) and one Jacobian-free product (one evaluation of G, G(X)
    precomputed as in GMRES) on the workload itself, `reps` calls each with
    `threads` torch threads: median seconds and cells per second."""
    import torch
    from oracle import discretization as D
    from oracle import jfnk as J
    import workloads as W
    old = torch.get_num_threads()
    torch.set_num_threads(threads)
    try:
        P = D.Problem.from_workload(wl)
        X = torch.as_tensor(wl.X0)
        dt = D.cfl_dt(P, X, wl.cfl_hydro)
        tr = []
        for _ in range(reps):
            t0 = time.perf_counter()
            D.residual(P, X, X, dt)
            tr.append(time.perf_counter() - t0)
        o = J.Options(precond=wl.precond)
        sc = J.scaling(P, X, o)
        G0 = D.G_operator(P, X, dt)
        v = torch.as_tensor(W.random_vector(wl, 3))
        tj = []
        for _ in range(reps):
            t0 = time.perf_counter()
            J.jv(P, X, G0, sc, v, dt, o)
            tj.append(time.perf_counter() - t0)
        del sc, G0, v
    finally:
        torch.set_num_threads(old)
    mr, mj = statistics.median(tr), statistics.median(tj)
    return {"threads": threads, "calls": reps, "residual_s": mr, "jv_s": mj,
            "residual_gcell_s": wl.ncell / mr / 1e9, "jv_gcell_s": wl.ncell / mj / 1e9}


def reference_main(args, ws, rank):
    n_small = args.ref_n
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(n_small, 1)
    secs = []
    threads = 1
    for _ in range(args.steps):
        s, threads = oracle_sample(n_small, 1)
        secs.append(s)
    mean = sum(secs) / len(secs)
    scale = (n_small / args.n) ** 3
    value = scale / mean          # steps/s of the full grid, from the sample by the cell ratio
    # ms_per_step is the time of the steps this run timed (one oracle step of
    # the sample each); value is the rate of the full-size workload derived
    # from it (its time per step: ms_per_step_full_size)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * mean,
            "ms_per_step_full_size": 1e3 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"convbox3d {args.n}^3 (problem 4)",
                       "parallelism": "replicas", "l2": "state larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"oracle implicit step at {n_small}^3 (same construction, same dt), "
                                       f"time scaled by the cell ratio ({args.n}/{n_small})^3",
                             "seconds_per_sample": mean, "host": cpu_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def kernel_main(args):
    """--only jv|precond|vjp: repeated Jacobian-free products, preconditioner
    applies or transposed residual Jacobian products (vjp, FP64) at one state
    of the workload, for kernel timing and profiling."""
    import torch
    from paper_1512_03662_gb300 import build as B
    B.build()
    import paper_1512_03662_gb300 as jf
    import workloads as W
    device = torch.device("cuda:0")
    stream = torch.cuda.Stream(device)
    wl = make_workload(args.n)
    prec = jf.FP64 if (args.precision == "fp64" or args.only == "vjp") else jf.MIXED
    # a single Jv or preconditioner call needs no Krylov basis: restart length 1
    o = jf.default_options(theta=wl.theta, precond=wl.precond, precision=prec, gmres_m=1, **OPT_OVERRIDES)
    S = jf.Solver.from_workload(wl, o, device=device, stream=stream)
    X = torch.as_tensor(wl.X0, dtype=torch.float64, device=device)
    dt = S.dt_from_cfl(X, wl.cfl_hydro)
    v = torch.as_tensor(W.random_vector(wl, 3), device=device).to(S.vdtype)
    out = torch.empty_like(v)
    if args.only == "jv":
        call = lambda: S.jv(X, dt, v, out)                  # noqa: E731
    elif args.only == "precond":
        call = lambda: S.precond_apply(X, dt, v, out)       # noqa: E731
    else:
        call = lambda: S.vjp_residual(X, dt, v)             # noqa: E731
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(args.steps):
            call()
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"only": args.only, "n": args.n, "precision": "fp64" if prec == jf.FP64 else "mixed",
                      "ms_per_call": ms,
                      "gcell_s": wl.ncell / (ms / 1e3) / 1e9}))


# Taylor-Green vortex 64^3 (Sect. 5.1.2), the paper's Table 1 (implicit
# columns: CFL_hydro, CFL_adv, Newton per step, GMRES per Newton, parabolic
# iterations per GMRES) and Table 2 (time and value of the peak kinetic
# energy decay rate), for comparison beside this solver's figures.
TGV_TABLE1 = {1e-1: (7.1, 0.5, 3.8, 16.6, 2.4), 1e-2: (70.0, 0.5, 3.1, 15.4, 2.5),
              1e-3: (820.0, 0.5, 2.7, 16.2, 2.5), 1e-4: (1.1e4, 0.5, 2.0, 16.1, 2.8),
              1e-5: (8.1e4, 0.5, 2.0, 22.2, 2.9), 1e-6: (4.9e5, 0.49, 4.5, 291.5, 3.0)}
TGV_TABLE2 = {1e-1: (8.1656, 1.2504e-2), 1e-2: (8.1695, 1.2496e-2), 1e-3: (8.1695, 1.2496e-2),
              1e-4: (8.1696, 1.2496e-2), 1e-5: (8.1695, 1.2498e-2), 1e-6: (8.1681, 1.2520e-2)}


def tgv_speed_max(X, nc):
    """max over cells of |u| with u the cell mean of the face velocities."""
    import torch
    n = round(nc ** (1.0 / 3.0))
    sq = 0.0
    for d in range(3):
        u = X[(2 + d) * nc:(3 + d) * nc].reshape(n, n, n)
        ub = 0.5 * (u + torch.roll(u, -1, dims=2 - d))
        sq = sq + ub * ub
    return float(sq.sqrt().max())


def tgv_kinetic_energy(X, nc):
    """Volume mean of rho_f u_f^2 / 2 summed over the face velocities."""
    import torch
    n = round(nc ** (1.0 / 3.0))
    rho = X[:nc].reshape(n, n, n)
    ke = 0.0
    for d in range(3):
        u = X[(2 + d) * nc:(3 + d) * nc].reshape(n, n, n)
        rf = 0.5 * (rho + torch.roll(rho, 1, dims=2 - d))
        ke = ke + float((0.5 * rf * u * u).mean())
    return ke


def study_tgv(args):
    """--study tgv: the Taylor-Green runs of Sect. 5.1.2 at 64^3.  For each
    Mach number: 100 steps at CFL_hydro = 1 to let the initial acoustic
    transient pass (as in the paper), then --steps steps at CFL_adv = 0.5
    (and 0.05 for M = 1e-6), reporting Newton iterations per step, GMRES
    iterations per Newton iteration and the simulated time per wall-clock
    second.  --decay adds a run from t = 0 to t = 20 at CFL_adv = 0.5 with
    the peak of the kinetic energy decay rate; --sweep adds GMRES iterations
    against CFL_hydro with and without the preconditioner (alpha1 = 1
    without, as in the paper's Fig. tgv)."""
    import torch
    from paper_1512_03662_gb300 import build as B
    B.build()
    import paper_1512_03662_gb300 as jf
    import workloads as W
    prec = jf.FP64 if args.precision == "fp64" else jf.MIXED
    n = args.study_n or 64
    h = 2.0 * math.pi / n
    machs = [float(m) for m in (args.machs or "1e-1,1e-2,1e-3,1e-4,1e-5,1e-6").split(",")]

    def solver(wl, **kw):
        o = jf.default_options(**{"theta": wl.theta, "precond": wl.precond, "precision": prec, **CLI_OPTS, **kw})
        return jf.Solver.from_workload(wl, o)

    def run(S, X, dt, steps, tol=NEWTON_TOL):
        """steps implicit steps; stops at the first step that fails (error
        status), whose message is returned beside the statistics"""
        stats, err = [], None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            try:
                stats.append(S.step(X, dt, tol, ETA))
            except jf.JFNKError as e:
                err = str(e)
                break
        torch.cuda.synchronize()
        return time.perf_counter() - t0, stats, err

    def summary(stats, err=None):
        if not stats:
            return {"steps_done": 0, "error": err}
        nn = sum(s["newton_iterations"] for s in stats)
        its = [g for s in stats for g in s["gmres_iterations"]]
        return {"newton_per_step": nn / len(stats), "gmres_per_newton": sum(its) / max(1, nn),
                "gmres_min": min(its), "gmres_max": max(its),
                "unconverged_linear_solves": sum(1 - c for s in stats for c in s["gmres_converged"]),
                "steps_converged": sum(1 for s in stats if s["converged"]), "steps_done": len(stats),
                "error": err}

    for mach in machs:
        wl = W.make_tgv(n, mach)
        S = solver(wl)
        X = torch.as_tensor(wl.X0, dtype=torch.float64, device="cuda")
        _, _, err = run(S, X, S.dt_from_cfl(X, 1.0), 100)
        if err:
            print(json.dumps({"study": "tgv", "mach": mach, "transient_error": err}), flush=True)
            continue
        Xt = X.clone()
        cs = 1.0 / mach          # background sound speed sqrt(gamma p_0 / rho_0) = u_0 / M_s
        for cfl_adv in ([0.5, 0.05] if mach <= 1e-6 else [0.5]):
            X.copy_(Xt)
            dt = cfl_adv * h / tgv_speed_max(X, wl.ncell)
            el, stats, err = run(S, X, dt, args.steps)
            done = max(1, len(stats))
            line = {"study": "tgv", "mach": mach, "n": n, "precision": args.precision, "cfl_adv": cfl_adv,
                    "cfl_hydro": dt * (tgv_speed_max(Xt, wl.ncell) + cs) / h, "dt": dt, "steps": args.steps,
                    "steps_per_s": done / el, "sim_time_per_s": done * dt / el,
                    "vcycles_per_gmres": S.options.mg_cycles, **summary(stats, err)}
            if cfl_adv == 0.5 and mach in TGV_TABLE1:
                line["paper_table1"] = dict(zip(["cfl_hydro", "cfl_adv", "newton_per_step", "gmres_per_newton",
                                                 "parabolic_per_gmres"], TGV_TABLE1[mach]))
            print(json.dumps(line), flush=True)
        if args.sweep:
            for cfl in (0.1, 1.0, 10.0, 100.0, 1e3, 1e4, 1e5):
                if cfl * mach > 1.0:     # CFL_adv ~ CFL_hydro M_s > 1: the SI scheme is unstable there
                    continue
                res = {"study": "tgv_sweep", "mach": mach, "cfl_hydro": cfl}
                for tag, kw in (("pbp", {}), ("none_alpha1", {"precond": 0, "alpha1": 1.0})):
                    S2 = solver(wl, **kw) if kw else S
                    X.copy_(Xt)
                    dt = S2.dt_from_cfl(X, cfl)
                    el, stats, err = run(S2, X, dt, 5)
                    res[tag] = summary(stats, err)
                print(json.dumps(res), flush=True)
        if args.decay:
            X = torch.as_tensor(wl.X0, dtype=torch.float64, device="cuda")
            dt = 0.5 * h / tgv_speed_max(X, wl.ncell)
            nsteps = int(math.ceil(20.0 / dt))
            ke = [tgv_kinetic_energy(X, wl.ncell)]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            its, err = 0, None
            for _ in range(nsteps):
                try:
                    st = S.step(X, dt, NEWTON_TOL, ETA)
                except jf.JFNKError as e:
                    err = str(e)
                    break
                its += st["gmres_iterations_total"]
                ke.append(tgv_kinetic_energy(X, wl.ncell))
            el = time.perf_counter() - t0
            if err or len(ke) < 3:
                print(json.dumps({"study": "tgv_decay", "mach": mach, "error": err, "steps_done": len(ke) - 1}),
                      flush=True)
                continue
            rate = [-(ke[k + 1] - ke[k - 1]) / (2 * dt) for k in range(1, len(ke) - 1)]
            k = max(range(len(rate)), key=lambda i: rate[i])
            line = {"study": "tgv_decay", "mach": mach, "dt": dt, "steps": nsteps, "wall_s": el,
                    "ke0": ke[0], "ke_end": ke[-1], "t_peak": (k + 1) * dt, "rate_peak": rate[k],
                    "gmres_total": its}
            if mach in TGV_TABLE2:
                line["paper_table2"] = {"t_peak": TGV_TABLE2[mach][0], "rate_peak": TGV_TABLE2[mach][1]}
            print(json.dumps(line), flush=True)


def vortex_run(jf, wl, u_exact, dt, nsteps, arm, prec, opts):
    """Advect the isentropic vortex nsteps steps of dt with the JFNK+PBP step
    (arm "jfnk") or the SI stepper (arm "si"); errors of u against u_exact
    as the paper defines them (L1, L2: means over the grid; Linf: max)."""
    import torch
    nc = wl.ncell
    theta = 0.5 if arm == "jfnk" else 1.0
    o = jf.default_options(**{"theta": theta, "precond": 1, "precision": prec, **opts})
    S = jf.Solver.from_workload(wl, o)
    X = torch.as_tensor(wl.X0, dtype=torch.float64, device="cuda")
    err, newton, gmres = None, 0, 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(nsteps):
        try:
            if arm == "jfnk":
                st = S.step(X, dt, o.newton_tol, o.eta)
                newton += st["newton_iterations"]
                gmres += st["gmres_iterations_total"]
                if not st["converged"]:
                    err = "Newton did not converge"
                    break
            else:
                S.si_step(X, dt)
        except jf.JFNKError as e:
            err = str(e)
            break
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    d = X[2 * nc:3 * nc] - u_exact
    ok = err is None and bool(torch.isfinite(d).all())
    r = {"wall_s": el, "L1": float(d.abs().mean()) if ok else None,
         "L2": float(d.pow(2).mean().sqrt()) if ok else None, "Linf": float(d.abs().max()) if ok else None,
         "error": err if err else (None if ok else "non-finite state")}
    if arm == "jfnk":
        r["newton_per_step"] = newton / nsteps
        r["gmres_per_newton"] = gmres / max(1, newton)
    return r


def study_vortex(args):
    """--study vortex: the advected isentropic vortex of Sects. 3.7 and 5.1.1
    at 64^2, advected to t = 0.4 at T_inf = 1, 1e2, 1e6, 1e10 (Mach 1e-1 ...
    1e-6) for a range of advective CFL numbers, with the JFNK+PBP step
    (Crank-Nicolson) and with the SI scheme as a time integrator (one SI
    solve per step, theta = 1).  Reports the L1, L2 and Linf errors of the
    velocity along the advection against the shifted initial field, as the
    paper defines them.
    --study params: the JFNK+PBP free parameters of Sect. 5.1.1 (perturbation
    formula and lambda, alpha1, eta) on the same vortex at CFL_adv = 0.3 and
    1, for M = 1e-1, 1e-4, 1e-6."""
    import torch
    from paper_1512_03662_gb300 import build as B
    B.build()
    import paper_1512_03662_gb300 as jf
    import workloads as W
    prec = jf.FP64 if args.precision == "fp64" else jf.MIXED
    n, t_end = 64, 0.4
    dx = 8.0 / n
    if args.study == "vortex":
        T_list, cfls = (1.0, 1e2, 1e6, 1e10), (0.01, 0.03, 0.1, 0.3, 1.0, 3.0)
        cases = [("jfnk", "default", {}), ("si", "default", {})]
    else:
        T_list, cfls = (1.0, 1e6, 1e10), (0.3, 1.0)
        cases = [("jfnk", "pert_old lambda 1e-7 (default)", {}),
                 ("jfnk", "pert_old lambda 1e-6", {"lam": 1e-6}),
                 ("jfnk", "pert_new lambda 1e-7", {"pert": 1}),
                 ("jfnk", "pert_new lambda 1e-6", {"pert": 1, "lam": 1e-6}),
                 ("jfnk", "alpha1 1", {"alpha1": 1.0}),
                 ("jfnk", "eta 1e-2", {"eta": 1e-2})]
    for T_inf in T_list:
        wl = W.make_isentropic_vortex(n, T_inf)
        nc = wl.ncell
        u_exact = torch.as_tensor(W.make_isentropic_vortex(n, T_inf, x_shift=t_end).X0[2 * nc:3 * nc],
                                  device="cuda")
        mach = 0.75 / (2.0 * math.pi * math.sqrt(wl.gamma * T_inf))
        for cfl_adv in cfls:
            nsteps = max(1, round(t_end / (cfl_adv * dx)))
            dt = t_end / nsteps
            for arm, name, kw in cases:
                opts = {"newton_tol": NEWTON_TOL, "eta": ETA, **CLI_OPTS, **kw}
                r = vortex_run(jf, wl, u_exact, dt, nsteps, arm, prec, opts)
                print(json.dumps({"study": args.study, "arm": arm, "variant": name, "T_inf": T_inf, "mach": mach,
                                  "cfl_adv": cfl_adv, "cfl_hydro": dt * (1.0 + math.sqrt(wl.gamma * T_inf)) / dx,
                                  "steps": nsteps, **r}), flush=True)


def study_inner(args):
    """--study inner: accuracy of the inner SI solve (the paper's eta' of
    Sect. 3.5, which the paper leaves for future investigation, noting that
    eta' <= 1e-6 behaves like a direct solve) and SI coefficients from each
    Newton iterate or frozen at X^n, on the Taylor-Green vortex 64^3 (M =
    1e-2, 1e-4, CFL_adv = 0.5, after 100 steps at CFL_hydro = 1), problem 2
    at 256^2 (conduction, CFL 100) and problem 4 at --n^3 (default 128^3,
    the benchmark's time step).  Arms: a fixed number of V-cycles per apply
    (1, 2, 4) with the inner residual measured after every apply, and V-cycles
    repeated until the measured relative residual reaches eta' = 1e-2, 1e-4,
    1e-6 or 1e-10 ("direct").  Reports GMRES iterations per Newton
    iteration, V-cycles per apply, the measured eta' (mean and maximum over
    the applies) and the step rate."""
    import torch
    from paper_1512_03662_gb300 import build as B
    B.build()
    import paper_1512_03662_gb300 as jf
    import workloads as W
    prec = jf.FP64 if args.precision == "fp64" else jf.MIXED
    cases = []
    for mach in (1e-2, 1e-4):
        wl = W.make_tgv(64, mach)
        S = jf.Solver.from_workload(wl, jf.default_options(theta=wl.theta, precond=wl.precond, precision=prec))
        X = torch.as_tensor(wl.X0, dtype=torch.float64, device="cuda")
        dt1 = S.dt_from_cfl(X, 1.0)
        for _ in range(100):
            S.step(X, dt1, NEWTON_TOL, ETA)
        dt = 0.5 * (2.0 * math.pi / 64) / tgv_speed_max(X, wl.ncell)
        cases.append((f"tgv64 M={mach:g}", wl, X.clone(), dt))
        del S
    wl = W.config(2)
    X = torch.as_tensor(wl.X0, dtype=torch.float64, device="cuda")
    S = jf.Solver.from_workload(wl, jf.default_options(theta=wl.theta, precond=wl.precond, precision=prec))
    cases.append(("problem2 256^2", wl, X, S.dt_from_cfl(X, wl.cfl_hydro)))
    del S
    n4 = args.study_n or 128
    wl = make_workload(n4)
    X = torch.as_tensor(wl.X0, dtype=torch.float64, device="cuda")
    S = jf.Solver.from_workload(wl, jf.default_options(theta=wl.theta, precond=wl.precond, precision=prec))
    cases.append((f"problem4 {n4}^3", wl, X, S.dt_from_cfl(X, wl.cfl_hydro)))
    del S
    arms = [(f"fixed {c} V({nu},{nu})", {"mg_cycles": c, "mg_nu1": nu, "mg_nu2": nu, "inner_monitor": 1})
            for c, nu in ((1, 1), (1, 2), (2, 2), (4, 2))]
    arms += [(f"eta' {tol:g}", {"inner_tol": tol, "inner_max_cycles": 60}) for tol in (1e-2, 1e-4, 1e-6, 1e-10)]
    arms += [("fixed 1 V(2,2), frozen at X^n", {"mg_cycles": 1, "pc_freeze": 1, "inner_monitor": 1})]
    for name, wl, X0, dt in cases:
        for arm, kw in arms:
            o = jf.default_options(**{"theta": wl.theta, "precond": wl.precond, "precision": prec, **kw})
            S = jf.Solver.from_workload(wl, o)
            X = X0.clone()
            nn = ng = napp = ncyc = 0
            emean, emax, err = [], 0.0, None
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            k = 0
            for k in range(args.steps):
                try:
                    st = S.step(X, dt, NEWTON_TOL, ETA)
                except jf.JFNKError as e:
                    err = str(e)
                    break
                nn += st["newton_iterations"]
                ng += st["gmres_iterations_total"]
                napp += st["precond_applies"]
                ncyc += st["inner_cycles"]
                emean.append(st["inner_res_mean"] * st["precond_applies"])
                emax = max(emax, st["inner_res_max"])
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            print(json.dumps({"study": "inner", "case": name, "arm": arm, "steps": args.steps,
                              "steps_per_s": args.steps / el if err is None else None,
                              "newton_per_step": nn / max(1, k + (err is None)),
                              "gmres_per_newton": ng / max(1, nn), "vcycles_per_apply": ncyc / max(1, napp),
                              "eta_inner_mean": sum(emean) / max(1, napp), "eta_inner_max": emax,
                              "error": err}), flush=True)
            del S
            torch.cuda.empty_cache()


def study_newton(args):
    """--study newton: Newton convergence of the benchmark workload (problem 4
    at --n^3, the benchmark's solver options) for each lambda of --lams
    (default 1e-7, 1e-8, 1e-9, 1e-10): per step the Newton iterations, GMRES
    iterations, ||F^|| at each iterate, ||R^-1 dX||_inf and the GMRES
    residual estimate; per lambda the step rate and the largest scaled
    difference of the final state from the first lambda's."""
    import torch
    from paper_1512_03662_gb300 import build as B
    B.build()
    import paper_1512_03662_gb300 as jf
    prec = jf.FP64 if args.precision == "fp64" else jf.MIXED
    lams = [float(x) for x in (args.lams or "1e-7,1e-8,1e-9,1e-10").split(",")]
    first = None
    for lam in lams:
        wl = make_workload(args.n)
        o = jf.default_options(theta=wl.theta, precond=wl.precond, precision=prec, **{**OPT_OVERRIDES, "lam": lam})
        S = jf.Solver.from_workload(wl, o)
        X = torch.as_tensor(wl.X0, dtype=torch.float64, device="cuda")
        dt = S.dt_from_cfl(X, wl.cfl_hydro)
        nn = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            st = S.step(X, dt, NEWTON_TOL, ETA)
            nn += st["newton_iterations"]
            print(json.dumps({"study": "newton", "lam": lam, "step": k, "newton": st["newton_iterations"],
                              "converged": st["converged"], "gmres": st["gmres_iterations"],
                              "fhat": st["fhat_norm"], "dx_inf": st["dx_inf"], "gmres_res": st["gmres_res"]}),
                  flush=True)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        _, R, _ = S.scaling(X)
        if first is None:
            first = X.clone()
        print(json.dumps({"study": "newton_summary", "lam": lam, "n": args.n, "steps": args.steps,
                          "steps_per_s": args.steps / el, "newton_per_step": nn / args.steps,
                          "max_scaled_diff_vs_first_lambda": float(((X - first) / R).abs().max())}), flush=True)
        del S
        torch.cuda.empty_cache()


def study_adjoint(args):
    """--study adjoint: the gradient of the adjoint workload (problem 5,
    128^2, 4 implicit steps at CFL_hydro = 50, FP64): loss = final kinetic
    energy, gradients with respect to the initial temperature perturbation
    field and K0 by one transposed Newton-system solve per step (jfnk_vjp),
    as torch.autograd does through JFNKStep.  Times the forward steps and
    the backward pass and reports the GMRES iterations of both."""
    import torch
    from paper_1512_03662_gb300 import build as B
    B.build()
    import paper_1512_03662_gb300 as jf
    import workloads as W
    wl = W.config(5)
    nc = wl.ncell
    o = jf.default_options(**{"theta": wl.theta, "precond": wl.precond, "precision": jf.FP64, "eta": 1e-10,
                              **CLI_OPTS})
    S = jf.Solver.from_workload(wl, o)
    X0 = torch.as_tensor(wl.X0, dtype=torch.float64, device="cuda")
    dt = S.dt_from_cfl(X0, wl.cfl_hydro)
    n = round(math.sqrt(nc))

    dV = wl.dx[0] * wl.dx[1]

    def kinetic_energy_grad(X):
        """d/dX of the sum over faces of rho_f u_f^2 / 2 dV (periodic in x,
        walls in y: the y slot 0 is the wall face, zero, and jfnk_vjp masks
        wall slots of the gradient it receives)"""
        Xg = X.detach().clone().requires_grad_(True)
        rho = Xg[:nc].reshape(n, n)
        ke = 0.0
        for c in range(2):
            u = Xg[(2 + c) * nc:(3 + c) * nc].reshape(n, n)
            rl = torch.roll(rho, 1, dims=1 - c)
            ke = ke + (0.25 * (rl + rho) * u * u).sum() * dV
        ke.backward()
        return Xg.grad.detach()

    for rep in range(2):                                   # the first repetition warms up
        traj = [X0.clone()]
        fstats = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(wl.n_steps):
            X = traj[-1].clone()
            fstats.append(S.step(X, dt, 1e-12, 1e-10))
            traj.append(X)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        g = kinetic_energy_grad(traj[-1])
        gk, bits = 0.0, []
        for k in range(wl.n_steps, 0, -1):
            gXn, gK0, st, code = S.vjp(traj[k - 1], traj[k], dt, g)
            g, gk = gXn, gk + gK0
            bits.append(st["gmres_iterations_total"])
        torch.cuda.synchronize()
        t2 = time.perf_counter()
    line = {"study": "adjoint", "workload": "adjoint2d 128^2 (problem 5), 4 steps, CFL_hydro 50, FP64",
            "forward_ms": 1e3 * (t1 - t0), "backward_ms": 1e3 * (t2 - t1), "backward_over_forward": (t2 - t1) / (t1 - t0),
            "forward_newton": [s["newton_iterations"] for s in fstats],
            "forward_gmres": [s["gmres_iterations_total"] for s in fstats],
            "adjoint_gmres": bits[::-1], "grad_norm": float(g.norm()), "dL_dK0": gk}
    print(json.dumps(line), flush=True)


def study_machsweep(args):
    """--study machsweep: the 3D vortex tube (problem 3: Gresho profile in
    x-y, uniform along z, periodic, seeded 1e-6 density noise, Crank-Nicolson,
    CFL_hydro = 1000, sound-wave preconditioner) at --study-n^3 (default 128)
    for each Mach number of --machs (default 1e-2, 1e-4, 1e-6): the
    workload's five steps with the FP64 handle and with the mixed handle from
    the same X^0.  Reports steps/s, Newton and GMRES iterations, and after
    each step the difference of the two states: scaled (max |dX| / R), in
    the velocity relative to max |u|, and in the pressure relative to the
    range of the pressure fluctuation (about M^2 p).  --cfl overrides
    CFL_hydro (at Mach 1e-2 the workload's 1000 is an advective CFL of 10,
    where GMRES stops at its iteration cap).  The same measures against the
    oracle, on a small grid, are a parity test."""
    import torch
    from paper_1512_03662_gb300 import build as B
    B.build()
    import paper_1512_03662_gb300 as jf
    import workloads as W
    n = args.study_n or 128
    machs = [float(m) for m in (args.machs or "1e-2,1e-4,1e-6").split(",")]

    def measures(wl, Xa, Xb, Rb):
        """differences of state Xa from the reference state Xb"""
        nc = wl.ncell
        d = (Xa - Xb)
        g1 = wl.gamma - 1.0
        pa = g1 * Xa[:nc] * Xa[nc:2 * nc]
        pb = g1 * Xb[:nc] * Xb[nc:2 * nc]
        ub = Xb[2 * nc:]
        return {"scaled": float((d / Rb).abs().max()),
                "velocity": float(d[2 * nc:].abs().max() / ub.abs().max()),
                "pressure": float((pa - pb).abs().max() / (pb.max() - pb.min()))}

    def run(wl, prec, steps, X0, dt):
        o = jf.default_options(**{"theta": wl.theta, "precond": wl.precond, "precision": prec, **CLI_OPTS})
        S = jf.Solver.from_workload(wl, o)
        if dt is None:
            dt = S.dt_from_cfl(X0, wl.cfl_hydro)
        X = X0.clone()
        traj, stats = [], []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            stats.append(S.step(X, dt, NEWTON_TOL, ETA))
            traj.append(X.clone())
        torch.cuda.synchronize()
        return S, traj, stats, time.perf_counter() - t0, dt

    for mach in machs:
        wl = W.config(3, n=(n, n, n), mach=mach)
        if args.cfl is not None:
            wl.cfl_hydro = args.cfl
        X0 = torch.as_tensor(wl.X0, dtype=torch.float64, device="cuda")
        line = {"study": "machsweep", "workload": f"vortextube3d {n}^3 (problem 3), CFL_hydro {wl.cfl_hydro:g}",
                "mach": mach, "cfl_adv_approx": mach * wl.cfl_hydro, "steps": wl.n_steps}
        arms, dt = {}, None
        for name, prec in (("fp64", jf.FP64), ("mixed", jf.MIXED)):
            S, traj, stats, sec, dt = run(wl, prec, wl.n_steps, X0, dt)
            nn = sum(s["newton_iterations"] for s in stats)
            line[name] = {"steps_per_s": wl.n_steps / sec, "newton_per_step": nn / len(stats),
                          "gmres_per_newton": sum(s["gmres_iterations_total"] for s in stats) / max(1, nn),
                          "steps_converged": sum(1 for s in stats if s["converged"])}
            arms[name] = (S, traj)
        S64, t64 = arms["fp64"]
        diffs = []
        for k in range(wl.n_steps):
            _, R, _ = S64.scaling(t64[k])
            diffs.append(measures(wl, arms["mixed"][1][k], t64[k], R))
        line["mixed_vs_fp64_per_step"] = diffs
        del arms, S64, t64
        torch.cuda.empty_cache()
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="cells per direction")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison arm")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-new-solver", action="store_true",
                    help="end-to-end arm on a solver of its own instead of the device arm's")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-probe", action="store_true",
                    help="skip the FP64 peak probe (the roofline then uses the unit-count peak)")
    ap.add_argument("--only", choices=["jv", "precond", "vjp"], default=None,
                    help="time only repeated Jv or preconditioner calls (profiling)")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--mg-cycles", type=int, default=None, help="multigrid V-cycles per preconditioner apply")
    ap.add_argument("--mg-nu1", type=int, default=None, help="pre-smoothing sweeps")
    ap.add_argument("--mg-nu2", type=int, default=None, help="post-smoothing sweeps")
    ap.add_argument("--eta", type=float, default=None,
                    help="GMRES relative tolerance (the paper's 1e-4 unless given)")
    ap.add_argument("--lam", type=float, default=None,
                    help="lambda of the perturbation size, Eq. pert_old (library default 1e-7)")
    ap.add_argument("--pc-freeze", type=int, default=None, choices=[0, 1],
                    help="1: preconditioner coefficients from X^n for the whole step")
    ap.add_argument("--study", choices=["tgv", "vortex", "params", "inner", "adjoint", "machsweep", "newton"],
                    default=None,
                    help="tgv: the Taylor-Green iteration and decay study of Sect. 5.1.2; vortex: the "
                         "isentropic-vortex accuracy study of Sects. 3.7 and 5.1.1; params: the JFNK+PBP "
                         "parameter variants of Sect. 5.1.1 on the vortex; inner: V-cycle count and frozen "
                         "coefficients; adjoint: forward and backward time of the adjoint workload; "
                         "machsweep: FP64 and mixed steps of the 3D vortex tube per Mach number; newton: Newton "
                         "convergence of the benchmark workload per lambda (JSON lines)")
    ap.add_argument("--lams", default=None, help="lambdas of --study newton (default 1e-7,1e-8,1e-9,1e-10)")
    ap.add_argument("--lam-arm", type=float, default=LAM_ARM,
                    help="lambda of the extra mixed-precision arm of the benchmark line (0: none)")
    ap.add_argument("--machs", default=None,
                    help="Mach numbers of --study tgv (default 1e-1,...,1e-6) or machsweep (1e-2,1e-4,1e-6)")
    ap.add_argument("--decay", action="store_true", help="--study tgv: decay run to t = 20")
    ap.add_argument("--study-n", type=int, default=None,
                    help="cells per direction of --study tgv (default 64) or machsweep (128)")
    ap.add_argument("--cfl", type=float, default=None, help="--study machsweep: CFL_hydro instead of 1000")
    ap.add_argument("--ref-n", type=int, default=64,
                    help="cells per direction of the oracle step of --impl reference")
    ap.add_argument("--cpu-n", type=int, default=64,
                    help="cells per direction of the oracle step of cpu_baseline")
    ap.add_argument("--oracle-reps", type=int, default=3,
                    help="cpu_baseline: oracle residual and Jv calls at full size, all threads")
    ap.add_argument("--no-oracle-kernels", action="store_true",
                    help="cpu_baseline without the full-size oracle residual and Jv timings")
    ap.add_argument("--no-oracle-1thread", action="store_true",
                    help="cpu_baseline without the single-thread full-size oracle timings")
    ap.add_argument("--sweep", action="store_true", help="--study tgv: GMRES iterations against CFL_hydro")
    args = ap.parse_args()
    if args.eta is not None:
        global ETA
        ETA = args.eta
    for k in ("mg_cycles", "mg_nu1", "mg_nu2", "pc_freeze", "lam"):
        if getattr(args, k) is not None:
            OPT_OVERRIDES[k] = getattr(args, k)
            CLI_OPTS[k] = getattr(args, k)
    if args.study == "tgv":
        study_tgv(args)
        return
    if args.study in ("vortex", "params"):
        study_vortex(args)
        return
    if args.study == "inner":
        study_inner(args)
        return
    if args.study == "adjoint":
        study_adjoint(args)
        return
    if args.study == "machsweep":
        study_machsweep(args)
        return
    if args.study == "newton":
        study_newton(args)
        return
    if args.only:
        kernel_main(args)
        return
    if args.warmup < 3:
        args.warmup = 3

    ws, rank, local = dist_init()
    if args.impl == "reference":
        reference_main(args, ws, rank)
        return

    import torch
    from paper_1512_03662_gb300 import build as B
    B.build()
    import paper_1512_03662_gb300 as jf

    device = torch.device(f"cuda:{local}")
    torch.cuda.set_device(device)
    stream = torch.cuda.Stream(device)
    wl = make_workload(args.n)
    peaks = load_peaks()
    probe = {"error": "skipped (--no-probe)"}
    if not args.no_probe:
        try:
            probe = fp64_probe(device, stream)
        except (OSError, RuntimeError) as e:
            probe = {"error": str(e)}

    clocks = ClockSampler(local)
    barrier(ws)
    clocks.start()
    S, X0, dt, ms_mixed, st_mixed, X_mixed = run_arm(jf, wl, jf.MIXED, args.steps, args.warmup, device, stream, True)
    so = S.options
    solver_cfg = {"newton_tol": NEWTON_TOL, "eta": ETA, "gmres_m": so.gmres_m, "precond": so.precond,
                  "mg_cycles": so.mg_cycles, "mg_nu1": so.mg_nu1, "mg_nu2": so.mg_nu2, "pc_freeze": so.pc_freeze}
    barrier(ws)
    clk = clocks.stop()
    ms_mixed = max_over_ranks(ws, ms_mixed)
    conv = {"mixed": convergence(st_mixed)}

    # the end-to-end arm right after the device arm, under the same conditions
    # (before the FP64 arm heats the GPU), with its own clock record
    e2e = None
    if not args.no_e2e:
        clocks_e2e = ClockSampler(local)
        barrier(ws)
        clocks_e2e.start()
        ms_e2e, nbytes, st_e2e = e2e_arm(jf, wl, jf.MIXED, args.steps, args.warmup, device, stream,
                                         None if args.e2e_new_solver else S)
        barrier(ws)
        clk_e2e = clocks_e2e.stop()
        ms_e2e = max_over_ranks(ws, ms_e2e)
        conv["e2e"] = convergence(st_e2e)
        e2e = {"value": ws * args.steps / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "clocks": clk_e2e}

    fp64 = None
    if not args.no_fp64:
        S64, _, _, ms64, st64, X64 = run_arm(jf, wl, jf.FP64, args.steps, args.warmup, device, stream, True)
        conv["fp64"] = convergence(st64)
        # the same steps in both precisions: max over unknowns of |X_mixed - X_fp64| / R(X_fp64)
        _, R64, _ = S64.scaling(X64)
        mixed_vs_fp64 = float(((X_mixed - X64) / R64).abs().max())
        # F(X^{n+1}; X^n) through jfnk_residual per second (each call forms b^n
        # from X^n and G(X^{n+1}): two evaluations of R_U)
        F = torch.empty_like(X64)
        S64.residual(X64, X0, dt, F)
        torch.cuda.synchronize()
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            r0.record(stream)
            for _ in range(5):
                S64.residual(X64, X0, dt, F)
            r1.record(stream)
        torch.cuda.synchronize()
        residual_gcell_s = 5 * wl.ncell / (r0.elapsed_time(r1) / 1e3) / 1e9
        del F, X64, R64
        ms64 = max_over_ranks(ws, ms64)
        fp64 = {"steps_per_s": ws * args.steps / (ms64 / 1e3), "ms_per_step": ms64 / args.steps,
                "newton_per_step": sum(s["newton_iterations"] for s in st64) / len(st64),
                "gmres_per_newton": sum(s["gmres_iterations_total"] for s in st64) /
                max(1, sum(s["newton_iterations"] for s in st64)),
                "jv_gcell_s": None, "residual_gcell_s": residual_gcell_s,
                "mixed_vs_fp64_max_scaled_diff": mixed_vs_fp64}
        jv64 = sum(s["jv_ms"] for s in st64)
        njv64 = sum(s["jv_evaluations"] for s in st64)
        if jv64 > 0:
            fp64["jv_gcell_s"] = njv64 * wl.ncell / (jv64 / 1e3) / 1e9
        del S64

    lam_arm = None
    if args.lam_arm > 0:
        OPT_OVERRIDES["lam"], lam0 = args.lam_arm, OPT_OVERRIDES.get("lam")
        clocks_l = ClockSampler(local)
        clocks_l.start()
        S_l, _, _, ms_l, st_l, X_l = run_arm(jf, wl, jf.MIXED, args.steps, args.warmup, device, stream, False)
        clk_l = clocks_l.stop()
        if lam0 is None:
            del OPT_OVERRIDES["lam"]
        else:
            OPT_OVERRIDES["lam"] = lam0
        conv["mixed_lam_arm"] = convergence(st_l)
        _, R_l, _ = S_l.scaling(X_mixed)
        ms_l = max_over_ranks(ws, ms_l)
        nl = sum(s["newton_iterations"] for s in st_l)
        lam_arm = {"lam": args.lam_arm, "steps_per_s": ws * args.steps / (ms_l / 1e3),
                   "ms_per_step": ms_l / args.steps, "newton_per_step": nl / len(st_l),
                   "gmres_per_newton": sum(s["gmres_iterations_total"] for s in st_l) / max(1, nl),
                   "max_scaled_diff_vs_headline": float(((X_l - X_mixed) / R_l).abs().max()),
                   "clocks": clk_l}
        del S_l, X_l, R_l

    steps_per_s = ws * args.steps / (ms_mixed / 1e3)
    njv = sum(s["jv_evaluations"] for s in st_mixed)
    jv_ms = sum(s["jv_ms"] for s in st_mixed)
    kms = [sum(s["jv_kernel_ms"][q] for s in st_mixed) for q in range(5)]
    launches = sum(s["kernel_launches"] for s in st_mixed)
    dom = max(range(5), key=lambda q: kms[q])
    name = JV_KERNELS[dom]
    per_launch_ms = kms[dom] / max(1, njv)
    flops = FP64_FLOPS_PER_CELL[name] * wl.ncell
    achieved_tflops = flops / (per_launch_ms / 1e3) / 1e12
    tinst = FP64_INST_PER_CELL[name] * wl.ncell / (per_launch_ms / 1e3) / 1e12
    hbm_gbs = HBM_BYTES_PER_CELL[name] * wl.ncell / (per_launch_ms / 1e3) / 1e9
    scale = wl.ncell / 128 ** 3
    stale = kernel_source_hash() != KERNEL_COUNTS_HASH
    if "tinst_s" in probe:
        peak_tinst, peak_tflops = probe["tinst_s"], probe["tflops"]
        peak_src = (f"measured: DFMA probe (libfp64probe.so, {probe['sms']} SMs x 8 blocks x 256 threads, "
                    f"8 independent chains), best of {probe['launches']} launches, median SM clock "
                    f"{probe['clocks'].get('sm_mhz')} MHz")
    else:
        peak_tinst, peak_tflops = FP64_PEAK_TINST, FP64_PEAK_TFLOPS
        peak_src = "derived: 152 SMs x 2 FP64 inst/clk x 2.07 GHz (probe failed)"
    ops_rate = (FP64_INST_PER_CELL[name] + INT_PIPE_OPS_PER_CELL[name]) * wl.ncell / (per_launch_ms / 1e3) / 1e12
    # the whole Jacobian-free product: FP64 instructions of its five kernels
    # over their summed device time
    jv_inst = sum(FP64_INST_PER_CELL[k] for k in JV_KERNELS) * wl.ncell * njv
    jv_tinst = jv_inst / (jv_ms / 1e3) / 1e12 if jv_ms > 0 else None
    # The kernel is bound by the FP64 pipe, which issues one DADD, DMUL or DFMA
    # per lane slot whatever its flop count, so the roofline is stated in FP64
    # instructions per second against the measured issue rate; the flop rate
    # (DFMA = 2) is reported beside it.  The products the kernel forms on the
    # integer pipes do not occupy the FP64 pipe: "fp64_ops_rate" counts them
    # with the FP64-pipe arithmetic, which is why it can exceed the FP64 pipe's
    # own peak ("ops_vs_fp64_peak").
    roofline = {"bound": "alu", "kernel": f"k_{name}", "achieved": tinst, "peak": peak_tinst,
                "unit": "T FP64 inst/s", "frac": tinst / peak_tinst,
                "traffic": None if stale else DRAM_BYTES_PER_CELL_128[name] * 128 ** 3 * scale,
                "traffic_note": "ncu DRAM bytes of a 128^3 launch scaled by the cell ratio",
                "peak_src": peak_src, "counts_stale": stale, "counts_hash": KERNEL_COUNTS_HASH,
                "fp64_inst_per_cell": FP64_INST_PER_CELL[name],
                "fp64_pipe_inst_per_cell": FP64_PIPE_INST_PER_CELL[name],
                "int_pipe_ops_per_cell": INT_PIPE_OPS_PER_CELL[name],
                "fp64_ops_rate": ops_rate, "ops_vs_fp64_peak": ops_rate / peak_tinst,
                "pipe_frac": FP64_PIPE_INST_PER_CELL[name] * wl.ncell / (per_launch_ms / 1e3) / 1e12 / peak_tinst,
                "achieved_tflops": achieved_tflops, "peak_tflops": peak_tflops,
                "frac_tflops": achieved_tflops / peak_tflops,
                "hbm_gbs": hbm_gbs, "hbm_frac": hbm_gbs / peaks["hbm_gbs"], "hbm_peak_src": peaks["src"],
                "algorithmic_bytes_per_cell": HBM_BYTES_PER_CELL[name],
                "jv_whole": {"fp64_inst_per_cell": sum(FP64_INST_PER_CELL[k] for k in JV_KERNELS),
                             "int_pipe_ops_per_cell": sum(INT_PIPE_OPS_PER_CELL[k] for k in JV_KERNELS),
                             "achieved": jv_tinst, "frac": jv_tinst / peak_tinst if jv_tinst else None,
                             "ms_per_product": jv_ms / max(1, njv)}}

    cpu = None
    if rank == 0 and not args.no_cpu:
        import torch as _t
        oracle_sample(16, 1)                                  # first-call overheads of the oracle
        s_step, threads, st_small = oracle_sample(args.cpu_n, 1, with_stats=True)
        v = (args.cpu_n / args.n) ** 3 / s_step
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"one oracle implicit step at {args.cpu_n}^3 (same construction and dt, same solver "
                         f"settings) took {s_step:.1f} s with {threads} threads; value = its rate x "
                         f"({args.cpu_n}/{args.n})^3",
               "step_small": {"n": args.cpu_n, "seconds": s_step, **st_small},
               "host": cpu_info()}
        if not args.no_oracle_kernels:
            cpu["kernels_at_full_size"] = [oracle_kernels(wl, _t.get_num_threads(), args.oracle_reps)]
            if not args.no_oracle_1thread:
                cpu["kernels_at_full_size"].append(oracle_kernels(wl, 1, 1))

    if rank == 0:
        line = {"metric": METRIC, "value": steps_per_s, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_mixed / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64 residual / f32 Krylov",
                "data": "synthetic",
                "config": {"workload": f"convbox3d {args.n}^3 (problem 4), CFL_hydro {wl.cfl_hydro:g}, "
                                       f"dt {dt:.4g}",
                           "parallelism": "replicas" if ws > 1 else "single",
                           "l2": "state (670 MB/vector) larger than L2, no flush", "solver": solver_cfg},
                "convergence": conv,
                "jv_gcell_s": njv * wl.ncell / (jv_ms / 1e3) / 1e9 if jv_ms > 0 else None,
                "newton_per_step": sum(s["newton_iterations"] for s in st_mixed) / len(st_mixed),
                "gmres_per_newton": sum(s["gmres_iterations_total"] for s in st_mixed) /
                max(1, sum(s["newton_iterations"] for s in st_mixed)),
                "fp64": fp64, "lambda_arm": lam_arm, "roofline": roofline, "fp64_probe": probe,
                "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk,
                "jv_kernel_ms_per_launch": {JV_KERNELS[q]: kms[q] / max(1, njv) for q in range(5)},
                "precond_ms_per_apply": sum(s["precond_ms"] for s in st_mixed) /
                max(1, sum(s["precond_applies"] for s in st_mixed)),
                "ortho_ms_per_iteration": sum(s["ortho_ms"] for s in st_mixed) / max(1, njv)}
        print(json.dumps(line), flush=True)
    # a rate is only claimed for steps that met the Newton tolerance
    if any(c["newton_capped"] for c in conv.values()):
        sys.stderr.write(f"bench: timed steps stopped without meeting the Newton tolerance: {conv}\n")
        sys.exit(3)


if __name__ == "__main__":
    main()

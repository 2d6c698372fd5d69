#!/usr/bin/env python
"""Benchmark of the space-time multigrid V-cycle (arXiv 1911.09548) on one GB300.

Workload (one "step" = one V-cycle, i.e. every step of the hot path: residuals,
block-Jacobi slab solves, nodal auxiliary-space corrections, time transfers,
coarsest solve, residual norm): Kuhn mesh of 16^3 cubes (26416 interior edges),
nu = 1e-3 in [0.25, 0.75]^3 and 1 outside, sigma log-uniform in [0.1, 10] per tet
(seed 0), T = 1, N_t = 256 slabs, DG(1) in time, V(2,2) with the hybrid smoother
SSASS, omega = 0.5, time coarsening on every level (the coarsening rule never
admits space coarsening here), 9 time levels.  Inputs are synthetic (st_inputs).

Metric: space-time DoFs smoothed per second = fine-level DoFs x fine-level S
applications per V-cycle (2 nu_pre + 2 nu_post = 8) x V-cycles / time; also the
time to a 1e-8 relative residual from x = 0 (p50/p99 over seeds).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun as N independent replicas (one excitation each).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="kuhn16_dg1_Nt256_V22", n=16, N_t=256, degree=1, T=1.0, nu_pre=2, nu_post=2,
                materials="two_material", seed=0)
METRIC = "space-time DoFs smoothed/s"
UNIT = "DoF/s"
CPU_SAMPLE_SLABS = 16
# DRAM bytes (read + write) of the supernodal products of one finest-level FP64 slab solve of
# this workload, from one ncu capture of the same kernels and factor; set to None when those
# kernels or the factor they read change
SLAB_SOLVE_TRAFFIC_FP64 = 2.396e9


def workload_config(world: int = 1) -> dict:
    """The workload as the bench line names it (both arms)."""
    W = WORKLOAD
    return {"workload": W["name"], "mesh": "Kuhn 16^3, 26416 interior edges", "N_t": W["N_t"],
            "degree": W["degree"], "cycle": "V(2,2) SSASS, omega 0.5", "materials": W["materials"],
            "dofs": 26416 * W["N_t"] * (W["degree"] + 1), "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (129 MB): f, x and r 108 MB each, slab factors read in every V-cycle"}


def smoothed_per_cycle(dofs, nu_pre, nu_post):
    return dofs * (2 * nu_pre + 2 * nu_post)


def measured_peak(key: str) -> float:
    """Measured peak of this machine's GB300 (MEASURED_PEAKS.json); 1938.7 TFLOP/s
    BF16 / 6794.5 GB/s HBM, the values measured for this machine, if the file is absent."""
    fallback = {"bf16_tflops": 1938.7, "hbm_gbs": 6794.5}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key])
    except (OSError, KeyError, ValueError):
        return fallback[key]


# FP32 FMA rate of the GB300, from its unit counts: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def roofline_of(slab_prec: int, achieved: float, fp64_peak: float, slab_ms: float) -> dict:
    """Roofline object of the finest-level slab solve for the arithmetic it runs in."""
    counts = "algorithmic flop: 8 per complex multiply-add of the factor"
    if slab_prec == 3:
        peak = measured_peak("bf16_tflops")
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "supernodal slab solve, finest level, BF16 on the tensor cores "
                "(k_tc_assemble, k_sn_tc3 on tiled depths, k_sn_tc2 + k_sn_tc_reduce on split-K ones)",
                "achieved_counts": counts + " (4 real BF16 ones)",
                "peak_source": "measured dense BF16 peak (MEASURED_PEAKS.json)", "ms_per_launch_group": slab_ms}
    if slab_prec in (1, 2):
        return {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                "kernel": "supernodal slab solve, finest level, %s on the FP32 pipes (k_sn_forward/backward, split-K "
                "near the root)" % ("FP32" if slab_prec == 1 else "double-float"), "achieved_counts": counts,
                "peak_source": "FP32 FMA rate from unit counts and clock (152 SMs x 128 lanes x 2 flop x 2.07 GHz)",
                "ms_per_launch_group": slab_ms}
    return {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
            "traffic": SLAB_SOLVE_TRAFFIC_FP64,
            "kernel": ("supernodal slab solve, finest level (k_sn_forward/backward, split-K near the "
                       "root; complex products with three real multiplications)"),
            "achieved_counts": counts,
            "peak_source": "FP64 FMA throughput measured in this run (st_mg_probe_fp64)",
            "ms_per_launch_group": slab_ms}


def percentile99(values):
    """99th percentile by the nearest rank of the sorted sample."""
    v = sorted(values)
    return v[min(len(v) - 1, int(round(0.99 * (len(v) - 1))))]


def reduce_max(value: float, dist=None, device="cpu") -> float:
    """Max over ranks (the slowest replica sets the job's time)."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, per_cycle: float, steps: int, ms_max: float) -> float:
    """Whole-job throughput: every replica smooths per_cycle DoFs per step."""
    return world * per_cycle * steps / (ms_max / 1e3)


# ------------------------------------------------------------------ CPU oracle leg
def _oracle_setup(seed: int = 0):
    """The oracle's finest-level slab operator of the workload (16^3, DG(1), tau = 1/256:
    SciPy SuperLU factor of the real block slab matrix) and its load; run in a process
    that never touches CUDA."""
    import st_inputs
    from oracle.load import spacetime_load
    from oracle.spacetime import SlabOperator, build_space_hierarchy

    W = WORKLOAD
    nu, sigma = st_inputs.materials(W["n"], W["materials"], W["seed"])
    sl = build_space_hierarchy(W["n"], 1, nu, sigma)
    t0 = time.time()
    slab = SlabOperator(sl[0], W["degree"], W["T"] / W["N_t"])
    t_setup = time.time() - t0
    f = spacetime_load(sl[0].mesh, st_inputs.excitation(seed), W["degree"], W["N_t"], W["T"])
    return slab, f, t_setup


def _sweep_worker(slab, f, reps, barrier, q):
    """One forked worker: `reps` oracle block-Jacobi sweeps S on its slabs, timed."""
    import numpy as np

    from oracle.spacetime import smoother_S
    x = np.zeros_like(f)
    barrier.wait(timeout=600)
    t_start = time.perf_counter()
    times = []
    for _ in range(reps):
        a = time.perf_counter()
        x = smoother_S(slab, f, x, 0.5)
        times.append(time.perf_counter() - a)
    q.put((times, t_start, time.perf_counter()))


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_parallel(nslabs: int, reps: int, workers: int, go=None):
    """The oracle as it stands on `workers` host cores: the slab factor is built once
    (factorisation excluded from the timing), then `workers` forked single-threaded
    processes each run `reps` sweeps S on their own `nslabs`-slab sample of the finest
    level (slabs w*nslabs ... of the 256, wrapping), started together behind a barrier.
    `go` (an Event) delays the timed sweeps, e.g. until a GPU measurement has ended.
    Returns the per-worker sweep times and the wall time of the parallel section."""
    import multiprocessing as mp

    slab, f, t_setup = _oracle_setup()
    if go is not None:
        go.wait()
    ctx = mp.get_context("fork")      # this process has no CUDA context: forking it is safe
    q = ctx.Queue()
    bar = ctx.Barrier(workers)
    nt = f.shape[0]
    procs = []
    for w in range(workers):
        idx = [(w * nslabs + j) % nt for j in range(nslabs)]
        procs.append(ctx.Process(target=_sweep_worker, args=(slab, f[idx].copy(), reps, bar, q), daemon=True))
    for pr in procs:
        pr.start()
    res = [q.get(timeout=1800) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    dofs = nslabs * f.shape[1] * f.shape[2]
    return {"times": [r[0] for r in res], "wall_s": wall, "dofs_per_sweep": dofs, "setup_s": t_setup,
            "workers": workers}


def _oracle_leg(q, go, nslabs, reps, workers):
    # one thread per worker: no BLAS or OpenMP thread pools inside the forked workers
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    try:
        q.put(oracle_parallel(nslabs, reps, workers, go))
    except Exception as e:  # reported, never silently dropped
        q.put({"error": repr(e)})


def cpu_baseline_desc(res, nslabs, skip=0):
    """Throughput of the oracle sample: all workers' timed sweeps over the wall time of
    the parallel section (the first `skip` sweeps of each worker untimed)."""
    n_w = res["workers"]
    sweeps = [t[skip:] for t in res["times"]]
    per_worker_s = [sum(t) for t in sweeps]
    n_sweeps = sum(len(t) for t in sweeps)
    value = res["dofs_per_sweep"] * n_sweeps / max(per_worker_s)
    return {"value": value, "unit": UNIT, "cores": n_w, "kind": "oracle",
            "sample": (f"{n_w} single-threaded oracle processes (one per host core), each running "
                       f"{len(sweeps[0])} block-Jacobi sweeps S on its own {nslabs} of the 256 slabs of the "
                       f"16^3 DG(1) finest level ({res['dofs_per_sweep']} DoFs per sweep; SciPy SuperLU slab "
                       f"solve and sparse products); factorisation ({res['setup_s']:.0f} s) excluded; timed "
                       f"after the GPU measurement, with the GPU idle"),
            "sweep_s_median": statistics.median(x for t in sweeps for x in t)}


def run_reference(args):
    """Reference arm: the oracle, as it stands, on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    workers = min(host_cores(), 32)
    res = oracle_parallel(CPU_SAMPLE_SLABS, args.warmup + args.steps, workers)
    base = cpu_baseline_desc(res, CPU_SAMPLE_SLABS, skip=args.warmup)
    value = base["value"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * base["sweep_s_median"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(), "impl": "reference", "cpu_baseline": base,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ precision (config 3)
def run_precision(args):
    """The mixed-precision workload: Kuhn 16^3, two materials, T = 1, N_t = 1024, DG(1),
    V(2,2), solved to a 1e-8 relative residual with the slab factor in FP64, FP32 and BF16
    (tensor cores); V-cycle counts, times, and the relative error of each final solution
    against the FP64 one."""
    import torch

    torch.cuda.set_device(0)
    from paper_1911_09548_gb300._build import build
    build()
    import paper_1911_09548_gb300 as stmg
    import st_inputs

    n, N_t = 16, 1024
    nu, sigma = st_inputs.materials(n, "two_material", 0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    rows, ref = {}, None
    for name, prec in (("fp64", 0), ("fp32", 1), ("bf16_tensor", 3), ("fp16_tensor", 4)):
        S = stmg.SpaceTimeSolver(n, nu, sigma, 1.0, N_t, 1, nu_pre=2, nu_post=2, stream=stream.cuda_stream,
                                 slab_prec=prec, autotune=args.autotune)
        f = S.load(st_inputs.excitation(0))
        x = S.zeros()
        S.solve(f, x, rtol=1e-8, maxit=60)          # warm-up (graph capture), discarded
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = S.solve(f, x, rtol=1e-8, maxit=60)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if ref is None:
            ref = x.clone()
        err = float(torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref))
        rows[name] = {"time_to_1e-8_s": dt, "v_cycles": out["iters"], "rel_res": out["rel_res"],
                      "ms_per_v_cycle": 1e3 * dt / max(out["iters"], 1), "rel_err_vs_fp64_solution": err}
        S.close()
    print(json.dumps({"mode": "precision", "metric": "time to 1e-8 relative residual, mixed vs FP64",
                      "config": {"mesh": "Kuhn 16^3, 26416 interior edges", "N_t": N_t, "degree": 1,
                                 "dofs": 26416 * N_t * 2, "cycle": "V(2,2)", "materials": "two_material",
                                 "autotune": bool(args.autotune)},
                      "results": rows}))
    return 0


# ------------------------------------------------------------------ memory-bound steps
def run_kernels(args):
    """Each memory-bound step of the hot path alone, on the workload's finest level
    (16^3, DG(1), N_t = 256: 13.5 M space-time DoFs), through the C ABI: time with CUDA
    events on the bench's stream, L2 flushed (a 512 MB write) before every repetition,
    against the step's algorithmic bytes (what it must read and write once).  The
    NVTX range "kernels" brackets the last repetition of every step (for a profiler)."""
    import torch

    torch.cuda.set_device(0)
    from paper_1911_09548_gb300._build import build
    build()
    import paper_1911_09548_gb300 as stmg
    import st_inputs

    stmg.st_mg_set_launch_overlap(args.launch_overlap)
    W = WORKLOAD
    nu, sigma = st_inputs.materials(W["n"], W["materials"], W["seed"])
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    S = stmg.SpaceTimeSolver(W["n"], nu, sigma, W["T"], W["N_t"], W["degree"], nu_pre=W["nu_pre"],
                             nu_post=W["nu_post"], stream=stream.cuda_stream, slab_prec=args.slab_prec)
    ne, nn, q, N_t = S.n_edge, S.n_node, S.q, W["N_t"]
    ncols = N_t * q
    nnz = int(stmg.st_mg_debug_get(S.h, 5, 0).size)
    f = S.load(st_inputs.excitation(0))
    gen = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand(S.level_shape(), dtype=torch.float64, device="cuda", generator=gen)
    r = S.zeros()
    y = S.zeros(nodal=True)
    z = torch.rand(S.level_shape(nodal=True), dtype=torch.float64, device="cuda", generator=gen)
    wv = S.zeros(nodal=True)
    rc = S.zeros(1)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device="cuda")
    B = stmg
    dof, ndof = ne * ncols, nn * ncols
    steps = {
        # name: (call, algorithmic bytes)
        "residual (r = f - L x)": (lambda: B.st_mg_residual(S.h, 0, f, x, r),
                                   24 * dof + 8 * (ne + 1) + nnz * (4 + 8 * (3 if W["degree"] == 1 else 2))),
        "G^T r": (lambda: B.st_mg_grad_T(S.h, 0, r, y), 8 * dof + 8 * ndof + 8 * (nn + 1) + 5 * 2 * ne),
        "time integration L_t^-1": (lambda: B.st_mg_time_integrate(S.h, 0, z, wv), 16 * ndof),
        "x += G w": (lambda: B.st_mg_grad_add(S.h, 0, wv, x), 16 * dof + 8 * ndof + 8 * ne),
        "time restriction": (lambda: B.st_mg_restrict(S.h, 0, r, rc), 8 * dof + 4 * dof),
        "time prolongation-add": (lambda: B.st_mg_prolong_add(S.h, 0, rc, x), 4 * dof + 16 * dof),
    }
    peak = measured_peak("hbm_gbs")
    rows = {}
    for name, (call, nbytes) in steps.items():
        call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for rep in range(args.steps):
            flush.zero_()
            if rep == args.steps - 1:
                torch.cuda.nvtx.range_push("kernels")
            e0.record(stream)
            call()
            e1.record(stream)
            torch.cuda.synchronize()
            if rep == args.steps - 1:
                torch.cuda.nvtx.range_pop()
            ms.append(e0.elapsed_time(e1))
        t = statistics.median(ms)
        gbs = nbytes / (t / 1e3) / 1e9
        rows[name] = {"us": 1e3 * t, "algorithmic_MB": nbytes / 1e6, "GB_s": gbs, "frac_of_hbm": gbs / peak}
    S.close()
    print(json.dumps({"mode": "kernels", "workload": W["name"], "slab_prec": args.slab_prec,
                      "hbm_peak_gbs": peak, "timing": "median of %d, CUDA events, L2 flushed before each" % args.steps,
                      "steps": rows}))
    return 0


# ------------------------------------------------------------------ convergence rates
def run_rates(args):
    """Two-grid convergence rates by the power iteration of Section 5.1 on the GPU:
    'Semi-time' (time coarsening only) and 'Full' (space and time) against lambda of eq.
    CoarseningRule (the paper's experiment E1 on the Kuhn cube 16^3 -> 8^3, DG(0),
    nu = sigma = 1, N_t = 16, lambda varied through tau; Dirichlet and, as in the
    paper's experiment, Neumann boundaries), then hybrid-smoother orderings (Section 4)
    at a small and a large lambda."""
    import torch

    torch.cuda.set_device(0)
    from paper_1911_09548_gb300._build import build
    build()
    import paper_1911_09548_gb300 as stmg
    import st_inputs

    nf, N_t = 16, 16
    nu, sigma = st_inputs.materials(nf, "unit")
    h2 = 3.0 / nf ** 2

    def rate(tau, bc=0, **opts):
        S = stmg.SpaceTimeSolver(nf, nu, sigma, tau * N_t, N_t, 0, n_space_levels=2, max_levels=2, bc=bc, **opts)
        x = torch.from_numpy(st_inputs.random_iterate((S.n_edge, N_t), 0)).cuda()
        r, _ = S.convergence_rate(x, max_iter=15)
        S.close()
        return r

    sweep = []
    for k in range(-12, 3, 2):
        tau = 2.0 ** k
        row = {"tau": tau, "lambda": tau / h2}
        for bc, name in ((0, "dirichlet"), (1, "neumann")):
            row[name] = {"semi_time": rate(tau, coarsen=1, bc=bc), "full": rate(tau, coarsen=2, bc=bc)}
        sweep.append(row)
    orderings = {}
    for tau in (2.0 ** -8, 1.0):
        orderings[f"lambda={tau / h2:.3g}"] = {p: rate(tau, coarsen=1, smoother=p)
                                                for p in ("SAS", "SA", "AS", "SSA", "ASS", "SSAS", "SSASS")}
    print(json.dumps({"mode": "rates", "metric": "two-grid convergence rate (power iteration, Section 5.1)",
                      "config": {"mesh": "Kuhn 16^3 -> 8^3", "degree": 0, "N_t": 16, "materials": "nu = sigma = 1",
                                 "cycle": "two-grid, SAS unless stated"},
                      "lambda_sweep": sweep, "orderings_semi_time": orderings}))
    return 0


# ------------------------------------------------------------------ serving
SERVE_SPACE_LEVELS = {4: 2, 8: 2, 16: 3, 24: 3}
SERVE_EDGES = {4: 316, 8: 3032, 16: 26416, 24: 91656}   # interior edges of the Kuhn meshes


def run_serve(args):
    """Request-loop benchmark: Poisson streams of solve requests over several meshes,
    N_t, DG degrees and conductivity scales (st_inputs.request_stream), each solved to
    a 1e-8 relative residual by the library's server (continuous batching, factor
    cache, mixed-precision slab apply).  Latency = completion (solution on the host)
    - arrival.  A warm-up pass first builds every class the streams use (factorisations
    excluded from latencies; classes stay resident while the memory budget allows)."""
    import numpy as np
    import torch

    torch.cuda.set_device(0)
    from paper_1911_09548_gb300._build import build
    build()
    import paper_1911_09548_gb300 as stmg
    import st_inputs

    rates = [float(v) for v in args.serve_rates.split(",")]
    meshes = [24] if args.serve_burst > 0 else [int(v) for v in args.serve_meshes.split(",")]
    nt_lo, nt_hi = (int(v) for v in args.serve_nt.split(","))
    nu_c = 2
    srv = stmg.SpaceTimeServer(slots=args.serve_slots, slab_prec=args.serve_prec, nu=nu_c, max_cycles=60)
    for n in meshes:
        srv.register(n, SERVE_SPACE_LEVELS[n], *st_inputs.materials(n, "two_material", 0))
    if args.serve_burst > 0:
        # every request arrives at once (offered rate: unbounded)
        rates = [float("inf")]
        burst = st_inputs.request_stream(args.serve_burst, 1e9, seed=7, meshes=(24,), nt_range=(128, 1024),
                                         degrees=(1,))
        for q in burst:
            q["t"], q["sigma_scale"] = 0.0, 1.0
        streams = [burst]
    else:
        streams = [st_inputs.request_stream(args.serve_requests, r, seed=i, meshes=meshes, nt_range=(nt_lo, nt_hi))
                   for i, r in enumerate(rates)]

    def submit(q, t_arr=0.0):
        return srv.submit(q["n_cube"], q["degree"], q["N_t"], 1.0 / q["N_t"], q["sigma_scale"],
                          st_inputs.excitation(q["seed"] % 100000), 1e-8, t_arr)

    # warm-up: one request per class (mesh, degree, N_t, tau / s)
    t0 = time.monotonic()
    seen = {}
    for st_ in streams:
        for q in st_:
            seen.setdefault((q["n_cube"], q["degree"], q["N_t"], q["N_t"] * q["sigma_scale"]), q)
    for q in seen.values():
        submit(q)
    srv.run_until_idle()
    warm_s = time.monotonic() - t0
    stw = srv.stats()

    rows = []
    for rate, stream in zip(rates, streams):
        s0 = srv.stats()
        lat, cyc, bad = [], [], 0
        i, done, max_q = 0, 0, 0
        t_start = time.monotonic()
        while done < len(stream):
            now = time.monotonic()
            while i < len(stream) and t_start + stream[i]["t"] <= now:
                submit(stream[i], t_start + stream[i]["t"])
                i += 1
            st_ = srv.stats()
            max_q = max(max_q, st_["queued"])
            if st_["queued"] + st_["active"] + st_["building"] == 0:
                if i < len(stream):
                    time.sleep(max(0.0, t_start + stream[i]["t"] - time.monotonic()))
                continue
            for rid in srv.step():
                r = srv.result(rid, want_x=False)
                lat.append(r["t_done"] - r["t_arrival"])
                cyc.append(r["cycles"])
                bad += r["status"] != 0
                done += 1
        dur = time.monotonic() - (t_start + stream[0]["t"])
        n_dofs = sum(SERVE_EDGES.get(q["n_cube"], 0) * q["N_t"] * (q["degree"] + 1) for q in stream)
        s1 = srv.stats()
        lat_s = sorted(lat)
        smoothed = (s1["dofs_smoothed"] - s0["dofs_smoothed"]) * 4 * nu_c
        rows.append({"offered_req_per_s": rate if rate != float("inf") else "all at t = 0",
                     "requests": len(stream), "duration_s": dur, "space_time_dofs": n_dofs,
                     "throughput_req_per_s": len(stream) / dur, "dofs_smoothed_per_s": smoothed / dur,
                     "latency_p50_s": float(np.percentile(lat_s, 50)), "latency_p99_s": float(np.percentile(lat_s, 99)),
                     "latency_max_s": lat_s[-1], "v_cycles_mean": float(np.mean(cyc)), "not_converged": bad,
                     "max_queue": max_q, "evictions": s1["evictions"] - s0["evictions"],
                     "deferrals": s1["deferrals"] - s0["deferrals"]})
    stf = srv.stats()
    srv.close()
    line = {"metric": "served solves to 1e-8 relative residual: throughput and p50/p99 latency", "unit": "s",
            "mode": "serve", "data": "synthetic",
            "config": {"meshes": meshes, "burst": args.serve_burst,
                       "N_t": (f"powers of two in [{nt_lo}, {nt_hi}]" if args.serve_burst == 0 else
                               "uniform over {128, 256, 512, 1024}"),
                       "degrees": [0, 1] if args.serve_burst == 0 else [1],
                       "sigma_scale": "log-uniform [0.1, 10] rounded to a power of two", "tau": "1 / N_t",
                       "slots_per_class": args.serve_slots, "slab_prec": args.serve_prec,
                       "cycle": f"V({nu_c},{nu_c})", "rtol": 1e-8,
                       "latency": "arrival to solution on the host (pageable copy)"},
            "warmup": {"classes": len(seen), "seconds": warm_s, "cache_entries": stw["cache_entries"],
                       "cache_bytes": stw["cache_bytes"], "cache_hits": stw["cache_hits"],
                       "cache_misses": stw["cache_misses"]},
            "rates": rows,
            "final": {"classes": stf["classes"], "class_bytes": stf["class_bytes"], "cache_bytes": stf["cache_bytes"]}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--solves", type=int, default=5, help="FP64 time-to-1e-8 solves (seeds) for p50/p99")
    ap.add_argument("--mixed-solves", type=int, default=20,
                    help="time-to-1e-8 solves (seeds) of each mixed-precision path for p50/p99")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--mixed", type=int, default=1, help="also measure the mixed-precision slab solve")
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="tiled / split-K thresholds chosen per level by timing at setup")
    ap.add_argument("--split-waves", default="",
                    help="comma-separated tiled / split-K threshold per time level, set after setup "
                         "(repeats an autotuned run's choice, e.g. under a profiler)")
    ap.add_argument("--split-k", type=int, default=0,
                    help="K columns of a split-K work item (0: the library default)")
    ap.add_argument("--tc-split-k", type=int, default=0,
                    help="complex K columns of a tensor-core split-K item (0: the library default)")
    ap.add_argument("--nd-leaf", type=int, default=0,
                    help="largest leaf of the slab matrices' nested dissection (0: the library default)")
    ap.add_argument("--launch-overlap", type=int, default=0, choices=[0, 1],
                    help="programmatic dependent launch of the library's kernels (st_mg_set_launch_overlap)")
    ap.add_argument("--config1-seeds", type=int, default=100,
                    help="excitations of the 4^3 DG(0) two-grid case solved to 1e-10 (0: skip)")
    ap.add_argument("--precision-line", type=int, default=1,
                    help="also time the 16^3, N_t = 1024 workload to 1e-8 in every slab arithmetic")
    ap.add_argument("--ragged", type=int, default=8,
                    help="excitations of the ragged-batch variant (N_t from {128, 256, 512, 1024}; 0: skip)")
    ap.add_argument("--batch", type=int, default=8,
                    help="problems per handle of the batched BF16 variant (0: skip it)")
    ap.add_argument("--slab-prec", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="slab-solve arithmetic of the main line: 0 FP64, 1 FP32, 2 double-float, 3 BF16 tensor "
                         "cores, 4 FP16 tensor cores")
    ap.add_argument("--residual-prec", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="residual arithmetic of the main line (st_mg_options.residual_prec)")
    ap.add_argument("--tc-mode", type=int, default=0, choices=[0, 1, 2],
                    help="tensor-core mode of every 16-bit level of the main line (st_mg_set_tc_mode)")
    ap.add_argument("--mode", default="bench", choices=["bench", "slab", "serve", "rates", "precision", "kernels"],
                    help="slab: set up the workload, run two finest-level slab solves and exit (for profilers); "
                         "serve: the request-loop benchmark (Poisson streams, p50/p99 latency)")
    ap.add_argument("--serve-rates", default="0.5,2,10", help="offered request rates (req/s), one stream each")
    ap.add_argument("--serve-requests", type=int, default=24, help="requests per rate")
    ap.add_argument("--serve-meshes", default="8,16,24")
    ap.add_argument("--serve-nt", default="64,2048", help="N_t range (powers of two)")
    ap.add_argument("--serve-slots", type=int, default=2)
    ap.add_argument("--serve-prec", type=int, default=3, choices=[0, 1, 2, 3, 4])
    ap.add_argument("--serve-burst", type=int, default=0,
                    help="instead of Poisson streams: this many requests at once on the 24^3 mesh, N_t uniform "
                         "over {128, 256, 512, 1024}, DG(1) (the batching workload)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "rates":
        return run_rates(args)
    if args.mode == "precision":
        return run_precision(args)
    if args.mode == "kernels":
        return run_kernels(args)

    import multiprocessing as mp

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    # CPU baseline (rank 0, N = 1): a spawned process, started before the first CUDA call,
    # builds the oracle's slab factor while the GPU works and runs its timed sweeps on all
    # host cores only after the GPU measurements have ended (`go`)
    cpu_q = cpu_proc = cpu_go = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.mode == "bench":
        ctx = mp.get_context("spawn")
        cpu_q, cpu_go = ctx.Queue(), ctx.Event()
        cpu_proc = ctx.Process(target=_oracle_leg, args=(cpu_q, cpu_go, CPU_SAMPLE_SLABS, 8,
                                                          min(host_cores(), 32)))
        cpu_proc.start()
    torch.cuda.set_device(local)

    from paper_1911_09548_gb300._build import build
    build()
    import paper_1911_09548_gb300 as stmg
    import st_inputs

    stmg.st_mg_set_launch_overlap(args.launch_overlap)
    W = WORKLOAD
    nu, sigma = st_inputs.materials(W["n"], W["materials"], W["seed"])
    # a dedicated stream: the library captures the V-cycle into a CUDA graph on it
    # (the legacy default stream cannot be captured)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    def make(prec, **kw):
        return stmg.SpaceTimeSolver(W["n"], nu, sigma, W["T"], W["N_t"], W["degree"], nu_pre=W["nu_pre"],
                                    nu_post=W["nu_post"], stream=stream.cuda_stream, slab_prec=prec,
                                    autotune=args.autotune, split_k=args.split_k,
                                    tc_split_k=args.tc_split_k, **kw)

    def time_cycles(Sx, fx, xx, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(args.warmup):
            Sx.vcycle(fx, xx)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            Sx.vcycle(fx, xx)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def time_slab(Sx, fx, xx, reps=3):
        """The dominant kernel group: the finest level's supernodal slab solve (forward
        and backward products of every nested-dissection depth), timed alone with CUDA
        events on the launching stream."""
        r = Sx.residual(fx, xx)
        y = Sx.zeros()
        stmg.st_mg_slab_solve(Sx.h, 0, r, y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            stmg.st_mg_slab_solve(Sx.h, 0, r, y)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def time_solves(Sx, n, maxit, keep=0):
        ms, iters, sols = [], [], []
        for s_ in range(n):
            fs = Sx.load(st_inputs.excitation(100 + s_ + 1000 * rank))
            xs = Sx.zeros()
            torch.cuda.synchronize()
            a = time.perf_counter()
            out = Sx.solve(fs, xs, rtol=1e-8, maxit=maxit)
            torch.cuda.synchronize()
            ms.append(1e3 * (time.perf_counter() - a))
            iters.append(out["iters"])
            if s_ < keep:
                sols.append(xs)
            del fs
        return ms, iters, sols

    def dist_of(ms, iters):
        if not ms:
            return None
        return {"p50": statistics.median(ms) / 1e3, "p99": percentile99(ms) / 1e3, "n": len(ms),
                "p99_rule": "nearest rank of the sorted sample (the maximum when n < 100)", "v_cycles": iters}

    t0 = time.time()
    S = make(args.slab_prec, nd_leaf=args.nd_leaf, residual_prec=args.residual_prec)
    if args.tc_mode and args.slab_prec >= 3:
        for l in range(S.n_levels):
            try:
                stmg.st_mg_set_tc_mode(S.h, l, args.tc_mode)
            except RuntimeError:
                pass   # a level without a 16-bit factor (the coarsest solve is FP64)
    if args.split_waves:
        for l, w in enumerate(int(v) for v in args.split_waves.split(",")):
            stmg.st_mg_set_split_waves(S.h, l, w)
    split_waves = [stmg.st_mg_split_waves(S.h, l) for l in range(S.n_levels)]
    setup_s = time.time() - t0
    n_levels, n_dof = S.n_levels, S.n_dof
    f = S.load(st_inputs.excitation(W["seed"] + rank))
    x = S.zeros()
    per_cycle = smoothed_per_cycle(S.n_dof, W["nu_pre"], W["nu_post"])
    if args.mode == "slab":
        r = S.residual(f, x)
        y = S.zeros()
        stmg.st_mg_slab_solve(S.h, 0, r, y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("slab_solves")   # lets a profiler select these launches
        e0.record(stream)
        for _ in range(2):
            stmg.st_mg_slab_solve(S.h, 0, r, y)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        st = stmg.st_mg_factor_stats(S.h, 0)
        if rank == 0:
            print(json.dumps({"mode": "slab", "slab_prec": args.slab_prec, "nd_leaf": args.nd_leaf,
                              "slab_solve_ms": e0.elapsed_time(e1) / 2, "setup_s": setup_s,
                              "split_waves_per_level": split_waves, **st}))
        S.close()
        return 0

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        S.vcycle(f, x)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    launches0 = stmg.st_mg_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed_vcycles")   # lets a profiler select these launches
    ev0.record(stream)
    for _ in range(args.steps):
        S.vcycle(f, x)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier()
    clk = clocks.stop()
    launches = stmg.st_mg_launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    ms_max = reduce_max(ms, dist, "cuda")
    value = replica_value(world, per_cycle, args.steps, ms_max)

    # dominant kernel: the supernodal slab solve of the finest level, timed alone
    st = stmg.st_mg_factor_stats(S.h, 0)
    least_fill_macs = st["macs_per_rhs"] if (args.nd_leaf in (0, 64) and args.slab_prec != 3) else None
    slab_ms = time_slab(S, f, x)
    flops_per_mac = 8.0 if W["degree"] == 1 else 2.0
    slab_flops = st["macs_per_rhs"] * flops_per_mac * W["N_t"]
    achieved = slab_flops / (slab_ms / 1e3) / 1e12
    fp64_peak = stmg.st_mg_probe_fp64(S.h)       # roof of the FP64 kernels, measured in this run

    # time to 1e-8 from x = 0, several excitations
    solve_ms, solve_iters, fp64_solutions = time_solves(S, args.solves, 60, keep=args.mixed_solves)

    # end to end through the public host-buffer API: H2D of f and x, one V-cycle,
    # residual norms, D2H of x, every step
    fh = torch.empty(S.level_shape(), dtype=torch.float64).pin_memory()
    xh = torch.zeros(S.level_shape(), dtype=torch.float64).pin_memory()
    fh.copy_(f.cpu())
    fnp, xnp = fh.numpy(), xh.numpy()
    if not args.no_e2e:
        S.solve_host(fnp, xnp, rtol=0.0, maxit=1)   # first call allocates the staging buffers
    e2e_times = []
    for _ in range(0 if args.no_e2e else max(1, args.steps)):
        a = time.perf_counter()
        S.solve_host(fnp, xnp, rtol=0.0, maxit=1)
        e2e_times.append(time.perf_counter() - a)
    e2e_value = world * per_cycle * len(e2e_times) / sum(e2e_times) if e2e_times else None
    S.close()
    S = None
    del f, x
    torch.cuda.synchronize()

    # other slab-solve arithmetics on the same workload: double-float (FP64-accurate on the
    # FP32 pipes), FP32 factor, BF16 factor on the tensor cores; each with its V-cycle
    # time, its finest slab solve against its roof, and time to 1e-8 with the error of
    # each solution against the FP64 one of the same excitation
    variants = {}
    if args.mixed:
        for vname, prec, kw in (("double_float", 2, {}), ("mixed_fp32", 1, {}), ("bf16_tensor", 3, {}),
                                ("fp16_tensor", 4, {}), ("bf16_tensor_fp32_residual", 3, {"residual_prec": 1})):
            Sm = make(prec, **kw)
            fm = Sm.load(st_inputs.excitation(W["seed"] + rank))
            xm = Sm.zeros()
            ms_m = reduce_max(time_cycles(Sm, fm, xm, args.steps), dist, "cuda")
            st_m = stmg.st_mg_factor_stats(Sm.h, 0)
            slab_ms_m = time_slab(Sm, fm, xm)
            msolve, miters, sols = time_solves(Sm, args.mixed_solves, 80, keep=len(fp64_solutions))
            merr = [float(torch.linalg.vector_norm(a_ - b_) / torch.linalg.vector_norm(b_))
                    for a_, b_ in zip(sols, fp64_solutions)]
            macs = st_m["macs_per_rhs"]
            tflops = macs * flops_per_mac * W["N_t"] / (slab_ms_m / 1e3) / 1e12
            v = {"value": replica_value(world, per_cycle, args.steps, ms_m), "unit": UNIT,
                 "ms_per_step": ms_m / args.steps, "slab_solve_ms": slab_ms_m,
                 "slab_factor_macs_per_rhs": macs, "slab_solve_tflops": tflops,
                 "time_to_1e-8_s": dist_of(msolve, miters), "rel_err_vs_fp64_solution": merr,
                 "residual": ("double-float (FP32 pairs, about 48 significant bits) with FP64 f and r"
                              if not kw else "FP32 inside each V-cycle, which runs in correction form around a "
                              "double-float residual (also the stopping test)"),
                 "coarsest_solve": "FP64"}
            if prec in (3, 4):
                peak = measured_peak("bf16_tflops")     # dense FP16 = dense BF16 rate on this part
                v["roofline"] = roofline_of(3, tflops, fp64_peak, slab_ms_m)
                if prec == 4:
                    v["roofline"]["kernel"] = v["roofline"]["kernel"].replace("BF16", "FP16")
                    v["roofline"]["peak_source"] = ("measured dense BF16 peak (MEASURED_PEAKS.json); dense FP16 "
                                                    "runs at the same nominal rate (2.25 PFLOP/s)")
                if least_fill_macs:
                    # the method's own count: the least-fill (64-unknown leaf) factor's products
                    lf = least_fill_macs * flops_per_mac * W["N_t"] / (slab_ms_m / 1e3) / 1e12
                    v["roofline"].update({"achieved": lf, "frac": lf / peak,
                                          "achieved_counts": "least-fill factor's complex multiply-adds "
                                          f"({least_fill_macs:.4g} per right-hand side, 64-unknown leaves) x 8 "
                                          "flop; the BF16 factor itself has 512-unknown leaves "
                                          f"({macs:.4g} per right-hand side)"})
            else:
                v["roofline"] = roofline_of(prec, tflops, fp64_peak, slab_ms_m)
            variants[vname] = v
            Sm.close()
            del fm, xm, sols
        del fp64_solutions

    # batched: `batch` excitations on one handle (problem-major slab columns), BF16
    # slab solve on the tensor cores; the same workload per problem
    if args.mixed and args.batch > 1:
        NB_ = args.batch
        Sb = make(3, n_batch=NB_)
        fb = Sb.zeros()
        for b in range(NB_):
            Sb.load(st_inputs.excitation(W["seed"] + 1 + b + 1000 * rank), f=fb, batch=b)
        xb = Sb.zeros()
        ms_b = reduce_max(time_cycles(Sb, fb, xb, args.steps), dist, "cuda")
        st_b = stmg.st_mg_factor_stats(Sb.h, 0)
        slab_ms_b = time_slab(Sb, fb, xb)
        tflops_b = st_b["macs_per_rhs"] * flops_per_mac * W["N_t"] * NB_ / (slab_ms_b / 1e3) / 1e12
        peak = measured_peak("bf16_tflops")
        variants["bf16_tensor_batched"] = {
            "value": replica_value(world, per_cycle * NB_, args.steps, ms_b), "unit": UNIT, "problems": NB_,
            "ms_per_step": ms_b / args.steps, "slab_solve_ms": slab_ms_b, "slab_solve_tflops": tflops_b,
            "slab_solve_frac_of_bf16_peak": tflops_b / peak, "bf16_peak_tflops": peak}
        if least_fill_macs:
            lf = least_fill_macs * flops_per_mac * W["N_t"] * NB_ / (slab_ms_b / 1e3) / 1e12
            variants["bf16_tensor_batched"]["slab_solve_frac_of_bf16_peak_least_fill"] = lf / peak
        Sb.close()
        del fb, xb

    # ragged batch: excitations with different slab counts over one horizon in one handle
    # (the batching configuration's N_t mix at the size of this workload's mesh)
    if args.mixed and args.ragged > 0:
        import numpy as np
        rng = np.random.Generator(np.random.PCG64(4242))
        nts = [int(v) for v in rng.permutation(np.repeat([1024, 512, 256, 128], (args.ragged + 3) // 4))[:args.ragged]]
        Sr = stmg.SpaceTimeSolver(W["n"], nu, sigma, W["T"], max(nts), W["degree"], nu_pre=W["nu_pre"],
                                  nu_post=W["nu_post"], stream=stream.cuda_stream, slab_prec=3, residual_prec=1,
                                  autotune=args.autotune, split_k=args.split_k, tc_split_k=args.tc_split_k,
                                  n_batch=len(nts), batch_nt=nts)
        fr = Sr.zeros()
        for b in range(len(nts)):
            Sr.load(st_inputs.excitation(W["seed"] + 200 + b + 1000 * rank), f=fr, batch=b)
        xr = Sr.zeros()
        ms_r = reduce_max(time_cycles(Sr, fr, xr, args.steps), dist, "cuda")
        per_r = smoothed_per_cycle(Sr.n_dof, W["nu_pre"], W["nu_post"])
        xr.zero_()
        torch.cuda.synchronize()
        a = time.perf_counter()
        out_r = Sr.solve(fr, xr, rtol=1e-8, maxit=80)
        torch.cuda.synchronize()
        t_r = time.perf_counter() - a
        variants["ragged_batch_bf16_fp32_residual"] = {
            "value": replica_value(world, per_r, args.steps, ms_r), "unit": UNIT, "problems": len(nts),
            "N_t_per_problem": nts, "dofs": Sr.n_dof, "ms_per_step": ms_r / args.steps,
            "time_to_1e-8_s": t_r, "v_cycles": out_r["iters"], "rel_res": out_r["rel_res"],
            "layout": "one handle: each problem enters the time hierarchy at the level whose step is its own; "
                      "one V-cycle advances all"}
        Sr.close()
        del fr, xr

    extra = {}
    if rank == 0 and args.config1_seeds > 0:
        extra["config1"] = run_config1(stmg, st_inputs, stream, args.config1_seeds)
    if rank == 0 and args.precision_line:
        extra["config3"] = precision_line(stmg, st_inputs, stream, args)

    cpu_base = None
    if cpu_proc is not None:
        cpu_go.set()
        res = cpu_q.get(timeout=1800)
        cpu_proc.join(timeout=60)
        cpu_base = cpu_baseline_desc(res, CPU_SAMPLE_SLABS) if "error" not in res else {"error": res["error"]}

    if rank == 0:
        cfg = workload_config(world)
        cfg.update({"time_levels": n_levels, "dofs": n_dof, "split_waves_per_level": split_waves,
                    "autotune": "given" if args.split_waves else bool(args.autotune),
                    "slab_prec": args.slab_prec, "launch_overlap": bool(args.launch_overlap),
                    "split_k": args.split_k or 32,
                    "l2": "inputs larger than L2 (129 MB): f and x %.0f MB each, finest slab factor "
                          "%.2f GB, all read in every V-cycle" % (n_dof * 8 / 1e6, st["factor_bytes"] / 1e9)})
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "time_to_1e-8_s": dist_of(solve_ms, solve_iters),
            "setup_s": setup_s,
            "roofline": roofline_of(args.slab_prec, achieved, fp64_peak, slab_ms),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * n_dof * 8,
                    "d2h_bytes_per_step": n_dof * 8 + 16},
            "gpu_launches": launches,
            "clocks": clk,
        }
        if cpu_base is not None:
            line["cpu_baseline"] = cpu_base
        for k_, v_ in variants.items():
            line[k_] = v_
        line.update(extra)
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_config1(stmg, st_inputs, stream, seeds: int) -> dict:
    """The plain method on the small case: Kuhn 4^3 (316 interior edges), nu = sigma = 1,
    T = 1, N_t = 16, DG(0), two-grid (8 coarse slabs solved by forward substitution),
    V(1,1) with SAS, omega 0.5, FP64, solved to 1e-10 from x = 0 for `seeds`
    excitations; time per solve (load excluded) and V-cycle counts."""
    import torch
    nu1, s1 = st_inputs.materials(4, "unit")
    S1 = stmg.SpaceTimeSolver(4, nu1, s1, 1.0, 16, 0, nu_pre=1, nu_post=1, max_levels=2,
                              stream=stream.cuda_stream)
    f1 = S1.zeros()
    x1 = S1.zeros()
    S1.load(st_inputs.excitation(0), f=f1)
    S1.solve(f1, x1, rtol=1e-10, maxit=60)      # warm-up (graph capture)
    ms, iters, bad = [], [], 0
    for s_ in range(seeds):
        S1.load(st_inputs.excitation(s_), f=f1)
        x1.zero_()
        torch.cuda.synchronize()
        a = time.perf_counter()
        out = S1.solve(f1, x1, rtol=1e-10, maxit=60)
        ms.append(1e3 * (time.perf_counter() - a))
        iters.append(out["iters"])
        bad += out["status"] != 0
    S1.close()
    per = smoothed_per_cycle(S1.n_dof, 1, 1)
    tot_ms = sum(ms)
    return {"workload": "kuhn4_dg0_Nt16_twogrid_V11", "dofs": S1.n_dof, "rtol": 1e-10, "seeds": seeds,
            "time_to_1e-10_s": {"p50": statistics.median(ms) / 1e3, "p99": percentile99(ms) / 1e3, "n": len(ms)},
            "v_cycles": {"min": min(iters), "max": max(iters), "mean": sum(iters) / len(iters)},
            "not_converged": bad, "dofs_smoothed_per_s": per * sum(iters) / (tot_ms / 1e3),
            "paper_context": "the paper reports 12 (Full) and 14 (Semi-time) V-cycles to 1e-10 on its own "
                             "weak-scaling problem (Section 6; CPU cluster)"}


def precision_line(stmg, st_inputs, stream, args) -> dict:
    """Larger single-GPU workload (16^3, N_t = 1024, DG(1), two materials, V(2,2), 54 M
    space-time DoFs, 11 time levels): time to 1e-8 with each slab arithmetic, V-cycle
    counts, and each solution's error against the FP64 one."""
    import torch
    n, N_t = 16, 1024
    nu, sigma = st_inputs.materials(n, "two_material", 0)
    rows, ref = {}, None
    for name, prec in (("fp64", 0), ("double_float", 2), ("fp32", 1), ("bf16_tensor", 3), ("fp16_tensor", 4)):
        S = stmg.SpaceTimeSolver(n, nu, sigma, 1.0, N_t, 1, nu_pre=2, nu_post=2, stream=stream.cuda_stream,
                                 slab_prec=prec, autotune=args.autotune)
        f = S.load(st_inputs.excitation(0))
        x = S.zeros()
        S.vcycle(f, x)                  # warm-up (graph capture), discarded
        x.zero_()
        torch.cuda.synchronize()
        a = time.perf_counter()
        out = S.solve(f, x, rtol=1e-8, maxit=60)
        torch.cuda.synchronize()
        dt = time.perf_counter() - a
        if ref is None:
            ref = x.clone()
        err = float(torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref))
        rows[name] = {"time_to_1e-8_s": dt, "v_cycles": out["iters"], "rel_res": out["rel_res"],
                      "ms_per_v_cycle": 1e3 * dt / max(out["iters"], 1), "rel_err_vs_fp64_solution": err}
        S.close()
        del f, x
    return {"workload": "kuhn16_dg1_Nt1024_V22", "dofs": 26416 * N_t * 2, "results": rows}

if __name__ == "__main__":
    sys.exit(main())

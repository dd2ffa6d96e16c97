#!/usr/bin/env python
"""Benchmark of the QTT linear-elasticity solve (AMEn sweep) on one or more GPUs.

One step = one complete solve A u = f of the 2D plane-strain steel plate on 2^10 x 2^10 nodes
(2,097,152 unknowns; E = 210 GPa, nu = 0.3, clamped left edge, gravity rho = 7850 plus a
downward traction of 1 MN/m^2 on the right edge; QTT with 10 levels, rank cap 64), from a
seeded rank-2 start, by the mixed-precision path the library calls MIXED_LOCAL: a binary64
sweep whose local systems are solved by binary32 preconditioned CG refined against the binary64
local residual.  Its tolerance (1e-9) is the one at which the solution's relative energy-norm
error against the Galerkin solution u_h is below 1e-6; the error is measured every run against
u_h stored as a QTT train by the oracle's generator script (tests/golden/).  The binary64 sweep
is timed on the same problem at the same tolerance (time to the same accuracy) and at the
tolerance that reaches 1e-8.  The operator and load are built once on the device before timing;
the e2e leg rebuilds them from the host parameters every step.

The timed loop runs with kernel sampling off; per-class device times come from a separate,
untimed profiling pass.

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas (one solve stream per
GPU, no collective on the data path): ``value`` is the total solves per second of all ranks.

``--impl reference`` runs the CPU FP64 oracle (plain numpy TT toolkit + AMEn) on the host: one
complete solve of the same workload, timed, and prints the same JSON line with
``"impl": "reference"``.
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

METRIC = "TT-solve time to rel. energy err 1e-6 (mixed vs FP64); solves/s, p50/p99 latency"
UNIT = "solves/s"

# Peaks used for the roofline fractions.  HBM / bf16 come from the measured peaks file when it is
# present; the CUDA-core peaks are derived from the SM count, lanes per SM and the maximum clock.
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP32_LANES_PER_SM = 128
FP64_NOMINAL_GFLOPS = 1250.0  # GB300 binary64 (CUDA cores and tensor cores alike)


def fp32_simt_peak_gflops(mhz: float = SM_MAX_MHZ) -> float:
    return SM_COUNT * FP32_LANES_PER_SM * 2.0 * mhz * 1e-3


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


PROBLEM = {"name": "steel2d"}  # set by --workload


def workload(levels: int, rank_cap: int, precision: str, tensor_cores: bool = False):
    from paper_2501_12151_gb300 import workloads as W
    if PROBLEM["name"] == "cube3d":
        pr = W.cantilever_3d(levels=levels, rank_cap=rank_cap, tol=1e-6, precision=precision)
        pr.opts.max_sweeps = 30
    elif PROBLEM["name"] == "quad2d":
        pr = W.quad_plate_2d(levels=levels, rank_cap=rank_cap, tol=1e-9, precision=precision)
    else:
        pr = W.steel_plate_2d(levels=levels, rank_cap=rank_cap, tol=1e-9, precision=precision)
    pr.opts.refine_tol = 1e-6
    pr.opts.tensor_cores = tensor_cores
    return pr


def workload_text(levels: int, rank_cap: int, precision: str, tol: float) -> str:
    if PROBLEM["name"] == "cube3d":
        return (f"3D cantilever (unit cube, clamped x=0, E 70 GPa, nu 0.33, gravity + seeded 8-mode Fourier force), "
                f"2^{levels} nodes per axis ({3 * 8 ** levels} DOF), QTT {levels} levels, rank cap {rank_cap}, "
                f"{precision}, tol {tol:g}, at most 30 sweeps")
    if PROBLEM["name"] == "quad2d":
        return (f"2D plane-strain steel on a general convex quadrilateral (corners (0,0) (1,0.1) (0.2,0.9) (1.3,1.4), "
                f"element Jacobians frozen at the centres), 2^{levels}x2^{levels} nodes ({2 * 4 ** levels} DOF), "
                f"QTT {levels} levels, rank cap {rank_cap}, {precision}, tol {tol:g}")
    return (f"2D plane-strain steel plate, 2^{levels}x2^{levels} nodes ({2 * 4 ** levels} DOF), QTT {levels} levels, "
            f"rank cap {rank_cap}, {precision}, tol {tol:g} (rel. energy err vs u_h measured below)")


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        # the raw samples stay on disk for inspection; TNFEM_CLOCKS_DIR chooses where
        out_dir = os.environ.get("TNFEM_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            # nvidia-smi's start-up (driver queries) is kept out of the timed region: wait for its
            # first sample (at most 5 s) before the caller starts timing
            t0 = time.perf_counter()
            while os.path.getsize(self.path) == 0 and self.proc.poll() is None and time.perf_counter() - t0 < 5.0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), float(parts[3]) if parts[3] not in ("[N/A]", "") else 0.0,
                                 parts[5], parts[6], parts[7], parts[8]))
                except ValueError:
                    continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


# ---------------------------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------------------------

def dist_init(gpus: int):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, world: int) -> float:
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------------------------
# the CPU oracle as it stands (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------------------------

def oracle_build(levels: int, rank_cap: int):
    """The FP64 oracle's operator and load for the workload (Kronecker-sum MPO, element-loop load
    vector, TT-SVD) and the seeded rank-2 start; returns them with the construction time."""
    import numpy as np
    from oracle import fem, mpo, tt
    from paper_2501_12151_gb300 import workloads as W
    pr = workload(levels, rank_cap, "fp64")
    t0 = time.perf_counter()
    Ao, _ = mpo.stiffness_mpo(pr.grid, pr.material)
    _, M = fem.assemble(pr.grid, pr.material)
    fv = fem.load_vector(pr.grid, pr.material, pr.loads, M) * np.tile(~fem.constrained_nodes(pr.grid), pr.grid.dim)
    fo = mpo.load_tt_dense(fv, pr.grid)
    t_build = time.perf_counter() - t0
    x0 = W.random_tt(pr.opts.seed, tt.modes(fo), [1] + [2] * (len(fo) - 1) + [1])
    return Ao, fo, x0, t_build


def oracle_solve(levels: int, rank_cap: int, tol: float, nswp: int):
    """One complete oracle solve: construction, then its AMEn from the seeded rank-2 start."""
    from oracle import amen, tt
    Ao, fo, x0, t_build = oracle_build(levels, rank_cap)
    t0 = time.perf_counter()
    x, info = amen.amen_solve(Ao, fo, x0, tol=tol, rmax=rank_cap, nswp=nswp)
    t_solve = time.perf_counter() - t0
    return {"t_build": t_build, "t_solve": t_solve, "sweeps": info.sweeps, "converged": bool(info.converged),
            "local_iters": int(info.local_iters), "ranks": tt.ranks(x), "threads": len(os.sched_getaffinity(0))}


def oracle_sample(levels: int, rank_cap: int, tol: float, sweeps_full: int, budget_s: float = 20.0):
    """cpu_baseline: the oracle's construction and its AMEn sweeps from the seeded start, one
    sweep per call, for about ``budget_s`` seconds; the rest of a ``sweeps_full``-sweep solve is
    extrapolated at the last (most expensive so far) sweep's time.  Ranks still grow after the
    sample (by the enrichment rank per sweep), so this is a lower bound on the oracle's time per
    solve and an upper bound on its solves/s."""
    from oracle import amen, tt
    Ao, fo, x, t_build = oracle_build(levels, rank_cap)
    times = []
    while sum(times) < budget_s and len(times) < sweeps_full:
        t0 = time.perf_counter()
        x, info = amen.amen_solve(Ao, fo, x, tol=tol, rmax=rank_cap, nswp=1, seed=len(times))
        times.append(time.perf_counter() - t0)
        if info.converged:
            break
    t_est = t_build + sum(times) + (sweeps_full - len(times)) * times[-1]
    return {"t_build": t_build, "t_est": t_est, "threads": len(os.sched_getaffinity(0)),
            "text": (f"oracle operator/load construction ({t_build:.1f} s) and {len(times)} of its AMEn sweeps "
                     f"({sum(times):.1f} s, last {times[-1]:.2f} s, ranks up to {max(tt.ranks(x))}); the remaining "
                     f"{sweeps_full - len(times)} of the {sweeps_full} sweeps of this run's binary64 solve extrapolated "
                     f"at the last sweep's time")}


# ---------------------------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------------------------

def golden_uh(ctx, levels: int):
    """u_h of the workload as a QTT train (written by tests/golden/make_steel_plate_golden.py from
    the oracle's Galerkin solve), imported into the library; None when the file is absent."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", f"steel_plate_L{levels}_uh_qtt.npz")
    if PROBLEM["name"] != "steel2d":
        return None
    if not os.path.exists(path):
        return None
    z = np.load(path)
    return ctx.tt_import([z[f"core{k}"] for k in range(len(z.files))])


def rel_energy_err(A, u, uh, nh):
    """||u - u_h||_A / ||u_h||_A from the explicitly formed difference (no cancellation)."""
    if uh is None:
        return None
    return A.energy_norm(u, uh) / nh


# DRAM bytes per launch of the two classes that can be the largest, from single-kernel ncu
# captures at the 2^10 x 2^10 working shape (profiles/): the three binary64 GEMM stages of one local
# matvec read 1.16 / 4.49 / 5.15 MB and write nothing (operands L2-resident; mean 3.6 MB); the
# fused CG moves ~0.19 MB per pass, and a launch of the solve runs ~19 passes on average
# (3.3k CG steps in 173 launches), so ~3.6 MB per launch (scaled by passes from the 51-pass capture).
TRAFFIC_NCU = {"contract64": 3.6e6, "cg32": 3.6e6}
TRAFFIC_NOTE = {"contract64": "ncu dram__bytes_read+write, mean of the 3 stage launches of one binary64 local matvec at "
                              "the working shape (profiles/gemm_kernel_double_local_matvec_steel2d_L10.md)",
                "cg32": "ncu DRAM bytes of a 51-pass fused-CG launch at the working shape scaled to the solve's mean "
                        "of ~19 passes per launch (profiles/fcg_kernel_steel2d_L10.md)"}

PROF_KERNEL = {"contract32": "gemm_kernel<float>", "contract64": "gemm_kernel<double>",
               "krylov": "CG vector kernels", "qr": "qr_*_kernel (Householder QR)",
               "svd": "svd_*_kernel (one-sided Jacobi SVD)", "other": "other kernels",
               "cg32": "fcg_kernel<float>", "cg64": "fcg_kernel<double>"}


def run_ours(args):
    import torch
    rank, world, local = dist_init(args.gpus)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the tnfem library has no CPU path)")
    torch.cuda.set_device(local)
    from paper_2501_12151_gb300 import tnfem
    # a dedicated stream: capturable into the sweep's CUDA graphs, and the one the events time
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = tnfem.Context(local, stream=stream.cuda_stream, torch_alloc=True)

    pr = workload(args.levels, args.rank_cap, args.precision, args.tensor_cores)
    pr.opts.tol = args.tol
    tb = [time.perf_counter()]
    A = ctx.stiffness(pr.grid, pr.material)
    tb.append(time.perf_counter())
    f = ctx.load(pr.grid, pr.material, pr.loads)
    tb.append(time.perf_counter())
    uh = golden_uh(ctx, args.levels)
    nh = A.energy_norm(uh) if uh is not None else None
    # L2 flush buffer (larger than the 129 MB L2), written between timed steps
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")

    def step():
        u, info = ctx.solve(A, f, pr.opts)
        return u, info

    # the warm-up repeats the timed loop's body (flush included), so that no first use of a kernel
    # or an event falls inside the timed region
    wev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for _ in range(args.warmup):
        flush.zero_()
        wev[0].record(stream)
        u, info = step()
        wev[1].record(stream)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = ctx.launches
    ctx.profile_start(0)
    infos = []
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            u, info = step()
            ev[i][1].record(stream)
            infos.append(info)
        t_end.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    launches = ctx.launches - launches0
    total_ms = t_start.elapsed_time(t_end)
    lat = sorted(a.elapsed_time(b) for a, b in ev)
    total_ms_max = max_over_ranks(total_ms, world)
    err_mixed = rel_energy_err(A, u, uh, nh)
    # a9's global confirmation of the last timed solution: ||f - A u|| / ||f|| in binary64 (dense
    # expansion where it fits the device, else the orthogonalised residual train); untimed
    t_res = time.perf_counter()
    global_res = None
    if args.global_residual:
        try:
            global_res = A.residual_norm(f, u)
        except tnfem.TnfemError as e:  # beyond the dense route the residual train may not fit
            global_res = f"not formed: {e}"
    t_res = time.perf_counter() - t_res

    # build time apart from solve time (the paper's time figure separates them): a second build of
    # the operator and the load after the timed loop, untimed by it; the first calls above also
    # carry the context's one-time start-up
    torch.cuda.synchronize()
    tw = [time.perf_counter()]
    A2 = ctx.stiffness(pr.grid, pr.material)
    tw.append(time.perf_counter())
    f2 = ctx.load(pr.grid, pr.material, pr.loads)
    tw.append(time.perf_counter())
    del A2, f2
    build_ms = {"stiffness": 1e3 * (tw[1] - tw[0]), "load": 1e3 * (tw[2] - tw[1]),
                "first_call_stiffness": 1e3 * (tb[1] - tb[0]), "first_call_load": 1e3 * (tb[2] - tb[1]),
                "timing": "host wall time of the synchronous build calls (host assembly, device rounding), "
                          "a repeat after the timed loop; first_call_* include the context's start-up"}

    # end to end through the public API: host parameters -> build -> solve -> cores to host
    e2e = None
    if not args.no_e2e:
        hs, _ = tnfem.host_stiffness(pr.grid, pr.material)
        hl = tnfem.host_load(pr.grid, pr.material, pr.loads)
        h2d = sum(c.nbytes for c in hs) + sum(c.nbytes for c in hl)
        e2e_steps = max(1, args.e2e_steps)
        walls = []
        d2h = 0
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            t1 = time.perf_counter()
            A2 = ctx.stiffness(pr.grid, pr.material)
            f2 = ctx.load(pr.grid, pr.material, pr.loads)
            u2, _ = ctx.solve(A2, f2, pr.opts)
            cores = u2.cores()
            d2h = sum(c.nbytes for c in cores)
            del A2, f2, u2
            torch.cuda.synchronize()
            walls.append(time.perf_counter() - t1)
        t_e2e = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": world * e2e_steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": e2e_steps,
               "ms_per_step": {"min": 1e3 * min(walls), "median": 1e3 * statistics.median(walls),
                               "max": 1e3 * max(walls)}}

    # binary64 sweep on the same problem: at the same tolerance (time to the same accuracy) and at
    # the tolerance of the 1e-8 target
    fp64 = None
    if args.fp64_steps > 0 and args.precision != "fp64":
        fp64 = {}
        arms = [("same_tol", args.tol, pr.opts.max_sweeps)]
        if args.fp64_tight_tol > 0:
            arms.append(("tight", args.fp64_tight_tol, 40))
        for key, tol, msw in arms:
            o64 = workload(args.levels, args.rank_cap, "fp64").opts
            o64.tol = tol
            o64.max_sweeps = msw
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.fp64_steps):
                u64, i64 = ctx.solve(A, f, o64)
            e1.record(stream)
            torch.cuda.synchronize()
            ms64 = e0.elapsed_time(e1) / args.fp64_steps
            fp64[key] = {"tol": tol, "ms_per_solve": ms64, "sweeps": i64["sweeps"], "converged": bool(i64["converged"]),
                         "rel_energy_err_vs_uh": rel_energy_err(A, u64, uh, nh)}
            if key == "same_tol":
                fp64["mixed_speedup_same_tol"] = ms64 / (total_ms / args.steps)
                fp64["rel_energy_diff_mixed_vs_fp64"] = A.energy_norm(u, u64) / A.energy_norm(u64)
        sweeps_fp64 = fp64["same_tol"]["sweeps"]
    else:
        sweeps_fp64 = infos[-1]["sweeps"]

    # profiling pass (untimed): every launch of every class timed on the device
    ctx.profile_start(1)
    for _ in range(args.prof_solves):
        step()
    prof = {c: ctx.profile_read(c) for c in tnfem.PROF_CLASSES}
    ctx.profile_start(0)

    if rank != 0:
        return None

    pk = measured_peaks()
    nprof = max(1, args.prof_solves)
    device_ms = {c: prof[c]["ms"] / nprof for c in prof}
    cls = max(device_ms, key=lambda c: device_ms[c])
    p = prof[cls]
    bf16 = pk.get("bf16_tflops")
    df_route = args.precision in ("mixed-local", "mixed-tf32") and args.tol >= 1e-7
    if cls in ("contract32", "cg32"):
        peak = fp32_simt_peak_gflops() * 1e-3
        peak_note = "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (CUDA-core binary32 FMA)"
    elif cls == "contract64" and df_route:
        # at loose tolerances the mixed path runs its large binary64 contractions in double-binary32
        # arithmetic: 12 binary32 instructions per emulated multiply-add
        peak = fp32_simt_peak_gflops() * 1e-3 / 12.0
        peak_note = ("derived: binary32 FMA peak (152 SMs x 128 lanes x 2 flop x 2070 MHz) / 12 binary32 "
                     "instructions per double-binary32 multiply-add (the class also holds small binary64 launches)")
    elif bf16:
        peak = bf16 * FP64_NOMINAL_GFLOPS / 2.25e6
        peak_note = (f"of measured: MEASURED_PEAKS bf16 {bf16} TFLOP/s x nominal binary64/bf16 ratio 1.25/2250 "
                     f"(binary64 FMA)")
    else:
        peak = FP64_NOMINAL_GFLOPS * 1e-3
        peak_note = "nominal GB300 binary64 rate 1.25 TFLOP/s"
    achieved = (p["flops"] / (p["ms"] * 1e-3) * 1e-12) if p["ms"] > 0 else 0.0
    by_class = {c: {"launches_per_solve": prof[c]["launches"] / nprof,
                    "device_ms_per_solve": device_ms[c],
                    "mean_us": (prof[c]["ms"] * 1e3 / prof[c]["sampled"]) if prof[c]["sampled"] else None,
                    "tflops": (prof[c]["flops"] / (prof[c]["ms"] * 1e-3) * 1e-12) if prof[c]["ms"] > 0 else None}
                for c in prof}
    measured_fma = {"fp64": ctx.fma_peak("fp64"), "fp32": ctx.fma_peak("fp32")}
    traffic = args.traffic if args.traffic is not None else (
        TRAFFIC_NCU.get(cls) if PROBLEM["name"] == "steel2d" and not df_route else None)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if peak else None, "traffic": traffic,
                "traffic_source": (TRAFFIC_NOTE.get(cls) if traffic is not None and args.traffic is None else
                                   ("--traffic" if traffic is not None else None)),
                "kernel": PROF_KERNEL[cls], "class": cls,
                "peak_source": peak_note,
                "fma_peak_measured_tflops": measured_fma,
                "launches_per_solve": p["launches"] / nprof,
                "avg_launch_us": (p["ms"] * 1e3 / p["sampled"]) if p["sampled"] else None,
                "flops_per_launch": (p["flops"] / p["sampled"]) if p["sampled"] else None,
                "timing": f"untimed profiling pass of {nprof} solves after the timed loop: every launch timed on the "
                          "device (globaltimer inside CUDA graphs, CUDA events outside)",
                "device_ms_by_class": device_ms,
                "by_class": by_class}

    cpu = None
    if PROBLEM["name"] == "quad2d" and not args.no_cpu_baseline:
        cpu = {"value": None, "unit": UNIT, "kind": "oracle",
               "sample": "none: the oracle's tensor-train operator builder covers boxes only"}
    elif not args.no_cpu_baseline:
        s = oracle_sample(args.levels, args.rank_cap, args.tol, sweeps_fp64)
        cpu = {"value": 1.0 / s["t_est"], "unit": UNIT, "cores": s["threads"], "kind": "oracle",
               "sample": s["text"], "estimate": "upper bound on the oracle's solves/s (its ranks still grow after the "
                                                "sampled sweeps); --impl reference times a complete oracle solve"}

    ms_per_step = total_ms_max / args.steps
    last = infos[-1]
    out = {
        "metric": METRIC,
        "value": world * args.steps / (total_ms_max * 1e-3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]},
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if args.precision != "fp64" else "f64",
        "data": "synthetic",
        "config": {"workload": workload_text(args.levels, args.rank_cap, args.precision, args.tol),
                   "levels": args.levels, "rank_cap": args.rank_cap, "precision": args.precision, "tol": args.tol,
                   "tensor_cores": bool(args.tensor_cores),
                   "parallelism": f"replicas{world}", "l2": "flushed between steps (256 MB write)"},
        "build_ms": build_ms,
        "accuracy": {"rel_energy_err_vs_uh": err_mixed,
                     "target": 1e-6,
                     "reference": ("Galerkin solution u_h of the oracle (element-loop assembly, V-cycle CG), "
                                   "stored as a QTT train accurate to 1e-10 in energy norm") if err_mixed is not None else
                                  "none stored for this workload: see fp64.rel_energy_diff_mixed_vs_fp64 and the "
                                  "global residual",
                     "global_rel_residual": global_res,
                     "global_residual_s": t_res if isinstance(global_res, float) else None,
                     "sweeps": last["sweeps"], "max_rank": last["max_rank"], "local_iters": last["local_iters"],
                     "converged": bool(last["converged"])},
        "gpu_launches": launches,
        "roofline": roofline,
        "e2e": e2e,
        "fp64": fp64,
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
    }
    return out


# ---------------------------------------------------------------------------------------------
# the reference arm: the CPU oracle as it stands
# ---------------------------------------------------------------------------------------------

def run_reference(args):
    """One complete oracle solve of the workload (operator and load construction plus AMEn to
    the same tolerance and rank cap, plain CG local solves), timed on the host's cores.  A solve
    takes minutes, so exactly one is run whatever --steps / --warmup say; ``steps`` reports it."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    s = oracle_solve(args.levels, args.rank_cap, args.tol, 40)
    t = s["t_build"] + s["t_solve"]
    value = 1.0 / t
    text = (f"one complete oracle solve: construction {s['t_build']:.1f} s, AMEn {s['t_solve']:.1f} s "
            f"({s['sweeps']} sweeps, {s['local_iters']} CG iterations, converged {s['converged']}, "
            f"max rank {max(s['ranks'])})")
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": 1,
        "warmup": 0,
        "steps_requested": args.steps,
        "ms_per_step": 1e3 * t,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_text(args.levels, args.rank_cap, "fp64 oracle", args.tol),
                   "levels": args.levels, "rank_cap": args.rank_cap, "precision": "fp64", "tol": args.tol,
                   "parallelism": "cpu"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": s["threads"], "kind": "oracle", "sample": text},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_served(args):
    """Config-5 serving: the first ``--served`` requests of the seeded stream of 512 (Poisson
    arrivals at 200/s; per request dimension, levels, E, nu, load and rank cap drawn from its own
    seed) submitted at their arrival times to the serving loop; solves/s = requests / (last
    completion - first arrival), latency = submit -> completion.  Next to it, the same requests
    solved one at a time in binary64 by one context (no overlap)."""
    import numpy as np
    import torch
    from paper_2501_12151_gb300 import tnfem
    from paper_2501_12151_gb300 import workloads as W
    arrivals, reqs = W.served_requests(seed=0, n=512, rate=200.0)
    n = min(args.served, len(reqs))
    arrivals, reqs = arrivals[:n], reqs[:n]
    srv = tnfem.Server(0, workers=args.serve_workers, hbm_budget=args.serve_budget)
    # warm-up (untimed): one small request of each dimension through the same workers
    for pr in (W.steel_plate_2d(levels=5, rank_cap=16, tol=1e-6, precision="mixed-local"),
               W.cantilever_3d(levels=3, rank_cap=16, tol=1e-6, precision="mixed-local")):
        for _ in range(args.serve_workers):
            srv.wait(srv.submit(pr.grid, pr.material, pr.loads, pr.opts), take=False)
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        ids = []
        for t_arr, pr in zip(arrivals, reqs):
            dt = t_arr - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids.append(srv.submit(pr.grid, pr.material, pr.loads, pr.opts))
        res = [srv.wait(i, take=False)[1] for i in ids]
        t_total = time.perf_counter() - t0
    srv.stop()
    lat = sorted(r["latency_us"] * 1e-3 for r in res)
    ok = sum(r["status"] in ("OK", "NOT_CONVERGED") for r in res)
    # one at a time, binary64, one context
    ctx = tnfem.Context(0)
    seq = []
    t1 = time.perf_counter()
    for pr in reqs[: args.serve_fp64]:
        o = W.SolveOpts(**{**pr.opts.__dict__, "precision": "fp64"})
        ts = time.perf_counter()
        A = ctx.stiffness(pr.grid, pr.material)
        f = ctx.load(pr.grid, pr.material, pr.loads)
        u, info = ctx.solve(A, f, o)
        u.cores()
        seq.append(1e3 * (time.perf_counter() - ts))
        del A, f, u
    t_seq = time.perf_counter() - t1
    dims = [pr.grid.dim for pr in reqs]
    return {
        "metric": "served TT solves: solves/s, p50/p99 latency (continuous batching)",
        "value": n / t_total, "unit": "solves/s", "n_gpus": 1, "steps": n, "warmup": 2 * args.serve_workers,
        "ms_per_step": 1e3 * t_total / n,
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
                       "max": lat[-1]},
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"served batch: first {n} of 512 seeded requests, Poisson arrivals at 200/s, "
                               f"2D L 6..10 / 3D L 5..9, E log-uniform 1e9..3e11, nu 0.2..0.45, gravity / traction / "
                               f"Fourier load, rank cap 16..96, mixed-local tol 1e-6",
                   "requests": n, "requests_2d": dims.count(2), "requests_3d": dims.count(3),
                   "workers": args.serve_workers, "parallelism": "one GPU, overlapping worker streams"},
        "served": {"completed": ok, "makespan_s": t_total,
                   "mean_run_ms": float(np.mean([r["run_us"] for r in res])) * 1e-3,
                   "mean_queued_ms": float(np.mean([r["queued_us"] for r in res])) * 1e-3,
                   "peak_within_estimate": all(r["peak_bytes"] <= r["est_bytes"] for r in res),
                   "statuses": sorted({r["status"] for r in res}),
                   "requests": [{"dim": pr.grid.dim, "levels": pr.grid.levels, "cap": pr.opts.rank_cap,
                                 "status": r["status"], "run_ms": round(r["run_us"] * 1e-3, 1),
                                 "latency_ms": round(r["latency_us"] * 1e-3, 1), "sweeps": r["info"]["sweeps"],
                                 "est_MiB": r["est_bytes"] >> 20, "peak_MiB": r["peak_bytes"] >> 20}
                                for pr, r in zip(reqs, res)]},
        "one_at_a_time_fp64": {"requests": len(seq), "solves_per_s": len(seq) / t_seq if seq else None,
                               "p50_ms": sorted(seq)[len(seq) // 2] if seq else None},
        "clocks": clk.summary(),
    }


def run_kernel_probe(args):
    """A few launches of each local-matvec engine at the solve's working shapes (for ncu): the
    binary32 contraction on CUDA cores and on the tcgen05 tensor cores, and the binary64 one,
    through the C ABI on seeded Gaussian inputs; then the fused CG kernel in both precisions.  Prints wall time per call (allocation and launch
    overheads included; kernel durations come from the profiler)."""
    import numpy as np
    import torch
    from paper_2501_12151_gb300 import tnfem
    from paper_2501_12151_gb300 import workloads as W
    r0, n, r1, a0, a1 = args.probe_shape
    ctx = tnfem.Context(0)

    def dev(a, dt):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()

    PhiL = W.rng(1).standard_normal((r0, a0, r0))
    A = W.rng(2).standard_normal((a0, n, n, a1))
    PhiR = W.rng(3).standard_normal((r1, a1, r1))
    x = W.rng(4).standard_normal((r0, n, r1))
    flops = 2.0 * n * r0 * r1 * (r0 * a0 + n * a0 * a1 + r1 * a1)
    out = {"probe": "local matvec", "shape": {"r0": r0, "n": n, "r1": r1, "a0": a0, "a1": a1}, "flops": flops}
    for dt, name in ((np.float32, "f32"), (np.float64, "f64")):
        if args.probe_f64_only and dt == np.float32:
            continue
        t = [dev(v, dt) for v in (PhiL, A, PhiR, x)]
        y = torch.zeros(r0 * n * r1, dtype=torch.float32 if dt == np.float32 else torch.float64, device="cuda")
        for e in ((0, 1, 2) if dt == np.float32 else (None,)):
            walls = []
            for _ in range(args.probe_reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if e is None:
                    ctx.op_local_matvec(r0, n, r1, a0, a1, *[v.data_ptr() for v in t], y.data_ptr())
                else:
                    ctx.op_local_matvec_f32(e, r0, n, r1, a0, a1, *[v.data_ptr() for v in t], y.data_ptr())
                torch.cuda.synchronize()
                walls.append(time.perf_counter() - t0)
            out[f"{name}_engine{e if e is not None else 'fp64'}_wall_us"] = 1e6 * min(walls)
    if args.probe_f64_only:
        return out
    # the fused CG kernel on a symmetric positive definite system of the same shape
    # (B = sum_beta PhiL_beta (x) M_beta (x) PhiR_beta, PSD factors, identity-shifted beta = 0 term),
    # a fixed number of steps (rtol 0)
    rs = W.rng(5)
    SL, SA, SR = np.zeros((r0, a0, r0)), np.zeros((a0, n, n, a1)), np.zeros((r1, a1, r1))
    for b in range(min(a0, a1)):
        Lb, Rb, Mb = rs.standard_normal((r0, r0)), rs.standard_normal((r1, r1)), rs.standard_normal((n, n))
        sh = 1.0 if b == 0 else 0.0
        SL[:, b, :] = Lb @ Lb.T / r0 + sh * np.eye(r0)
        SR[:, b, :] = Rb @ Rb.T / r1 + sh * np.eye(r1)
        SA[b, :, :, b] = Mb @ Mb.T / n + sh * np.eye(n)
    g = rs.standard_normal((r0, n, r1))
    for dt, name in ((np.float32, "f32"), (np.float64, "f64")):
        t = [dev(v, dt) for v in (SL, SA, SR, g)]
        walls = []
        try:
            for _ in range(args.probe_reps):
                xg = torch.zeros(r0 * n * r1, dtype=t[0].dtype, device="cuda")
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                its, _ = ctx.op_local_cg("fp64" if dt == np.float64 else "fp32", 1, r0, n, r1, a0, a1,
                                         *[v.data_ptr() for v in t], xg.data_ptr(), 0.0, args.probe_cg_steps)
                torch.cuda.synchronize()
                walls.append(time.perf_counter() - t0)
        except tnfem.TnfemError as e:  # the fused kernel's shape limits (the sweep then steps per launch)
            out[f"{name}_fused_cg"] = str(e)
            continue
        out[f"{name}_fused_cg_steps"] = its
        out[f"{name}_fused_cg_wall_us"] = 1e6 * min(walls)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--levels", type=int, default=10)
    ap.add_argument("--rank-cap", type=int, default=64)
    ap.add_argument("--precision", choices=["mixed", "mixed-local", "fp64"], default="mixed-local")
    ap.add_argument("--tensor-cores", action="store_true", help="binary32 contractions on tcgen05")
    ap.add_argument("--tol", type=float, default=1e-9, help="sweep tolerance of the timed solves")
    ap.add_argument("--fp64-tight-tol", type=float, default=1e-11, help="binary64 tolerance for the 1e-8 target")
    ap.add_argument("--prof-solves", type=int, default=2, help="solves in the untimed profiling pass")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the dominant kernel from an ncu capture (roofline.traffic)")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-global-residual", dest="global_residual", action="store_false",
                    help="skip the global residual confirmation of the last solution")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--kernel-probe", action="store_true",
                    help="only launch the local-matvec engines and the fused CG kernel a few times at --probe-shape (for ncu)")
    ap.add_argument("--probe-shape", type=int, nargs=5, default=[49, 4, 49, 51, 51], metavar=("R0", "N", "R1", "A0", "A1"))
    ap.add_argument("--probe-reps", type=int, default=3)
    ap.add_argument("--probe-f64-only", action="store_true", help="only the binary64 local matvec in the probe")
    ap.add_argument("--probe-cg-steps", type=int, default=50, help="steps of the fused CG launch in the probe")
    ap.add_argument("--served", type=int, default=0, help="run the served batch with this many requests instead")
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-budget", type=int, default=0, help="device-memory budget of the server (0: 80%% of free)")
    ap.add_argument("--serve-fp64", type=int, default=16, help="requests of the one-at-a-time binary64 baseline")
    ap.add_argument("--workload", choices=["steel2d", "cube3d", "quad2d"], default="steel2d",
                    help="steel2d: the 2^10 x 2^10 steel plate (default); cube3d: the 3D cantilever (use with "
                         "--levels 7 --rank-cap 96 --tol 1e-6 --fp64-tight-tol 0 --no-cpu-baseline); quad2d: steel "
                         "on a general quadrilateral (use with --fp64-tight-tol 0 --no-cpu-baseline)")
    args = ap.parse_args(argv)
    PROBLEM["name"] = args.workload
    if args.served > 0:
        out = run_served(args)
    elif args.kernel_probe:
        out = run_kernel_probe(args)
    else:
        out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

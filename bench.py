"""Benchmark of the GB300 S_N step (one JSON line on stdout).

Default workload (the lattice at production size): 1400 x 1400 Cartesian grid
on [0,7]^2 (dx = 0.005), 16 polar x 32 azimuthal = 512 ordinates, MUSCL-minmod
upwind fluxes, Heun (two stages per step), psi stored in FP32, dt = dx/2
(1280 steps to T = 3.2). A "step" is one time step of the whole path (both
Heun stages: fluxes, collision, scalar flux, FP64 QoI partials) over the grid.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference] [--workload NAME]

--impl reference times the FP64 CPU oracle on the host on a bounded sample of
the same workload (same metric and unit).
"""
from __future__ import annotations

import argparse
import collections
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "S_N cell-ordinate updates/s"
UNIT = "updates/s"
QOI_BYTES = 392   # sizeof(rt_qoi_t): the QoI read-back of one problem

WORKLOADS = {
    # name: (mesh, n, n_p, n_phi, order, integrator, storage, dt_factor, t_end); n_p = 0 selects the
    # tessellation rule of order n_phi (Sec. 5.1.1, 4 n_phi^2 ordinates) instead of the product rule
    "lattice1400_muscl_heun_fp32": ("lattice", 1400, 16, 32, 2, "heun", "fp32", 0.5, 3.2),
    "lattice1400_muscl_heun_bf16": ("lattice", 1400, 16, 32, 2, "heun", "bf16", 0.5, 3.2),
    "lattice1400_o1_euler_fp32": ("lattice", 1400, 16, 32, 1, "euler", "fp32", 0.5, 3.2),
    "enclosure1300_tri_o1_euler_fp32": ("enclosure", 1300, 8, 32, 1, "euler", "fp32", 0.0, 2.6),
    "lattice70_o1_euler_fp32": ("lattice", 70, 4, 16, 1, "euler", "fp32", 0.5, 3.2),
    "lattice560_muscl_heun_fp32": ("lattice", 560, 16, 32, 2, "heun", "fp32", 0.5, 3.2),
    "lattice840_muscl_heun_fp32": ("lattice", 840, 16, 32, 2, "heun", "fp32", 0.5, 3.2),
    "lattice840_muscl_heun_bf16": ("lattice", 840, 16, 32, 2, "heun", "bf16", 0.5, 3.2),
    "enclosure650_tri_o1_euler_fp32": ("enclosure", 650, 8, 32, 1, "euler", "fp32", 0.0, 2.6),
    # the paper's production scheme on triangles: Green-Gauss + Venkatakrishnan, Heun
    "enclosure1300_tri_o2_heun_fp32": ("enclosure", 1300, 8, 32, 2, "heun", "fp32", 0.0, 2.6),
    "enclosure650_tri_o2_heun_fp32": ("enclosure", 650, 8, 32, 2, "heun", "fp32", 0.0, 2.6),
    # the paper's own angular resolution: tessellation order 22 (1936 ordinates)
    "lattice1400_muscl_heun_tess22_fp32": ("lattice", 1400, 0, 22, 2, "heun", "fp32", 0.5, 3.2),
}
DEFAULT = "lattice1400_muscl_heun_fp32"


def bytes_per_update(order, integrator, storage, mesh="lattice"):
    """Algorithmic HBM bytes per cell-ordinate per step (state traffic only):
    Euler reads psi^n and writes psi^{n+1}; Heun stage 1 reads psi^n and writes
    psi1, stage 2 reads psi1 and psi^n and writes psi^{n+1}. Second order on
    triangles adds, per stage, the limited gradient (two FP32 values) written
    by the gradient pass and read back by the stage pass, and the gradient
    pass's read of the stage input."""
    es = 2 if storage == "bf16" else 4
    base = (2 if integrator == "euler" else 5) * es
    if mesh != "lattice" and order == 2:
        stages = 1 if integrator == "euler" else 2
        base += stages * (es + 16)
    return base


KERNEL_SOURCES = {"cart": ["cart_kernel.cuh", "device_common.cuh"],
                  "tri": ["tri_staged_kernel.cu", "tri_kernel.cu", "device_common.cuh"],
                  "tri2": ["tri2_kernel.cu", "device_common.cuh"]}


def kernel_sha(kind):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_2505_17284_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload, kind):
    """DRAM bytes per cell-ordinate per step of the stage kernel, from the
    'traffic:' line of a committed ncu summary under profiles/ for this
    workload, or None when there is none or the kernel sources changed since
    the capture (the summary records their hash)."""
    import glob
    sha = kernel_sha(kind)
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as fh:
            for line in fh:
                if not line.startswith("traffic:"):
                    continue
                kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
                if kv.get("workload") == workload and kv.get("kernel") == kind and kv.get("sha") == sha:
                    return float(kv["bytes_per_update"]), os.path.relpath(path, ROOT)
    return None, None


def make_problem(spec):
    import sn_inputs as si
    mesh, n, n_p, n_phi, order, integ, storage, dtf, t_end = spec
    if mesh == "lattice":
        p = si.lattice_problem(n, t_end=t_end)
        dt = dtf * p.mesh.dx
    else:
        p = si.enclosure_problem(n, jitter=0.2, seed=0, t_end=t_end)
        dt = 0.0
    return p, dt


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle baseline
def oracle_sample(spec, budget_s, workers=1):
    """Time the FP64 oracle on a bounded sample of the workload: the same
    scheme and ordinate set on a smaller grid, sized to about budget_s seconds
    of work, in `workers` single-threaded processes at once (each its own copy
    of the sample: the oracle is a serial numpy program, so the host's cores
    are used by running several); returns (updates/s summed over the
    processes, description, seconds)."""
    code = r"""
import json, sys, time, numpy as np
sys.path.insert(0, %r)
import oracle, sn_inputs as si
mesh, n_full, n_p, n_phi, order, integ, storage, dtf, t_end = %r
Q = oracle.product_quadrature(n_p, n_phi) if n_p else oracle.tessellation_quadrature(n_phi)
MQ = len(Q[0])
budget = %r
def build(n):
    if mesh == "lattice":
        p = si.lattice_problem(n); dt = dtf * p.mesh.dx
        op = oracle.CartesianOracle(p, Q, order=order)
    else:
        p = si.enclosure_problem(n, jitter=0.2, seed=0)
        op = oracle.TriangleOracle(p, Q, order=order)
        dt = oracle.triangle_dt(op, t_end)[1]
    return p, op, dt
n = 14 if mesh == "lattice" else 10
p, op, dt = build(n)
psi = np.zeros((p.mesh.n_cells, MQ))
t0 = time.perf_counter(); oracle.run(op, psi, dt, 1, integ); t1 = time.perf_counter()
rate = p.mesh.n_cells * MQ / (t1 - t0)
steps = 3
n2 = int(max(14, min(n_full, (rate * budget / steps / MQ) ** 0.5 / (1 if mesh == "lattice" else 1.41))))
if mesh == "lattice": n2 = max(7, n2 // 7 * 7)
p, op, dt = build(n2)
psi = np.zeros((p.mesh.n_cells, MQ))
t0 = time.perf_counter(); oracle.run(op, psi, dt, steps, integ); t1 = time.perf_counter()
print(json.dumps({"rate": p.mesh.n_cells * MQ * steps / (t1 - t0), "n": n2, "steps": steps,
                  "cells": p.mesh.n_cells, "seconds": t1 - t0}))
""" % (ROOT, list(spec), budget_s)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                              env=env) for _ in range(workers)]
    outs = []
    for pr in procs:
        out, err = pr.communicate(timeout=900)
        if pr.returncode != 0:
            raise RuntimeError("oracle baseline failed: " + err[-2000:])
        outs.append(json.loads(out.strip().splitlines()[-1]))
    d = outs[0]
    mesh = spec[0]
    desc = (f"FP64 numpy oracle, {workers} process{'es' if workers > 1 else ''} of 1 thread each: "
            f"{'lattice' if mesh == 'lattice' else 'enclosure triangles'} "
            f"{d['n']}x{d['n']} ({d['cells']} cells) x {spec[2] * spec[3] if spec[2] else 4 * spec[3] ** 2} ordinates, "
            f"{d['steps']} steps of the same scheme in each; rate scaled per cell-ordinate update")
    return sum(o["rate"] for o in outs), desc, max(o["seconds"] for o in outs)


# ------------------------------------------------------------------ replicas (N > 1)
# Under torchrun every rank solves its own copy of the workload (no data-path
# collective: one solve does not shard across GPUs); the job's time is the
# slowest rank's and its throughput the units of all ranks over that time.
def replica_env():
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, device):
    """The largest x over all ranks of the default process group (x itself
    when there is none)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms_max):
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (ms)."""
    return units_per_rank * world / (ms_max * 1e-3)


# ------------------------------------------------------------------ ours
def run_ours(args, spec):
    import numpy as np
    import torch
    from paper_2505_17284_gb300 import build as B, rt

    rank, world, local = replica_env()
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        B.build()
    if dist:
        tdist.barrier()
    rt.load_library()

    mesh, n, n_p, n_phi, order, integ, storage, dtf, t_end = spec
    problem, dt = make_problem(spec)
    quad = rt.rt_quad_product(n_p, n_phi) if n_p else rt.rt_quad_tessellation(n_phi)
    integ_c = rt.RT_HEUN if integ == "heun" else rt.RT_EULER
    stor_c = rt.RT_BF16 if storage == "bf16" else rt.RT_FP32
    # Cartesian tiles from the autotuner (timed once per device and shape, before
    # any timed region) unless given on the command line
    tune = mesh == "lattice" and not args.no_tune and args.tile_x == 0 and args.tile_y == 0
    solver = rt.Solver(problem, quad, order=order, integrator=integ_c, storage=stor_c, dt=dt,
                       tile_x=args.tile_x, tile_y=args.tile_y, tune=tune)
    info = solver.info
    K, W = args.steps, args.warmup
    if K + W > info.n_steps:
        raise SystemExit(f"steps + warmup ({K + W}) exceed the {info.n_steps} steps of the workload")
    stream = torch.cuda.current_stream()
    solver.step(W)
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    solver.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    q = solver.qoi()
    ms = max_over_ranks(ms, "cuda")
    dof = info.n_cells * info.M
    value = job_value(dof * K, world, ms)
    bpu = bytes_per_update(order, integ, storage, mesh)
    # stage launches, plus one QoI-box launch per step (Cartesian problems with
    # boxes); second order on triangles runs a gradient launch before each stage
    launches_per_step = info.stages_per_step * (2 if (mesh != "lattice" and order == 2) else 1) + \
        (1 if info.n_box_items else 0)
    achieved_gbs = dof * bpu * K / (ms * 1e-3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    solver.close()

    # end to end through the C ABI from host buffers: create (H2D of the problem),
    # K steps, QoI read-back (D2H), destroy
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s2 = rt.Solver(problem, quad, order=order, integrator=integ_c, storage=stor_c, dt=dt,
                   tile_x=args.tile_x, tile_y=args.tile_y, tune=tune)
    s2.step(K)
    q2 = s2.qoi()
    s2.close()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    n_cells = info.n_cells
    if mesh == "lattice":
        # per-cell material and region bytes, the quadrature, 16 bytes per QoI-box face
        n_faces = sum(2 * round((b[1] - b[0]) / problem.mesh.dx) + 2 * round((b[3] - b[2]) / problem.mesh.dy)
                      for b in problem.extra.get("boxes", ()))
        h2d = 2 * n_cells + 3 * info.M_pad * 4 + 16 * n_faces
    else:
        h2d = n_cells * (16 + 32) + 3 * info.M_pad * 4
    d2h = QOI_BYTES

    kind = "cart" if mesh == "lattice" else ("tri2" if order == 2 else "tri")
    tb, traffic_src = profiled_traffic(args.workload, kind)
    traffic = tb * dof if tb is not None else None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if storage == "bf16" else "f32",
        "data": "synthetic (seeded lattice/enclosure geometry, psi0 = 0)",
        "config": {"workload": args.workload, "grid": f"{n}x{n}" if mesh == "lattice" else f"{n}x{n} split, jittered",
                   "cells": n_cells, "ordinates": info.M, "order": order, "integrator": integ,
                   "psi_storage": storage, "dt": info.dt, "n_steps_total": info.n_steps,
                   "tile": [info.tile_x, info.tile_y], "work_items": info.n_work_items,
                   "tile_choice": "rt_autotune (cached per device and shape)" if tune else
                                  ("command line" if (args.tile_x or args.tile_y) else "library model"),
                   "l2": f"inputs larger than L2 (psi {dof * (2 if storage == 'bf16' else 4) / 1e9:.2f} GB per buffer)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": peak, "unit": "GB/s",
                     "frac": achieved_gbs / peak, "traffic": traffic,
                     "traffic_per": "step (all stage launches), DRAM read + write bytes",
                     "traffic_source": traffic_src,
                     "kernel": {"cart": "cart_stage_kernel",
                                "tri": "tri_staged_kernel" if info.variant == 3 else "tri_stage_kernel",
                                "tri2": "tri_grad_kernel + tri_stage2_kernel"}[kind],
                     "bytes_per_update": bpu, "peak_source": f"{peak_src} hbm_gbs",
                     "achieved_basis": "algorithmic bytes per cell-ordinate x cell-ordinates x steps / event time of the steps"},
        "e2e": {"value": dof * K / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h / K,
                "seconds": e2e_s, "includes": "rt_create from host arrays + K steps + rt_qoi read-back + rt_destroy"},
        "gpu_launches": K * launches_per_step,
        "clocks": clk,
        "qoi_after": {"step": q["step"], "abs_int_blue": float(q["abs_int"][1]) if mesh == "lattice" else None,
                      "mass": q["mass"], "box_out_now": [float(v) for v in q["box_out_now"]],
                      "box_out_int": [float(v) for v in q["box_out_int"]]},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        rate, desc, secs = oracle_sample(spec, budget_s=args.cpu_budget, workers=cores)
        rate1, desc1, secs1 = oracle_sample(spec, budget_s=args.cpu_budget, workers=1)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
                               "seconds": secs, "single_thread": {"value": rate1, "cores": 1, "sample": desc1,
                                                                  "seconds": secs1}}
    if dist:
        tdist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def run_reference(args, spec):
    rank, _, _ = replica_env()
    if rank != 0:
        return   # the oracle runs on rank 0 alone; the other ranks exit without work
    K, W = args.steps, args.warmup
    per_step = max(0.5, min(20.0, 150.0 / (K + W)))
    import numpy as np
    import oracle
    import sn_inputs as si
    mesh, n_full, n_p, n_phi, order, integ, storage, dtf, t_end = spec
    Q = oracle.product_quadrature(n_p, n_phi) if n_p else oracle.tessellation_quadrature(n_phi)
    # size the sample so that one step costs about per_step seconds
    def build(n):
        if mesh == "lattice":
            p = si.lattice_problem(n)
            op = oracle.CartesianOracle(p, Q, order=order)
            return p, op, dtf * p.mesh.dx
        p = si.enclosure_problem(n, jitter=0.2, seed=0)
        op = oracle.TriangleOracle(p, Q)
        return p, op, oracle.triangle_dt(op, t_end)[1]
    p, op, dt = build(14 if mesh == "lattice" else 10)
    M = len(Q[0])
    t0 = time.perf_counter()
    oracle.run(op, np.zeros((p.mesh.n_cells, M)), dt, 1, integ)
    rate = p.mesh.n_cells * M / (time.perf_counter() - t0)
    n = int(max(14, min(n_full, math.sqrt(rate * per_step / M))))
    if mesh == "lattice":
        n = max(7, n // 7 * 7)
    p, op, dt = build(n)
    psi = np.zeros((p.mesh.n_cells, M))
    psi, _, _ = oracle.run(op, psi, dt, W, integ)
    t0 = time.perf_counter()
    oracle.run(op, psi, dt, K, integ)
    secs = time.perf_counter() - t0
    value = p.mesh.n_cells * M * K / secs
    desc = f"FP64 numpy oracle on {n}x{n} cells x {M} ordinates, same scheme, {K} steps (bounded sample)"
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
           "steps": K, "warmup": W, "ms_per_step": secs * 1e3 / K, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": args.workload, "sample_grid": f"{n}x{n}", "ordinates": M},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ------------------------------------------------------------------ sweeps and serving
EXTRA_WORKLOADS = {
    # lattice DP-1 sweep: 256 instances, grids {70,140,280,560}^2, M in {64,128,256}, MUSCL Heun FP32
    "sweep256": dict(kind="sweep", k=256, grids=(70, 140, 280, 560)),
    # the same draws restricted to small grids, where one solve cannot fill the GPU
    "sweep256_small": dict(kind="sweep", k=256, grids=(70, 140)),
    # lattice DP-2 sweep: 256 instances, 49 per-block sigma_a and sigma_s each, same grids and ordinates
    "sweep256_dp2": dict(kind="sweep", k=256, grids=(70, 140, 280, 560), dp=2),
    # Poisson stream of 200 mixed lattice / enclosure requests to the benchmarks' end times
    "serve200": dict(kind="serve", count=200, horizon=1.0),
}


def _quads(rt, cache, n_p, n_phi):
    key = (n_p, n_phi)
    if key not in cache:
        cache[key] = rt.rt_quad_product(n_p, n_phi)
    return cache[key]


def sweep_jobs(rt, k, grids, seed=0, dp=1):
    import sn_inputs as si
    from paper_2505_17284_gb300.sweep import Job
    qc, jobs = {}, []
    if dp == 2:
        for inst in si.dp2_instances(k, seed, grids=grids):
            p = si.lattice_dp2_problem(inst.n, inst.sigma_a, inst.sigma_s)
            jobs.append(Job(p, _quads(rt, qc, inst.n_p, inst.n_phi), 2, rt.RT_HEUN, 0.5 * p.mesh.dx))
        return jobs
    for inst in si.sweep_instances(k, seed, grids=grids):
        p = si.lattice_problem(inst.n, sigma_a_blue=inst.sigma_a, sigma_s_scatter=inst.sigma_s)
        jobs.append(Job(p, _quads(rt, qc, inst.n_p, inst.n_phi), 2, rt.RT_HEUN, 0.5 * p.mesh.dx))
    return jobs


def _peak():
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs")
    except Exception:
        pk = None
    return (pk, "measured hbm_gbs") if pk else (6800.0, "fallback hbm_gbs")


def run_sweep(args, w):
    import torch
    from paper_2505_17284_gb300 import build as B, rt, autotune
    from paper_2505_17284_gb300 import sweep as S
    B.build()
    rt.load_library()
    dp = w.get("dp", 1)
    jobs = sweep_jobs(rt, w["k"], w["grids"], dp=dp)
    if args.profile_step:
        # one batched step of the first --profile-step instances (for profilers): two untimed steps, then one
        # inside cudaProfilerStart/Stop (for ncu --profile-from-start off); --profile-tuned takes the per-group
        # options of tune_groups (timed before the profiled region) instead of one tile_y for the batch
        import torch
        sub = jobs[:args.profile_step]
        configs, table = (S.tune_groups(sub, steps=2) if args.profile_tuned else (None, None))
        b = rt.Batch([j.problem for j in sub], [j.quad for j in sub], dts=[j.dt for j in sub],
                     orders=[j.order for j in sub], integrators=[j.integrator for j in sub],
                     tile_y=0 if args.profile_tuned else (args.tile_y or 16), configs=configs)
        b.step(1)
        b.step(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0 = b.launches()
        torch.cuda.profiler.start()
        e0.record()
        b.step(1)
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"workload": args.workload, "instances": len(sub),
                          "options": table if args.profile_tuned else {"tile_y": args.tile_y or 16},
                          "launches": b.launches() - n0, "ms_one_batched_step": e0.elapsed_time(e1)}))
        b.close()
        return
    # autotuned tiles: one rt_autotune per distinct shape for the one-at-a-time
    # path, and the batch-level segment length for the batched path
    shapes = {}
    for j in jobs:
        shapes.setdefault((j.problem.mesh.nx, j.M), j)
    for j in shapes.values():
        autotune.tuned_config(j.problem, j.quad, j.order, j.integrator, rt.RT_FP32, j.dt, steps=3)
    by_shape = args.batch_tune == "shape"
    configs, group_table = S.tune_groups(jobs, tile_ys=(0, 16, 24, 32, 48), variants=(0, 1), steps=3,
                                         by_shape=by_shape)
    clocks = ClockSampler(0)
    clocks.start()
    phases = {}
    qb, tb, steps_b = S.solve_batched(jobs, configs=configs, phases=phases)
    batched_launches = phases.pop("gpu_launches")
    qp, tp, per, steps_p = S.solve_plain(jobs, tune=True)
    clk = clocks.stop()
    diff = max(S.qoi_rel_diff(a, b) for a, b in zip(qb, qp))
    peak, peak_src = _peak()
    nbytes = S.state_bytes(jobs, steps_b)
    ideal = nbytes / (peak * 1e9)
    updates = sum(float(j.n_cells) * j.M * n for j, n in zip(jobs, steps_b))
    k = len(jobs)
    box = 1 if all(j.problem.extra.get("boxes") for j in jobs) else 0
    out = {
        "metric": "batched solves/s", "value": k / tb, "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": tb * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": f"synthetic (seeded lattice DP-{dp} sweep)",
        "config": {"workload": args.workload, "instances": k, "grids": list(w["grids"]), "ordinates": [64, 128, 256],
                   **({"sigma_a": "U[5,15]", "sigma_s": "U[0.5,1.5]"} if dp == 1 else
                      {"sigma_a_ij": "blue blocks U[5,15], others U[0,0.5]",
                       "sigma_s_ij": "blue blocks U[0,0.5], others U[0.5,1.5]", "materials": 49}),
                   "scheme": "MUSCL Heun", "psi_storage": "fp32",
                   "step": "one whole sweep (all instances to their N_t = 0.914 n)",
                   "batch_configs": group_table,
                   "batch_configs_basis": "per group of one ordinate count" + (" and grid" if by_shape else "")
                                          + ": tile_y x variant (0 = library choice, 1 = per-lane directions), ms "
                                          "per step of that group alone",
                   "plain_tiles": "rt_autotune per shape", "l2": "working set of the large-grid instances > L2"},
        "plain": {"solves_per_s": k / tp, "seconds": tp, "path": "rt_create + rt_step(N_t) + rt_qoi + rt_destroy per instance"},
        "batched_seconds": tb,
        "batched_phases_s": phases,
        "speedup_vs_plain": tp / tb,
        "amdahl_bound": tp / ideal,
        "amdahl_basis": "plain seconds / seconds of the sweep's algorithmic state bytes at the HBM peak",
        "qoi_max_rel_diff_batched_vs_plain": diff,
        "updates_per_s_batched": updates / tb,
        "roofline": {"bound": "hbm", "achieved": nbytes / tb / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": nbytes / tb / 1e9 / peak, "traffic": None, "kernel": "cart_stage_kernel (batched)",
                     "peak_source": peak_src},
        "e2e": {"value": k / tb, "unit": "solves/s", "h2d_bytes_per_step": None, "d2h_bytes_per_step": k * QOI_BYTES,
                "includes": "batch creation from host arrays, all steps, QoI read-back, destroy"},
        "gpu_launches": {"batched": batched_launches,
                         "plain": sum((2 + box) * n + 1 + box for n in steps_p),
                         "basis": "batched: rt_batch_launches (per step 2 stage launches per kernel-variant group and "
                                  "1 QoI-box launch for all groups; per instance 1 initial-state launch and 1 initial "
                                  "box launch); plain: per step 2 stage launches (+1 box launch), per instance 1 init "
                                  "(+1)"},
        "clocks": clk,
    }
    print(json.dumps(out))


def serve_requests(rt, count, horizon, storage, seed=0, arrivals=None):
    import numpy as np
    import sn_inputs as si
    from paper_2505_17284_gb300.serve import Request, estimate_bytes
    from paper_2505_17284_gb300.sweep import Job
    specs = si.serve_requests(count, seed, horizon)
    qc = {}
    reqs = []
    for i, sp in enumerate(specs):
        q = _quads(rt, qc, sp.n_p, sp.n_phi)
        if sp.kind == "lattice":
            make = (lambda sp=sp, q=q: Job(si.lattice_problem(sp.n, t_end=sp.t_end), q, 2, rt.RT_HEUN, 0.5 * 7.0 / sp.n))
            nb = estimate_bytes(sp.n * sp.n, sp.M, storage)
        else:
            make = (lambda sp=sp, q=q, i=i: Job(si.enclosure_problem(sp.n, jitter=0.2, seed=i, t_end=sp.t_end), q, 1,
                                                rt.RT_EULER, 0.0))
            nb = estimate_bytes(2 * sp.n * sp.n, sp.M, storage, triangles=True)
        reqs.append(Request(rid=i, arrival=0.0 if arrivals is None else float(arrivals[i]), make=make, est_bytes=nb))
    return reqs, specs


def _oracle_request(task):
    """The FP64 oracle on one request of the serving stream (run in a spawned
    worker process): returns (rid, QoIs at its final time, seconds)."""
    import oracle
    import sn_inputs as si
    rid, kind, n, n_p, n_phi, t_end = task
    t0 = time.perf_counter()
    Q = oracle.product_quadrature(n_p, n_phi)
    if kind == "lattice":
        p = si.lattice_problem(n, t_end=t_end)
        op = oracle.CartesianOracle(p, Q, order=2)
        n_t = oracle.n_steps_for(t_end, 0.5 * 7.0 / n)
        dt, integ = t_end / n_t, "heun"
    else:
        p = si.enclosure_problem(n, jitter=0.2, seed=rid, t_end=t_end)
        op = oracle.TriangleOracle(p, Q, order=1)
        n_t, dt = oracle.triangle_dt(op, t_end)
        integ = "euler"
    import numpy as np
    psi, acc, S = oracle.run(op, np.zeros((p.mesh.n_cells, n_p * n_phi)), dt, n_t, integ)
    q = {"mass": S["mass"], "abs_int": [float(v) for v in acc.abs_int], "outflow_int": float(acc.outflow_int)}
    return rid, q, time.perf_counter() - t0


def oracle_request_cost(sp):
    """Rough oracle seconds of one request (serial numpy rates: lattice MUSCL
    Heun about 4e6, first-order triangles about 1.5e7 cell-ordinate steps per
    second)."""
    M = sp.n_p * sp.n_phi
    if sp.kind == "lattice":
        n_t = math.ceil(sp.t_end / (0.5 * 7.0 / sp.n) - 1e-9)
        return sp.n * sp.n * M * n_t / 4e6
    n_t = math.ceil(sp.t_end / (0.9 * 0.22 * 1.3 / sp.n))
    return 2 * sp.n * sp.n * M * n_t / 1.5e7


def serve_oracle_baseline(specs, budget_s, workers):
    """CPU baseline of the serving stream: the FP64 oracle solves the cheapest
    requests that fit about budget_s seconds on `workers` host cores (one
    single-threaded process per core). Returns ({rid: QoIs}, solves/s, wall
    seconds, description)."""
    import multiprocessing as mp
    order = sorted(range(len(specs)), key=lambda i: oracle_request_cost(specs[i]))
    chosen, tot = [], 0.0
    seen = set()
    for i in order:
        sp = specs[i]
        dup = sp.kind == "lattice" and (sp.n, sp.n_p, sp.n_phi, sp.t_end) in seen
        c = 0.0 if dup else oracle_request_cost(sp)
        if tot + c > budget_s * workers:
            break
        chosen.append(i)
        tot += c
        if sp.kind == "lattice":
            seen.add((sp.n, sp.n_p, sp.n_phi, sp.t_end))
    # lattice requests with the same grid and ordinates are the same problem: solve each once
    key = lambda i: (specs[i].kind, specs[i].n, specs[i].n_p, specs[i].n_phi, specs[i].t_end,
                     i if specs[i].kind != "lattice" else -1)
    first = {}
    for i in chosen:
        first.setdefault(key(i), i)
    tasks = [(i, specs[i].kind, specs[i].n, specs[i].n_p, specs[i].n_phi, specs[i].t_end) for i in first.values()]
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    t0 = time.perf_counter()
    try:
        with mp.get_context("spawn").Pool(processes=workers) as pool:
            res = pool.map(_oracle_request, tasks, chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    wall = time.perf_counter() - t0
    by_key = {key(rid): q for rid, q, _ in res}
    out = {i: by_key[key(i)] for i in chosen}
    kinds = collections.Counter(f"{specs[i].kind} {specs[i].n}^2 x {specs[i].n_p * specs[i].n_phi}" for i in chosen)
    desc = (f"FP64 numpy oracle, {workers} single-threaded processes, the {len(chosen)} cheapest of the "
            f"{len(specs)} requests to their final times ({len(tasks)} distinct problems): "
            + ", ".join(f"{v} x {k}" for k, v in sorted(kinds.items())))
    return out, len(tasks) / wall if wall > 0 else None, wall, desc


def run_serve(args, w):
    import numpy as np
    import sn_inputs as si
    from paper_2505_17284_gb300 import build as B, rt
    from paper_2505_17284_gb300 import serve as SV
    from paper_2505_17284_gb300.sweep import qoi_rel_diff
    B.build()
    rt.load_library()
    count, horizon = w["count"], w["horizon"]
    policy = args.serve_policy
    # capacity: the whole stream present at the start (closed loop), FP32
    reqs, specs = serve_requests(rt, count, horizon, rt.RT_FP32)
    t0 = time.perf_counter()
    SV.Server(storage=rt.RT_FP32, policy=policy).run(reqs, realtime=False)
    cap = count / (time.perf_counter() - t0)
    rate = 0.8 * cap
    arr = si.poisson_arrivals(count, rate, seed=0)
    clocks = ClockSampler(0)
    clocks.start()
    res = {}
    for name, stor in (("fp32", rt.RT_FP32), ("bf16", rt.RT_BF16)):
        reqs, _ = serve_requests(rt, count, horizon, stor, arrivals=arr)
        srv = SV.Server(storage=stor, policy=policy)
        served = srv.run(reqs, realtime=True)
        res[name] = {"served": served, "span": max(s.finished for s in served), "launches": srv.launches}
    reqs, _ = serve_requests(rt, count, horizon, rt.RT_FP32, arrivals=arr)
    fifo = SV.serve_fifo(reqs, rt.RT_FP32, realtime=True)
    clk = clocks.stop()
    span_fifo = max(s.finished for s in fifo)
    q32 = {s.rid: s.qoi for s in res["fp32"]["served"]}
    q16 = {s.rid: s.qoi for s in res["bf16"]["served"]}
    qf = {s.rid: s.qoi for s in fifo}
    d_bf16 = [qoi_rel_diff(q16[i], q32[i]) for i in range(count)]
    d_plain = [qoi_rel_diff(q32[i], qf[i]) for i in range(count)]
    lat32 = [s.latency for s in res["fp32"]["served"]]
    lat16 = [s.latency for s in res["bf16"]["served"]]
    latf = [s.latency for s in fifo]
    pf, p32 = SV.percentiles(latf), SV.percentiles(lat32)

    def slowest(served, k=5):
        out = []
        for sv in sorted(served, key=lambda x: -x.latency)[:k]:
            sp = specs[sv.rid]
            out.append({"rid": sv.rid, "request": f"{sp.kind} {sp.n}^2 x {sp.n_p * sp.n_phi}",
                        "arrival": round(sv.arrival, 3), "start": round(sv.admitted, 3),
                        "finished": round(sv.finished, 3), "latency": round(sv.latency, 3)})
        return out
    out = {
        "metric": "served solves/s", "value": count / res["fp32"]["span"], "unit": "solves/s", "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": res["fp32"]["span"] * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded request stream)",
        "config": {"workload": args.workload, "requests": count, "arrivals": f"Poisson, seed 0, rate {rate:.3f}/s "
                   f"= 0.8 x closed-loop served capacity {cap:.3f}/s",
                   "mix": "50/50 lattice (n 70..700 step 70, MUSCL Heun) / enclosure triangles (n 130..650 step "
                          "130, first order Euler), M in {64,128,256,512}",
                   "end_times": f"lattice {3.2 * horizon:g}, enclosure {2.6 * horizon:g}"
                                + (" (the benchmarks' own)" if horizon == 1.0 else f" (x{horizon:g} of the benchmarks')"),
                   "scheduler": policy + (" (oldest first; younger requests join while the advanced set moves at "
                                          "most 2 GB of state per step and their remaining work is at most a quarter "
                                          "of the oldest one's; the rest held on the device)"
                                          if policy == "fcfs_fill" else " (every admitted request advances)"),
                   "admission": "free slot (64), device memory within 85% of the free HBM at start and within the "
                                "live free memory", "chunk_steps": 16, "step": "the whole stream"},
        "latency_s": {"fp32": p32, "bf16": SV.percentiles(lat16), "plain_fifo_fp32": pf},
        "solves_per_s": {"fp32": count / res["fp32"]["span"], "bf16": count / res["bf16"]["span"],
                         "plain_fifo_fp32": count / span_fifo},
        "slowest": {"fp32": slowest(res["fp32"]["served"]), "plain_fifo_fp32": slowest(fifo)},
        "p99_vs_plain": pf["p99"] / p32["p99"],
        "p50_vs_plain": pf["p50"] / p32["p50"],
        "qoi_rel_diff": {"bf16_vs_fp32_max": max(d_bf16), "bf16_vs_fp32_median": float(np.median(d_bf16)),
                         "served_fp32_vs_plain_max": max(d_plain)},
        "e2e": {"value": count / res["fp32"]["span"], "unit": "solves/s", "h2d_bytes_per_step": None,
                "d2h_bytes_per_step": count * QOI_BYTES, "includes": "problem build on the host, admission, all steps, "
                                                               "QoI read-back, removal"},
        "gpu_launches": {"fp32": res["fp32"]["launches"], "bf16": res["bf16"]["launches"],
                         "basis": "rt_batch_launches of the served batch: initial-state, stage and QoI-box launches "
                                  "(the plain FIFO server's launches not included)"},
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        workers = max(1, (os.cpu_count() or 2) - 1)
        oq, sps, wall, desc = serve_oracle_baseline(specs, args.serve_oracle_budget, workers)
        e32 = [qoi_rel_diff(q32[i], oq[i]) for i in sorted(oq)]
        e16 = [qoi_rel_diff(q16[i], oq[i]) for i in sorted(oq)]
        out["cpu_baseline"] = {"value": sps, "unit": "solves/s", "cores": workers, "kind": "oracle", "sample": desc,
                               "seconds": wall}
        out["qoi_rel_err_vs_oracle"] = {
            "requests": len(oq), "fp32": {"max": max(e32), "median": float(np.median(e32))},
            "bf16": {"max": max(e16), "median": float(np.median(e16))},
            "basis": "largest relative difference over mass, time-integrated absorption per region and outflow "
                     "(each at least 1e-3 of the balance scale) against the FP64 oracle, on the requests of the "
                     "cpu_baseline sample"}
    print(json.dumps(out))


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS) + sorted(EXTRA_WORKLOADS))
    ap.add_argument("--tile-x", type=int, default=0)
    ap.add_argument("--tile-y", type=int, default=0)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="Cartesian tiles from the library's model, not the autotuner")
    ap.add_argument("--profile-step", type=int, default=0,
                    help="sweeps: time one batched step of the first N instances and stop (for profilers)")
    ap.add_argument("--batch-tune", default="group", choices=["group", "shape"],
                    help="sweeps: tune kernel options per group of one ordinate count, or per ordinate count and grid")
    ap.add_argument("--profile-tuned", action="store_true",
                    help="with --profile-step: the per-group options of the sweep's tuner")
    ap.add_argument("--serve-policy", default="fcfs_fill", choices=["fcfs_fill", "all"])
    ap.add_argument("--serve-oracle-budget", type=float, default=150.0,
                    help="seconds of oracle work per host core for the serving stream's CPU baseline")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    return args


def main():
    args = parse_args()
    if args.workload in EXTRA_WORKLOADS:
        w = EXTRA_WORKLOADS[args.workload]
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle is timed on single solves "
                              "(the default workload); sweeps and streams are GPU-only reports"}))
            return
        (run_sweep if w["kind"] == "sweep" else run_serve)(args, w)
        return
    spec = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, spec)
    else:
        run_ours(args, spec)


if __name__ == "__main__":
    main()

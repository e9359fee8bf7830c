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

WORKLOADS = {
    # name: (mesh, n, n_p, n_phi, order, integrator, storage, dt_factor, t_end)
    "lattice1400_muscl_heun_fp32": ("lattice", 1400, 16, 32, 2, "heun", "fp32", 0.5, 3.2),
    "lattice1400_muscl_heun_bf16": ("lattice", 1400, 16, 32, 2, "heun", "bf16", 0.5, 3.2),
    "lattice1400_o1_euler_fp32": ("lattice", 1400, 16, 32, 1, "euler", "fp32", 0.5, 3.2),
    "enclosure1300_tri_o1_euler_fp32": ("enclosure", 1300, 8, 32, 1, "euler", "fp32", 0.0, 2.6),
    "lattice70_o1_euler_fp32": ("lattice", 70, 4, 16, 1, "euler", "fp32", 0.5, 3.2),
    "lattice560_muscl_heun_fp32": ("lattice", 560, 16, 32, 2, "heun", "fp32", 0.5, 3.2),
    "lattice840_muscl_heun_fp32": ("lattice", 840, 16, 32, 2, "heun", "fp32", 0.5, 3.2),
    "enclosure650_tri_o1_euler_fp32": ("enclosure", 650, 8, 32, 1, "euler", "fp32", 0.0, 2.6),
}
DEFAULT = "lattice1400_muscl_heun_fp32"


def bytes_per_update(order, integrator, storage):
    """Algorithmic HBM bytes per cell-ordinate per step (state traffic only):
    Euler reads psi^n and writes psi^{n+1}; Heun stage 1 reads psi^n and writes
    psi1, stage 2 reads psi1 and psi^n and writes psi^{n+1}."""
    es = 2 if storage == "bf16" else 4
    return (2 if integrator == "euler" else 5) * es


KERNEL_SOURCES = {"cart": ["cart_kernel.cuh", "device_common.cuh"], "tri": ["tri_kernel.cu", "device_common.cuh"]}


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
def oracle_sample(spec, budget_s):
    """Time the FP64 oracle (single thread) on a bounded sample of the workload:
    the same scheme and ordinate set on a smaller grid, sized to about budget_s
    seconds of work; returns (updates/s, description, seconds)."""
    code = r"""
import json, sys, time, numpy as np
sys.path.insert(0, %r)
import oracle, sn_inputs as si
mesh, n_full, n_p, n_phi, order, integ, storage, dtf, t_end = %r
budget = %r
def build(n):
    if mesh == "lattice":
        p = si.lattice_problem(n); dt = dtf * p.mesh.dx
        op = oracle.CartesianOracle(p, oracle.product_quadrature(n_p, n_phi), order=order)
    else:
        p = si.enclosure_problem(n, jitter=0.2, seed=0)
        op = oracle.TriangleOracle(p, oracle.product_quadrature(n_p, n_phi))
        dt = oracle.triangle_dt(op, t_end)[1]
    return p, op, dt
n = 14 if mesh == "lattice" else 10
p, op, dt = build(n)
psi = np.zeros((p.mesh.n_cells, n_p * n_phi))
t0 = time.perf_counter(); oracle.run(op, psi, dt, 1, integ); t1 = time.perf_counter()
rate = p.mesh.n_cells * n_p * n_phi / (t1 - t0)
steps = 3
n2 = int(max(14, min(n_full, (rate * budget / steps / (n_p * n_phi)) ** 0.5 / (1 if mesh == "lattice" else 1.41))))
if mesh == "lattice": n2 = max(7, n2 // 7 * 7)
p, op, dt = build(n2)
psi = np.zeros((p.mesh.n_cells, n_p * n_phi))
t0 = time.perf_counter(); oracle.run(op, psi, dt, steps, integ); t1 = time.perf_counter()
print(json.dumps({"rate": p.mesh.n_cells * n_p * n_phi * steps / (t1 - t0), "n": n2, "steps": steps,
                  "cells": p.mesh.n_cells, "seconds": t1 - t0}))
""" % (ROOT, list(spec), budget_s)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle baseline failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    mesh = spec[0]
    desc = (f"FP64 numpy oracle, 1 thread: {'lattice' if mesh == 'lattice' else 'enclosure triangles'} "
            f"{d['n']}x{d['n']} ({d['cells']} cells) x {spec[2] * spec[3]} ordinates, {d['steps']} steps of the "
            f"same scheme; rate scaled per cell-ordinate update")
    return d["rate"], desc, d["seconds"]


# ------------------------------------------------------------------ ours
def run_ours(args, spec):
    import numpy as np
    import torch
    from paper_2505_17284_gb300 import build as B, rt

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
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
    quad = rt.rt_quad_product(n_p, n_phi)
    integ_c = rt.RT_HEUN if integ == "heun" else rt.RT_EULER
    stor_c = rt.RT_BF16 if storage == "bf16" else rt.RT_FP32
    solver = rt.Solver(problem, quad, order=order, integrator=integ_c, storage=stor_c, dt=dt,
                       tile_x=args.tile_x, tile_y=args.tile_y)
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
    if dist:
        t = torch.tensor([ms], device="cuda")
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        ms = float(t.item())
    dof = info.n_cells * info.M
    updates = dof * K * world
    value = updates / (ms * 1e-3)
    bpu = bytes_per_update(order, integ, storage)
    launches_per_step = info.stages_per_step
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
                   tile_x=args.tile_x, tile_y=args.tile_y)
    s2.step(K)
    q2 = s2.qoi()
    s2.close()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    n_cells = info.n_cells
    if mesh == "lattice":
        h2d = 2 * n_cells + 3 * info.M_pad * 4
    else:
        h2d = n_cells * (16 + 32) + 3 * info.M_pad * 4
    d2h = 336

    tb, traffic_src = profiled_traffic(args.workload, "cart" if mesh == "lattice" else "tri")
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
                   "l2": f"inputs larger than L2 (psi {dof * (2 if storage == 'bf16' else 4) / 1e9:.2f} GB per buffer)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": peak, "unit": "GB/s",
                     "frac": achieved_gbs / peak, "traffic": traffic,
                     "traffic_per": "step (all stage launches), DRAM read + write bytes",
                     "traffic_source": traffic_src,
                     "kernel": "cart_stage_kernel" if mesh == "lattice" else "tri_stage_kernel",
                     "bytes_per_update": bpu, "peak_source": f"{peak_src} hbm_gbs",
                     "achieved_basis": "algorithmic bytes per cell-ordinate x cell-ordinates x steps / event time of the steps"},
        "e2e": {"value": dof * K / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h / K,
                "seconds": e2e_s, "includes": "rt_create from host arrays + K steps + rt_qoi read-back + rt_destroy"},
        "gpu_launches": K * launches_per_step,
        "clocks": clk,
        "qoi_after": {"step": q["step"], "abs_int_blue": float(q["abs_int"][1]) if mesh == "lattice" else None,
                      "mass": q["mass"]},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, desc, secs = oracle_sample(spec, budget_s=args.cpu_budget)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
                               "seconds": secs}
    if dist:
        tdist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def run_reference(args, spec):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    K, W = args.steps, args.warmup
    per_step = max(0.5, min(20.0, 150.0 / (K + W)))
    import numpy as np
    import oracle
    import sn_inputs as si
    mesh, n_full, n_p, n_phi, order, integ, storage, dtf, t_end = spec
    # size the sample so that one step costs about per_step seconds
    def build(n):
        if mesh == "lattice":
            p = si.lattice_problem(n)
            op = oracle.CartesianOracle(p, oracle.product_quadrature(n_p, n_phi), order=order)
            return p, op, dtf * p.mesh.dx
        p = si.enclosure_problem(n, jitter=0.2, seed=0)
        op = oracle.TriangleOracle(p, oracle.product_quadrature(n_p, n_phi))
        return p, op, oracle.triangle_dt(op, t_end)[1]
    p, op, dt = build(14 if mesh == "lattice" else 10)
    M = n_p * n_phi
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--tile-x", type=int, default=0)
    ap.add_argument("--tile-y", type=int, default=0)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    spec = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, spec)
    else:
        run_ours(args, spec)


if __name__ == "__main__":
    main()

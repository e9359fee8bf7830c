"""Batched parameter sweeps.

Many independent problems solved together through the batch entry points (one
launch per stage over the work items of every unfinished problem, replayed as
a captured CUDA graph while the membership holds), against the same problems
solved one at a time through the single-problem entry points (create, step to
N_t, read the QoIs, destroy). The paper's design-parameter studies (Sec. 3.1.3)
are sweeps of this kind; the paper itself solves them one at a time.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import rt


@dataclass
class Job:
    """One problem of a sweep: geometry/materials (sn_inputs.Problem), a
    quadrature (xi, eta, mu, w), the scheme and the target step (0 = default)."""
    problem: object
    quad: tuple
    order: int = 2
    integrator: int = rt.RT_HEUN
    dt: float = 0.0

    @property
    def n_cells(self) -> int:
        return self.problem.mesh.n_cells

    @property
    def M(self) -> int:
        return len(self.quad[0])


def _sync():
    import torch
    torch.cuda.synchronize()


def solve_plain(jobs, storage=rt.RT_FP32, tune=True):
    """Solve the jobs one after another (a fresh solver each). Returns (QoI
    dicts, total seconds, seconds per job, steps per job)."""
    out, per, steps = [], [], []
    _sync()
    t0 = time.perf_counter()
    for j in jobs:
        a = time.perf_counter()
        s = rt.Solver(j.problem, j.quad, order=j.order, integrator=j.integrator, storage=storage, dt=j.dt, tune=tune)
        s.step()
        out.append(s.qoi())
        steps.append(int(s.info.n_steps))
        s.close()
        per.append(time.perf_counter() - a)
    _sync()
    return out, time.perf_counter() - t0, per, steps


def solve_batched(jobs, storage=rt.RT_FP32, tile_y=0, phases=None, configs=None):
    """Solve the jobs together in one batch. Returns (QoI dicts, seconds from
    batch creation to the last QoI read, steps per job); `phases`, if a dict,
    receives the seconds of creation, stepping and read-back and the kernel
    launches of the batch (rt_batch_launches). `configs`: per-job
    kernel options (dicts of tile_y / variant / vec, as from tune_groups)."""
    _sync()
    t0 = time.perf_counter()
    b = _batch(jobs, storage, tile_y, configs)
    _sync()
    t1 = time.perf_counter()
    b.run()
    _sync()
    t2 = time.perf_counter()
    out = [b.qoi(i) for i in range(len(jobs))]
    launches = b.launches()
    b.close()
    _sync()
    t3 = time.perf_counter()
    if phases is not None:
        phases.update(create=t1 - t0, run=t2 - t1, read_and_destroy=t3 - t2, gpu_launches=launches)
    return out, t3 - t0, [q["n_steps"] for q in out]


def _batch(jobs, storage, tile_y=0, configs=None):
    return rt.Batch([j.problem for j in jobs], [j.quad for j in jobs], storage=storage, dts=[j.dt for j in jobs],
                    orders=[j.order for j in jobs], integrators=[j.integrator for j in jobs], tile_y=tile_y,
                    configs=configs)


def _ms_per_step(jobs, storage, steps, tile_y=0, configs=None):
    """CUDA-event milliseconds per batch step after one warm-up step; None if
    the options are invalid for some member (RT_EINVAL)."""
    import torch
    try:
        b = _batch(jobs, storage, tile_y, configs)
    except rt.RTError as e:
        if e.code != rt.RT_EINVAL:
            raise
        return None
    b.step(1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    b.step(steps)
    e1.record()
    torch.cuda.synchronize()
    b.close()
    return e0.elapsed_time(e1) / steps


def group_key(j):
    """Jobs that share a kernel-variant group of the batch under every option:
    the same ordinate count, order and integrator."""
    return (j.M, j.order, j.integrator)


def tune_groups(jobs, storage=rt.RT_FP32, tile_ys=(0, 16, 24, 32, 48), variants=(0, 1), steps=3, by_shape=False):
    """Per-group tuner: for each group of jobs with one ordinate count, order
    and integrator (and, with by_shape, one cell count), the (tile_y, variant)
    pair with the shortest batch step, timed on that group's jobs alone. Small
    grids with 4 quadrants of 64 ordinates, for example, run faster on the
    per-lane-direction kernel (variant 1) than on the chunk-uniform one the
    library picks for large grids. Returns (per-job config dicts, {group:
    {"tile_y/variant": ms}})."""
    groups = {}
    for i, j in enumerate(jobs):
        groups.setdefault(group_key(j) + ((j.n_cells,) if by_shape else ()), []).append(i)
    configs = [None] * len(jobs)
    table = {}
    for key, idx in groups.items():
        sub = [jobs[i] for i in idx]
        times = {}
        for ty in tile_ys:
            for var in variants:
                cf = {"tile_y": ty, "variant": var}
                ms = _ms_per_step(sub, storage, steps, configs=[cf] * len(sub))
                if ms is not None:
                    times[(ty, var)] = ms
        if not times:
            raise ValueError(f"no (tile_y, variant) pair is valid for the jobs with M, order, integrator = {key}")
        best = min(times, key=times.get)
        for i in idx:
            configs[i] = {"tile_y": best[0], "variant": best[1]}
        name = "M%d_o%d_%s" % (key[0], key[1], "heun" if key[2] == rt.RT_HEUN else "euler")
        table[name + ("_cells%d" % key[3] if by_shape else "")] = {
            "best": {"tile_y": best[0], "variant": best[1]},
            "ms_per_step": {"%d/%d" % tv: round(ms, 4) for tv, ms in times.items()}}
    return configs, table


def tune_batch(jobs, storage=rt.RT_FP32, candidates=(0, 16, 24, 32, 48, 64), steps=4):
    """Batch-level tuner: the segment length shared by the batch's Cartesian
    problems, timed with CUDA events over `steps` steps of the whole batch
    after one warm-up step. Returns (best tile_y, {tile_y: ms per step})."""
    times = {}
    for ty in candidates:
        ms = _ms_per_step(jobs, storage, steps, tile_y=ty)
        if ms is not None:   # None: segment too long for the shared memory of some member
            times[ty] = ms
    best = min(times, key=times.get)
    return best, times


def state_bytes(jobs, steps, storage=rt.RT_FP32, bytes_per_update=None):
    """Algorithmic HBM bytes of solving the jobs: per cell-ordinate and step,
    Euler reads psi^n and writes psi^(n+1) (2 values), Heun moves 5 values."""
    es = 2 if storage == rt.RT_BF16 else 4
    tot = 0.0
    for j, n in zip(jobs, steps):
        per = bytes_per_update if bytes_per_update else (5 if j.integrator == rt.RT_HEUN else 2) * es
        tot += float(j.n_cells) * j.M * n * per
    return tot


def qoi_rel_diff(a: dict, b: dict) -> float:
    """Largest relative difference between two results of the final mass and
    the time-integrated QoIs (absorption per region, boundary outflow). Each
    is relative to its own size but at least 1e-3 of the problem's balance
    scale max(mass, sum of absorption, |outflow|) (the three terms of the
    particle balance), as in the parity tests: a QoI that is still tiny (an
    absorber or boundary the wave has barely reached) carries the rounding of
    the state near it, not an error of its own."""
    ai, bi = np.atleast_1d(a["abs_int"]), np.atleast_1d(b["abs_int"])
    scale = max(abs(b["mass"]), float(np.sum(np.abs(bi))), abs(b["outflow_int"]), 1e-300)
    floor = 1e-3 * scale
    d = abs(a["mass"] - b["mass"]) / max(abs(b["mass"]), floor)
    for x, y in zip(ai, bi):
        d = max(d, abs(x - y) / max(abs(y), floor))
    d = max(d, abs(a["outflow_int"] - b["outflow_int"]) / max(abs(b["outflow_int"]), floor))
    return d

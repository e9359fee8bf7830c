"""Serving loop with continuous batching.

Solve requests arrive over time. The server keeps one batch of slots on the
GPU: an arrived request is admitted (its problem built, its state created and
initialised on the device) as soon as a slot is free and its device memory
fits both the server's budget and the device memory free at that moment; a
problem that reaches its own N_t is retired (QoIs read back, memory freed)
and its slot and memory go to the next request. State stays on the device
from admission to retirement. Latency is retirement time minus arrival time.

Which admitted problems the shared launches advance is the scheduler's
choice (policy "fcfs_fill", the default): the oldest request always runs,
and younger ones join it, oldest first, while the per-step state traffic of
the chosen set stays within `fill_bytes` and the remaining work of the joiners
(state traffic of their remaining steps) adds up to at most `join_share` of
the oldest one's; the others are held on the device (rt_batch_hold) until
capacity frees up. Large requests thus run in arrival order at nearly the
speed they would have alone (two large ones never share the GPU, which would
delay the older one's finish and stretch the tail), while small requests ride
along and finish early. Policy "all" advances every admitted problem together
(processor sharing, which stretches large requests by the number sharing the
GPU).

The plain baseline is a first-in first-out server that solves one request
at a time with the single-problem entry points, run against the same arrival
times (serve_fifo).
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
from typing import Callable

import numpy as np

from . import rt
from .sweep import Job


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the stream
    make: Callable[[], Job]        # builds the job (host work, counted in the latency)
    est_bytes: int                 # device memory to reserve at admission


@dataclass
class Served:
    rid: int
    arrival: float
    admitted: float
    finished: float
    qoi: dict
    slot: int = -1

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def estimate_bytes(n_cells: int, M: int, storage=rt.RT_FP32, triangles=False, order=1) -> int:
    """Upper estimate of a problem's device memory: two psi buffers (ordinates
    padded to 32), two phi buffers and per-cell metadata (larger for
    triangles: neighbours, edge geometry, areas), plus fixed overhead; second
    order on triangles adds the limited gradient (two FP32 values per cell and
    ordinate) and its reconstruction geometry."""
    es = 2 if storage == rt.RT_BF16 else 4
    Mpad = (M + 31) // 32 * 32
    per_cell = 2 * Mpad * es + 16 + (96 if triangles else 8)
    if triangles and order == 2:
        per_cell += 2 * Mpad * 4 + 48
    return int(n_cells * per_cell + (8 << 20))


def step_bytes(job, storage=rt.RT_FP32) -> float:
    """Algorithmic state bytes one time step of a job moves (psi reads and
    writes; Heun 5 values per cell and ordinate, Euler 2)."""
    es = 2 if storage == rt.RT_BF16 else 4
    Mpad = (job.M + 31) // 32 * 32
    return float(job.n_cells) * Mpad * es * (5 if job.integrator == rt.RT_HEUN else 2)


def live_free_bytes() -> int:
    """Device memory available right now: free in the driver plus what
    PyTorch's caching allocator holds but does not use."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    return int(free + torch.cuda.memory_reserved() - torch.cuda.memory_allocated())


@dataclass
class Server:
    storage: int = rt.RT_FP32
    capacity: int = 64             # slots
    chunk: int = 16                # steps per enqueue
    policy: str = "fcfs_fill"      # or "all" (every admitted problem advances)
    fill_bytes: float = 2.0e9      # per-step state traffic of the advanced set (fcfs_fill)
    join_share: float = 0.25       # joiners' remaining work, at most this share of the oldest's
    mem_fraction: float = 0.85     # of the device memory free at start: the server's budget
    reserve: int = 2 << 30         # bytes kept free for the allocator's own use
    max_ahead: int = 2             # chunks enqueued ahead of the device
    log: list = field(default_factory=list)
    launches: int = 0              # kernel launches of the last run (rt_batch_launches)

    def select(self, active, weight, remaining):
        """Slots to advance: all (policy "all"), or the oldest, joined in
        arrival order by requests that keep the per-step traffic within
        fill_bytes and whose remaining work fits in join_share of the
        oldest's remaining work."""
        order = sorted(active, key=lambda s: (active[s][0].arrival, active[s][0].rid))
        if self.policy == "all":
            return set(order)
        first = order[0]
        chosen, acc = {first}, weight[first]
        left = self.join_share * weight[first] * remaining[first]
        for s in order[1:]:
            work = weight[s] * remaining[s]
            if acc + weight[s] <= self.fill_bytes and work <= left:
                chosen.add(s)
                acc += weight[s]
                left -= work
        return chosen

    def run(self, requests, realtime=True):
        """Serve `requests` (arrival times relative to the start); with
        realtime=False every request is present at the start (closed loop).
        Returns the list of Served, in completion order."""
        import torch
        free, _ = torch.cuda.mem_get_info()
        budget = int(free * self.mem_fraction) - self.reserve
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        active = {}                     # slot -> (request, admitted time, bytes)
        weight = {}                     # slot -> state bytes per step
        held = set()
        used = 0
        events = collections.deque()
        done = []
        b = rt.Batch([], [], storage=self.storage, capacity=self.capacity)
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        try:
            while pending or waiting or active:
                t = now()
                while pending and (not realtime or pending[0].arrival <= t):
                    waiting.append(pending.popleft())
                while (waiting and len(active) < self.capacity and used + waiting[0].est_bytes <= budget
                       and waiting[0].est_bytes + self.reserve <= live_free_bytes()):
                    r = waiting.popleft()
                    j = r.make()
                    slot = b.add(j.problem, j.quad, order=j.order, integrator=j.integrator, dt=j.dt)
                    active[slot] = (r, now(), r.est_bytes)
                    weight[slot] = step_bytes(j, self.storage)
                    used += r.est_bytes
                if not active:
                    if waiting:
                        raise RuntimeError(f"request {waiting[0].rid} needs {waiting[0].est_bytes} bytes, "
                                           f"more than the budget of {budget}")
                    if pending:
                        time.sleep(max(0.0, pending[0].arrival - now()))
                    continue
                remaining = {}
                for slot in active:
                    d, n = b.progress(slot)
                    remaining[slot] = n - d
                run = self.select(active, weight, remaining)
                for slot in active:
                    h = slot not in run
                    if h != (slot in held):
                        b.hold(slot, h)
                        (held.add if h else held.discard)(slot)
                b.step(self.chunk)
                ev = torch.cuda.Event()
                ev.record()
                events.append(ev)
                finished = []
                for slot in run:
                    d, n = b.progress(slot)
                    if d >= n:
                        finished.append(slot)
                if finished:
                    for slot in finished:
                        q = b.qoi(slot)          # synchronises
                        r, adm, nb = active.pop(slot)
                        weight.pop(slot)
                        held.discard(slot)
                        done.append(Served(r.rid, r.arrival, adm, now(), q, slot))
                        b.remove(slot)
                        used -= nb
                    events.clear()
                elif len(events) > self.max_ahead:
                    events.popleft().synchronize()
        finally:
            try:
                self.launches = b.launches()
            finally:
                b.close()
        return done


def serve_fifo(requests, storage=rt.RT_FP32, realtime=True, tune=False):
    """The plain server: first in, first out, one request at a time through
    the single-problem entry points (build, create, step to N_t, read the QoIs,
    destroy), against the requests' arrival times. Returns the list of Served
    in completion order."""
    import torch
    pending = sorted(requests, key=lambda r: r.arrival)
    done = []
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0
    for r in pending:
        if realtime and r.arrival > now():
            time.sleep(r.arrival - now())
        start = now()
        j = r.make()
        s = rt.Solver(j.problem, j.quad, order=j.order, integrator=j.integrator, storage=storage, dt=j.dt, tune=tune)
        s.step()
        q = s.qoi()
        s.close()
        torch.cuda.synchronize()
        done.append(Served(r.rid, r.arrival, start, now(), q))
    return done


def plain_service_times(requests, storage=rt.RT_FP32, tune=False):
    """Solve every request alone, one after another; returns ({rid: seconds},
    {rid: QoIs}). Each time covers building the job, creating the solver,
    stepping to N_t, reading the QoIs and destroying it."""
    import torch
    times, qois = {}, {}
    for r in requests:
        torch.cuda.synchronize()
        a = time.perf_counter()
        j = r.make()
        s = rt.Solver(j.problem, j.quad, order=j.order, integrator=j.integrator, storage=storage, dt=j.dt, tune=tune)
        s.step()
        qois[r.rid] = s.qoi()
        s.close()
        torch.cuda.synchronize()
        times[r.rid] = time.perf_counter() - a
    return times, qois


def fifo_latencies(requests, service):
    """Latencies of a single first-in first-out server with the given service
    times, for the requests' arrival times."""
    end = 0.0
    lat = {}
    for r in sorted(requests, key=lambda r: r.arrival):
        start = max(r.arrival, end)
        end = start + service[r.rid]
        lat[r.rid] = end - r.arrival
    return lat, end


def percentiles(values, ps=(50, 99)):
    v = np.asarray(list(values), dtype=float)
    return {f"p{p}": float(np.percentile(v, p)) for p in ps}

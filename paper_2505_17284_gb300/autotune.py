"""Autotuned Cartesian kernel configurations, cached per device and problem shape.

The timing is native (rt_autotune: every candidate strip width, segment length
and direction family is built as a solver and timed with CUDA events); this
module keys the winners by device and problem shape and keeps them in a JSON
file, so that each shape is tuned once per device. The configuration does not
depend on material values, only on the grid, the ordinate count, the scheme and
the storage type.
"""
from __future__ import annotations

import json
import os
import threading

from . import rt

_PKG = os.path.dirname(os.path.abspath(__file__))
CACHE_PATH = os.environ.get("RT_GB300_TUNE_CACHE", os.path.join(_PKG, "tune_cache.json"))
_lock = threading.Lock()
_mem: dict | None = None


def device_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|sm{p.multi_processor_count}"


def shape_key(problem, M: int, order: int, integrator: int, storage: int) -> str:
    m = problem.mesh
    return f"{device_key()}|cart{m.nx}x{m.ny}|M{M}|o{order}|i{integrator}|s{storage}"


def _load() -> dict:
    global _mem
    if _mem is None:
        try:
            with open(CACHE_PATH) as fh:
                _mem = json.load(fh)
        except (OSError, ValueError):
            _mem = {}
    return _mem


def _save(d: dict):
    tmp = CACHE_PATH + f".{os.getpid()}.tmp"
    try:
        with open(tmp, "w") as fh:
            json.dump(d, fh, indent=1, sort_keys=True)
        os.replace(tmp, CACHE_PATH)
    except OSError:
        pass   # a read-only location: keep the in-memory cache only


def tuned_config(problem, quad, order, integrator, storage=rt.RT_FP32, dt=0.0, t_end=None, steps=4,
                 refresh=False) -> dict:
    """{tile_x, tile_y, variant, vec, ms_per_step} for this problem shape on the
    current device: from the cache, else from rt_autotune (then cached)."""
    key = shape_key(problem, len(quad[0]), order, integrator, storage)
    with _lock:
        d = _load()
        if not refresh and key in d:
            return dict(d[key])
    cfg, ms = rt.rt_autotune(problem, quad, order, integrator, storage, dt, t_end, steps)
    cfg["ms_per_step"] = ms
    with _lock:
        d = _load()
        d[key] = cfg
        _save(d)
    return dict(cfg)


def clear_cache():
    global _mem
    with _lock:
        _mem = {}
        try:
            os.remove(CACHE_PATH)
        except OSError:
            pass

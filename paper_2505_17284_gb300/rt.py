"""Thin Python binding of the C ABI declared in include/rt.h.

The functions keep the C names (rt_create, rt_step, rt_qoi, ...) and only
marshal arguments; every step of the S_N path runs in the CUDA kernels of
librt_gb300.so. Loading fails loudly when the library has not been built.

`Solver` and `Batch` are small conveniences over the same calls: they build
the C structs from numpy arrays, allocate device memory through PyTorch's
caching allocator (callbacks handed to the library) and enqueue on PyTorch's
current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "librt_gb300.so")

RT_OK, RT_EINVAL, RT_ENOMEM, RT_ECUDA, RT_ETIMEOUT, RT_ENONFINITE, RT_ESTATE = range(7)
RT_MESH_CARTESIAN, RT_MESH_TRIANGLES = 0, 1
RT_BC_VACUUM, RT_BC_INFLOW, RT_BC_PERIODIC = 0, 1, 2
RT_EULER, RT_HEUN = 0, 1
RT_FP32, RT_BF16 = 0, 1
RT_MAX_REGIONS = 16
RT_MAX_BOXES = 4
STATUS_NAMES = {0: "RT_OK", 1: "RT_EINVAL", 2: "RT_ENOMEM", 3: "RT_ECUDA", 4: "RT_ETIMEOUT",
                5: "RT_ENONFINITE", 6: "RT_ESTATE"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class rt_mesh(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32),
                ("x0", C.c_double), ("y0", C.c_double), ("dx", C.c_double), ("dy", C.c_double),
                ("n_vert", C.c_int64), ("vxy", _dp), ("n_tri", C.c_int64), ("tri", _ip)]


class rt_materials(C.Structure):
    _fields_ = [("n_mat", C.c_int32), ("sigma_a", _dp), ("sigma_s", _dp), ("Q", _dp),
                ("cell_mat", _ip), ("cell_region", _ip), ("n_regions", C.c_int32),
                ("n_boxes", C.c_int32), ("boxes", _dp)]


class rt_quadrature(C.Structure):
    _fields_ = [("M", C.c_int64), ("xi", _dp), ("eta", _dp), ("w", _dp)]


class rt_boundary(C.Structure):
    _fields_ = [("side_kind", C.c_int32 * 4), ("inflow", C.c_double * 4)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class rt_options(C.Structure):
    _fields_ = [("order", C.c_int32), ("integrator", C.c_int32), ("storage", C.c_int32),
                ("tile_x", C.c_int32), ("tile_y", C.c_int32), ("variant", C.c_int32),
                ("dt", C.c_double), ("t_end", C.c_double),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p), ("stream", C.c_void_p),
                ("vec", C.c_int32), ("pad", C.c_int32)]


class rt_qoi_t(C.Structure):
    _fields_ = [("t", C.c_double), ("step", C.c_int64), ("n_steps", C.c_int64),
                ("n_regions", C.c_int32), ("status", C.c_int32),
                ("abs_now", C.c_double * RT_MAX_REGIONS), ("abs_int", C.c_double * RT_MAX_REGIONS),
                ("mass", C.c_double), ("outflow_now", C.c_double), ("outflow_int", C.c_double),
                ("source_int", C.c_double), ("n_boxes", C.c_int32), ("pad", C.c_int32),
                ("box_out_now", C.c_double * RT_MAX_BOXES), ("box_out_int", C.c_double * RT_MAX_BOXES)]


class rt_info_t(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("M", C.c_int64), ("M_pad", C.c_int64), ("n_steps", C.c_int64),
                ("dt", C.c_double), ("t_end", C.c_double),
                ("kind", C.c_int32), ("order", C.c_int32), ("integrator", C.c_int32), ("storage", C.c_int32),
                ("tile_x", C.c_int32), ("tile_y", C.c_int32), ("n_work_items", C.c_int32),
                ("stages_per_step", C.c_int32), ("device_bytes", C.c_int64), ("variant", C.c_int32),
                ("vec", C.c_int32), ("regrouped", C.c_int32), ("n_box_items", C.c_int32)]


class rt_problem(C.Structure):
    _fields_ = [("mesh", rt_mesh), ("mat", rt_materials), ("quad", rt_quadrature), ("bc", rt_boundary),
                ("order", C.c_int32), ("integrator", C.c_int32), ("dt", C.c_double), ("t_end", C.c_double),
                ("tile_y", C.c_int32), ("variant", C.c_int32), ("vec", C.c_int32), ("pad", C.c_int32)]


RT_STAGE_EULER, RT_STAGE_HEUN1, RT_STAGE_HEUN2 = 0, 1, 2
RT_NOALLOC_MAX_WORK_ITEMS = 8192
RT_MAX_MATERIALS = 64


class rt_cart_stage_args(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("dx", C.c_double), ("dy", C.c_double),
                ("M_pad", C.c_int32), ("vec", C.c_int32), ("order", C.c_int32), ("stage", C.c_int32),
                ("storage", C.c_int32), ("tile_y", C.c_int32), ("n_mat", C.c_int32), ("n_regions", C.c_int32),
                ("sigma_a", C.c_double * RT_MAX_MATERIALS), ("sigma_s", C.c_double * RT_MAX_MATERIALS),
                ("Q", C.c_double * RT_MAX_MATERIALS),
                ("inflow", C.c_double * 4), ("dt", C.c_double),
                ("psi_in", C.c_void_p), ("psi_n", C.c_void_p), ("psi_out", C.c_void_p),
                ("phi_in", C.c_void_p), ("phi_out", C.c_void_p), ("cell_mat", C.c_void_p),
                ("cell_region", C.c_void_p), ("xi", C.c_void_p), ("eta", C.c_void_p), ("w", C.c_void_p),
                ("qoi_out", C.c_void_p), ("status_out", C.c_void_p), ("stream", C.c_void_p),
                ("step", C.c_int64), ("xi_host", C.POINTER(C.c_float))]


# exported functions: name -> (restype, argtypes)
SIGNATURES = {
    "rt_quad_product": (C.c_int, [C.c_int32, C.c_int32, _dp, _dp, _dp, _dp]),
    "rt_quad_tessellation": (C.c_int, [C.c_int32, _dp, _dp, _dp, _dp]),
    "rt_create": (C.c_int, [C.POINTER(rt_mesh), C.POINTER(rt_materials), C.POINTER(rt_quadrature),
                            C.POINTER(rt_boundary), C.POINTER(rt_options), C.POINTER(C.c_void_p)]),
    "rt_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "rt_qoi": (C.c_int, [C.c_void_p, C.POINTER(rt_qoi_t)]),
    "rt_info": (C.c_int, [C.c_void_p, C.POINTER(rt_info_t)]),
    "rt_get_psi": (C.c_int, [C.c_void_p, _dp, C.c_int64]),
    "rt_get_psi_cells": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.c_int64, _dp]),
    "rt_get_phi": (C.c_int, [C.c_void_p, _dp, C.c_int64]),
    "rt_set_psi": (C.c_int, [C.c_void_p, _dp, C.c_int64]),
    "rt_device_state": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_int32)]),
    "rt_state_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "rt_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "rt_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "rt_debug_set": (C.c_int, [C.c_void_p, C.c_char_p, C.c_int64]),
    "rt_destroy": (None, [C.c_void_p]),
    "rt_last_error": (C.c_char_p, []),
    "rt_batch_create": (C.c_int, [C.c_int32, C.POINTER(rt_problem), C.c_int32, C.POINTER(rt_options),
                                  C.POINTER(C.c_void_p)]),
    "rt_batch_add": (C.c_int, [C.c_void_p, C.POINTER(rt_problem), C.POINTER(C.c_int32)]),
    "rt_batch_remove": (C.c_int, [C.c_void_p, C.c_int32]),
    "rt_batch_hold": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "rt_batch_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "rt_batch_progress": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "rt_batch_launches": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "rt_batch_run": (C.c_int, [C.c_void_p, C.c_int64]),
    "rt_batch_qoi": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(rt_qoi_t)]),
    "rt_batch_get_psi": (C.c_int, [C.c_void_p, C.c_int32, _dp, C.c_int64]),
    "rt_batch_destroy": (None, [C.c_void_p]),
    "rt_cart_stage_noalloc": (C.c_int, [C.POINTER(rt_cart_stage_args)]),
    "rt_autotune": (C.c_int, [C.POINTER(rt_mesh), C.POINTER(rt_materials), C.POINTER(rt_quadrature),
                              C.POINTER(rt_boundary), C.POINTER(rt_options), C.c_int32, C.POINTER(rt_options),
                              C.POINTER(C.c_double)]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load librt_gb300.so and declare its signatures; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2505_17284_gb300.build.build() "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _fns():
    return load_library()


class RTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code):
    if code != RT_OK:
        raise RTError(code, _fns().rt_last_error().decode())
    return code


# -- thin wrappers with the C names ------------------------------------------------------
def rt_quad_product(n_p: int, n_phi: int):
    M = n_p * n_phi
    xi, eta, mu, w = (np.zeros(M) for _ in range(4))
    check(_fns().rt_quad_product(n_p, n_phi, _ptr(xi), _ptr(eta), _ptr(mu), _ptr(w)))
    return xi, eta, mu, w


def rt_quad_tessellation(N: int):
    M = 4 * N * N
    xi, eta, mu, w = (np.zeros(M) for _ in range(4))
    check(_fns().rt_quad_tessellation(N, _ptr(xi), _ptr(eta), _ptr(mu), _ptr(w)))
    return xi, eta, mu, w


def rt_create(mesh, mat, quad, bc, opts):
    h = C.c_void_p()
    check(_fns().rt_create(C.byref(mesh), C.byref(mat), C.byref(quad), C.byref(bc), C.byref(opts), C.byref(h)))
    return h


def rt_step(h, n: int):
    return check(_fns().rt_step(h, int(n)))


def rt_qoi(h) -> rt_qoi_t:
    q = rt_qoi_t()
    check(_fns().rt_qoi(h, C.byref(q)))
    return q


def rt_info(h) -> rt_info_t:
    i = rt_info_t()
    check(_fns().rt_info(h, C.byref(i)))
    return i


def rt_get_psi(h, n_cells: int, M: int) -> np.ndarray:
    out = np.empty((n_cells, M))
    check(_fns().rt_get_psi(h, _ptr(out), out.size))
    return out


def rt_get_psi_cells(h, cells, M: int) -> np.ndarray:
    idx = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
    out = np.empty((idx.size, M))
    check(_fns().rt_get_psi_cells(h, idx.ctypes.data_as(C.POINTER(C.c_int64)), idx.size, _ptr(out)))
    return out


def rt_get_phi(h, n_cells: int) -> np.ndarray:
    out = np.empty(n_cells)
    check(_fns().rt_get_phi(h, _ptr(out), out.size))
    return out


def rt_set_psi(h, psi: np.ndarray):
    a = np.ascontiguousarray(psi, dtype=np.float64)
    return check(_fns().rt_set_psi(h, _ptr(a), a.size))


def rt_device_state(h):
    p, f, s = C.c_void_p(), C.c_void_p(), C.c_int32()
    check(_fns().rt_device_state(h, C.byref(p), C.byref(f), C.byref(s)))
    return p.value, f.value, s.value


def rt_get_state(h) -> bytes:
    n = C.c_size_t()
    check(_fns().rt_state_size(h, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    check(_fns().rt_get_state(h, buf, n.value))
    return buf.raw


def rt_set_state(h, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    return check(_fns().rt_set_state(h, buf, len(blob)))


def rt_debug_set(h, key: str, value: int):
    return check(_fns().rt_debug_set(h, key.encode(), int(value)))


def rt_destroy(h):
    if h:
        _fns().rt_destroy(h)


def rt_cart_stage_noalloc(args: rt_cart_stage_args):
    return check(_fns().rt_cart_stage_noalloc(C.byref(args)))


def rt_last_error() -> str:
    return _fns().rt_last_error().decode()


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


# -- conveniences --------------------------------------------------------------------------
class _Keep:
    """Holds the numpy arrays referenced by C structs until the call returns."""

    def __init__(self):
        self.refs = []

    def f64(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.refs.append(a)
        return a.ctypes.data_as(_dp)

    def i32(self, a):
        a = np.ascontiguousarray(a, dtype=np.int32)
        self.refs.append(a)
        return a.ctypes.data_as(_ip)


def make_structs(problem, quad, keep: _Keep):
    """C structs for a problem from sn_inputs (mesh, materials, boundary) and a
    quadrature (xi, eta, mu, w)."""
    m = problem.mesh
    mesh = rt_mesh()
    if hasattr(m, "nx"):
        mesh.kind = RT_MESH_CARTESIAN
        mesh.nx, mesh.ny, mesh.x0, mesh.y0, mesh.dx, mesh.dy = m.nx, m.ny, m.x0, m.y0, m.dx, m.dy
    else:
        mesh.kind = RT_MESH_TRIANGLES
        mesh.n_vert = m.vertices.shape[0]
        mesh.vxy = keep.f64(m.vertices.reshape(-1))
        mesh.n_tri = m.triangles.shape[0]
        mesh.tri = keep.i32(m.triangles.reshape(-1))
    mt = problem.materials
    mat = rt_materials()
    mat.n_mat = len(mt.sigma_a)
    mat.sigma_a, mat.sigma_s, mat.Q = keep.f64(mt.sigma_a), keep.f64(mt.sigma_s), keep.f64(mt.Q)
    mat.cell_mat, mat.cell_region = keep.i32(mt.cell_mat), keep.i32(mt.cell_region)
    mat.n_regions = max(mt.n_regions, int(np.max(mt.cell_region)) + 1)
    boxes = np.asarray(problem.extra.get("boxes", ()), dtype=np.float64).reshape(-1, 4)
    mat.n_boxes = boxes.shape[0]
    if mat.n_boxes:
        mat.boxes = keep.f64(boxes.reshape(-1))
    xi, eta, _, w = quad
    q = rt_quadrature()
    q.M = len(xi)
    q.xi, q.eta, q.w = keep.f64(xi), keep.f64(eta), keep.f64(w)
    bc = rt_boundary()
    for s in range(4):
        bc.side_kind[s] = int(problem.boundary.kind[s])
        bc.inflow[s] = float(problem.boundary.inflow[s])
    return mesh, mat, q, bc


def qoi_dict(q: rt_qoi_t, n_regions: int) -> dict:
    """QoIs as a dict of floats and arrays (box entries of length n_boxes)."""
    R, B = n_regions, q.n_boxes
    return {"t": q.t, "step": q.step, "n_steps": q.n_steps, "abs_now": np.array(q.abs_now[:R]),
            "abs_int": np.array(q.abs_int[:R]), "mass": q.mass, "outflow_now": q.outflow_now,
            "outflow_int": q.outflow_int, "source_int": q.source_int,
            "box_out_now": np.array(q.box_out_now[:B]), "box_out_int": np.array(q.box_out_int[:B])}


class TorchAllocator:
    """Device memory from PyTorch's caching allocator, handed to the library as
    C callbacks, plus the current stream of the current device."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        self.stream = torch.cuda.current_stream(self.device)

        def _alloc(n, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(n), self.device, self.stream))
            except Exception:
                return None

        def _free(p, ctx):
            if p:
                torch.cuda.caching_allocator_delete(int(p))

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)

    def fill(self, opts: rt_options):
        opts.alloc = self.alloc
        opts.free = self.free
        opts.alloc_ctx = None
        opts.stream = self.stream.cuda_stream


def make_options(order=1, integrator=RT_EULER, storage=RT_FP32, dt=0.0, t_end=1.0, tile_x=0, tile_y=0,
                 allocator: TorchAllocator | None = None, stream=None, variant=0, vec=0) -> rt_options:
    o = rt_options()
    o.order, o.integrator, o.storage = order, integrator, storage
    o.tile_x, o.tile_y, o.variant, o.vec = tile_x, tile_y, variant, vec
    o.dt, o.t_end = dt, t_end
    if allocator is not None:
        allocator.fill(o)
    if stream is not None:
        o.stream = stream
    return o


def rt_autotune(problem, quad, order=2, integrator=RT_HEUN, storage=RT_FP32, dt=0.0, t_end=None, steps=4,
                variant=0, vec=0):
    """Time the candidate Cartesian configurations of this problem on the
    current device (rt_autotune); returns ({tile_x, tile_y, variant, vec},
    ms per step of the fastest)."""
    keep = _Keep()
    mesh, mat, q, bc = make_structs(problem, quad, keep)
    alloc = TorchAllocator()
    opts = make_options(order, integrator, storage, dt, problem.t_end if t_end is None else t_end, 0, 0, alloc,
                        variant=variant, vec=vec)
    best = rt_options()
    ms = C.c_double()
    check(_fns().rt_autotune(C.byref(mesh), C.byref(mat), C.byref(q), C.byref(bc), C.byref(opts), int(steps),
                             C.byref(best), C.byref(ms)))
    return {"tile_x": best.tile_x, "tile_y": best.tile_y, "variant": best.variant, "vec": best.vec}, ms.value


class Solver:
    """One problem on the GPU: create -> step -> qoi, through the C ABI.
    tune=True takes the kernel configuration from the autotuner (cached per
    device and problem shape; see autotune.py) instead of tile_x/tile_y/variant/vec."""

    def __init__(self, problem, quad, order=1, integrator=RT_EULER, storage=RT_FP32, dt=0.0, t_end=None,
                 tile_x=0, tile_y=0, use_torch_allocator=True, variant=0, vec=0, tune=False):
        if tune and hasattr(problem.mesh, "nx"):
            from . import autotune
            cfg = autotune.tuned_config(problem, quad, order, integrator, storage, dt, t_end)
            tile_x, tile_y, variant, vec = cfg["tile_x"], cfg["tile_y"], cfg["variant"], cfg["vec"]
        keep = _Keep()
        mesh, mat, q, bc = make_structs(problem, quad, keep)
        self.allocator = TorchAllocator() if use_torch_allocator else None
        opts = make_options(order, integrator, storage, dt, problem.t_end if t_end is None else t_end,
                            tile_x, tile_y, self.allocator, variant=variant, vec=vec)
        self.h = rt_create(mesh, mat, q, bc, opts)
        self.info = rt_info(self.h)
        self.n_cells, self.M = int(self.info.n_cells), int(self.info.M)
        self.n_regions = mat.n_regions

    def step(self, n=None):
        rt_step(self.h, self.info.n_steps if n is None else n)
        return self

    def qoi(self) -> dict:
        q = rt_qoi(self.h)
        R = self.n_regions
        return qoi_dict(q, R)

    def psi(self) -> np.ndarray:
        return rt_get_psi(self.h, self.n_cells, self.M)

    def psi_cells(self, cells) -> np.ndarray:
        """psi of the given cells ([n, M], caller's orders) without copying the whole state."""
        return rt_get_psi_cells(self.h, cells, self.M)

    def phi(self) -> np.ndarray:
        return rt_get_phi(self.h, self.n_cells)

    def set_psi(self, psi):
        rt_set_psi(self.h, psi)

    def close(self):
        if getattr(self, "h", None):
            rt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_problem(problem, quad, keep, order=2, integrator=RT_HEUN, dt=0.0, tile_y=0, variant=0, vec=0):
    """rt_problem for a problem from sn_inputs and a quadrature (xi, eta, mu, w)."""
    pr = rt_problem()
    mesh, mat, q, bc = make_structs(problem, quad, keep)
    pr.mesh, pr.mat, pr.quad, pr.bc = mesh, mat, q, bc
    pr.order, pr.integrator, pr.dt, pr.t_end = order, integrator, float(dt), float(problem.t_end)
    pr.tile_y, pr.variant, pr.vec = tile_y, variant, vec
    return pr, (problem.mesh.n_cells, len(quad[0]), mat.n_regions)


class Batch:
    """Many problems advanced together (rt_batch_*): a fixed number of slots,
    problems added and removed between steps."""

    def __init__(self, problems=(), quads=(), order=2, integrator=RT_HEUN, storage=RT_FP32, dts=None,
                 tile_x=0, tile_y=0, use_torch_allocator=True, variant=0, vec=0, capacity=0, integrators=None,
                 orders=None, configs=None):
        """configs: optional per-problem dicts of tile_y / variant / vec (rt_problem's
        own kernel options; a missing or 0 value takes the batch option)."""
        keep = _Keep()
        k = len(problems)
        arr = (rt_problem * max(k, 1))()
        self.shapes = {}
        for i, (p, qd) in enumerate(zip(problems, quads)):
            o = order if orders is None else orders[i]
            ig = integrator if integrators is None else integrators[i]
            cf = {} if configs is None or configs[i] is None else configs[i]
            arr[i], self.shapes[i] = make_problem(p, qd, keep, o, ig, 0.0 if dts is None else dts[i],
                                                  cf.get("tile_y", 0), cf.get("variant", 0), cf.get("vec", 0))
        self.allocator = TorchAllocator() if use_torch_allocator else None
        opts = make_options(storage=storage, tile_x=tile_x, tile_y=tile_y, allocator=self.allocator, variant=variant,
                            vec=vec)
        self.h = C.c_void_p()
        check(_fns().rt_batch_create(k, arr, capacity, C.byref(opts), C.byref(self.h)))
        self.k = k

    def add(self, problem, quad, order=2, integrator=RT_HEUN, dt=0.0, tile_y=0, variant=0, vec=0) -> int:
        keep = _Keep()
        pr, shape = make_problem(problem, quad, keep, order, integrator, dt, tile_y, variant, vec)
        slot = C.c_int32()
        check(_fns().rt_batch_add(self.h, C.byref(pr), C.byref(slot)))
        self.shapes[slot.value] = shape
        return slot.value

    def remove(self, slot: int):
        check(_fns().rt_batch_remove(self.h, slot))
        self.shapes.pop(slot, None)

    def hold(self, slot: int, hold: bool = True):
        check(_fns().rt_batch_hold(self.h, slot, 1 if hold else 0))

    def step(self, n: int):
        check(_fns().rt_batch_step(self.h, int(n)))
        return self

    def progress(self, slot: int):
        done, total = C.c_int64(), C.c_int64()
        check(_fns().rt_batch_progress(self.h, slot, C.byref(done), C.byref(total)))
        return done.value, total.value

    def launches(self) -> int:
        n = C.c_int64()
        check(_fns().rt_batch_launches(self.h, C.byref(n)))
        return n.value

    def run(self, max_steps=0):
        check(_fns().rt_batch_run(self.h, int(max_steps)))
        return self

    def qoi(self, i) -> dict:
        q = rt_qoi_t()
        check(_fns().rt_batch_qoi(self.h, i, C.byref(q)))
        R = self.shapes[i][2]
        return qoi_dict(q, R)

    def psi(self, i) -> np.ndarray:
        n, M, _ = self.shapes[i]
        out = np.empty((n, M))
        check(_fns().rt_batch_get_psi(self.h, i, _ptr(out), out.size))
        return out

    def close(self):
        if getattr(self, "h", None):
            _fns().rt_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Failure detection on the host side: an allocator that returns NULL.

The library takes device memory only from the caller's allocator callback
(rt_options.alloc). A callback that fails on its k-th call, for every k that
rt_create or rt_batch_add reaches, must make the call return RT_ENOMEM, hand
back every block it had taken (nothing leaks) and leave a batch as it was. No
GPU fault is involved: the failure is injected on the host, in the callback.
"""
import ctypes as C

import numpy as np
import pytest

import sn_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2505_17284_gb300 import build, rt as rtmod
    build.build()
    rtmod.load_library()
    return rtmod


class FailingAllocator:
    """PyTorch's caching allocator behind the library's callbacks, returning
    NULL on call number fail_at (counting from the last reset; 0 = never) and
    tracking the blocks that are live."""

    def __init__(self, rt):
        import torch
        self.torch = torch
        self.device = torch.cuda.current_device()
        self.stream = torch.cuda.current_stream()
        self.calls, self.fail_at, self.live = 0, 0, set()

        def _alloc(n, ctx):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            p = int(torch.cuda.caching_allocator_alloc(int(n), self.device, self.stream))
            self.live.add(p)
            return p

        def _free(p, ctx):
            if p:
                self.live.discard(int(p))
                torch.cuda.caching_allocator_delete(int(p))

        self.alloc = rt.ALLOC_FN(_alloc)
        self.free = rt.FREE_FN(_free)

    def reset(self, fail_at):
        self.calls, self.fail_at = 0, fail_at

    def fill(self, opts):
        opts.alloc, opts.free, opts.alloc_ctx = self.alloc, self.free, None
        opts.stream = self.stream.cuda_stream


def _create(rt, fa, problem, quad, **kw):
    keep = rt._Keep()
    mesh, mat, q, bc = rt.make_structs(problem, quad, keep)
    opts = rt.make_options(t_end=problem.t_end, allocator=fa, **kw)
    h = C.c_void_p()
    code = rt._fns().rt_create(C.byref(mesh), C.byref(mat), C.byref(q), C.byref(bc), C.byref(opts), C.byref(h))
    return code, h


@pytest.mark.parametrize("kind", ["lattice", "triangles"])
def test_rt_create_enomem_at_every_allocation(rt, kind):
    if kind == "lattice":
        p, kw = si.lattice_problem(28, t_end=0.5), dict(order=2, integrator=rt.RT_HEUN, dt=0.0625)
    else:
        p, kw = si.enclosure_problem(10, t_end=0.3), dict(order=2, integrator=rt.RT_HEUN)
    quad = rt.rt_quad_product(2, 16)
    fa = FailingAllocator(rt)
    fa.reset(0)
    code, h = _create(rt, fa, p, quad, **kw)
    assert code == rt.RT_OK
    n_calls = fa.calls
    assert n_calls >= 5 and len(fa.live) == n_calls
    rt.rt_step(h, 2)
    ok_q = rt.rt_qoi(h)
    rt.rt_destroy(h)
    assert not fa.live
    for k in range(1, n_calls + 1):
        fa.reset(k)
        code, h = _create(rt, fa, p, quad, **kw)
        assert code == rt.RT_ENOMEM, (k, code)
        assert not h.value
        assert "allocator returned NULL" in rt.rt_last_error()
        assert not fa.live, f"blocks leaked after a failure at allocation {k}"
    # the context and the allocator still work
    fa.reset(0)
    code, h = _create(rt, fa, p, quad, **kw)
    assert code == rt.RT_OK
    rt.rt_step(h, 2)
    assert rt.rt_qoi(h).mass == ok_q.mass
    rt.rt_destroy(h)
    assert not fa.live


def test_rt_batch_add_enomem_leaves_the_batch_unchanged(rt):
    import torch
    p0 = si.lattice_problem(21, t_end=0.6)
    p1 = si.lattice_problem(28, t_end=0.6)
    q0, q1 = rt.rt_quad_product(2, 8), rt.rt_quad_product(2, 16)
    fa = FailingAllocator(rt)
    keep = rt._Keep()
    arr = (rt.rt_problem * 1)()
    arr[0], _ = rt.make_problem(p0, q0, keep, 2, rt.RT_HEUN, 0.5 * p0.mesh.dx)
    opts = rt.make_options(allocator=fa)
    b = C.c_void_p()
    fa.reset(0)
    rt.check(rt._fns().rt_batch_create(1, arr, 2, C.byref(opts), C.byref(b)))
    before = set(fa.live)
    pr1, _ = rt.make_problem(p1, q1, keep, 2, rt.RT_HEUN, 0.5 * p1.mesh.dx)
    slot = C.c_int32(-1)
    fa.reset(0)
    rt.check(rt._fns().rt_batch_add(b, C.byref(pr1), C.byref(slot)))
    n_calls = fa.calls
    rt.check(rt._fns().rt_batch_remove(b, slot.value))
    assert fa.live == before
    for k in range(1, n_calls + 1):
        fa.reset(k)
        code = rt._fns().rt_batch_add(b, C.byref(pr1), C.byref(slot))
        assert code == rt.RT_ENOMEM, (k, code)
        assert fa.live == before, f"blocks leaked after a failure at allocation {k}"
    # the member already in the batch runs as if nothing happened
    fa.reset(0)
    rt.check(rt._fns().rt_batch_run(b, 0))
    out = np.empty((p0.mesh.n_cells, 16))
    rt.check(rt._fns().rt_batch_get_psi(b, 0, rt._ptr(out), out.size))
    s = rt.Solver(p0, q0, order=2, integrator=rt.RT_HEUN, dt=0.5 * p0.mesh.dx)
    s.step()
    assert np.array_equal(out, s.psi())
    s.close()
    rt._fns().rt_batch_destroy(b)
    torch.cuda.synchronize()
    assert not fa.live

"""C-ABI checks that need no GPU: the library loads, exports every function
that include/rt.h declares, the host-only quadrature helper agrees with the
oracle's rule, and argument validation rejects bad input with RT_EINVAL
before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import sn_inputs as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rt():
    from paper_2505_17284_gb300 import build, rt as rtmod
    build.build()
    rtmod.load_library()
    return rtmod


def declared_functions():
    text = open(os.path.join(ROOT, "include", "rt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:rt_status|void|const char\*)\s+(rt_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(rt):
    names = declared_functions()
    assert len(names) >= 20
    lib = C.CDLL(rt.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(rt.SIGNATURES), set(names) ^ set(rt.SIGNATURES)


@pytest.mark.parametrize("n_p,n_phi", [(1, 4), (4, 16), (8, 16), (8, 32), (16, 32), (24, 8)])
def test_quad_product_matches_oracle(rt, n_p, n_phi):
    xi, eta, mu, w = rt.rt_quad_product(n_p, n_phi)
    oxi, oeta, omu, ow = oracle.product_quadrature(n_p, n_phi)
    for a, b in ((xi, oxi), (eta, oeta), (mu, omu), (w, ow)):
        assert np.max(np.abs(a - b)) < 5e-15
    assert abs(w.sum() - 2 * np.pi) < 1e-13


def test_quad_product_rejects_bad_sizes(rt):
    with pytest.raises(rt.RTError) as e:
        rt.rt_quad_product(0, 8)
    assert e.value.code == rt.RT_EINVAL
    with pytest.raises(rt.RTError):
        rt.rt_quad_product(65, 8)


@pytest.mark.parametrize("N", [1, 2, 3, 8, 22])
def test_quad_tessellation_matches_oracle(rt, N):
    xi, eta, mu, w = rt.rt_quad_tessellation(N)
    oxi, oeta, omu, ow = oracle.tessellation_quadrature(N)
    for a, b in ((xi, oxi), (eta, oeta), (mu, omu), (w, ow)):
        assert np.max(np.abs(a - b)) < 5e-14
    with pytest.raises(rt.RTError) as e:
        rt.rt_quad_tessellation(0)
    assert e.value.code == rt.RT_EINVAL


def _create(rt, problem, quad, **kw):
    keep = rt._Keep()
    mesh, mat, q, bc = rt.make_structs(problem, quad, keep)
    for k, v in kw.get("mutate", {}).items():
        obj, field = k.split(".")
        target = {"mesh": mesh, "mat": mat, "q": q, "bc": bc}[obj]
        if field == "side_kind":
            target.side_kind[0] = v
        else:
            setattr(target, field, v)
    opts = rt.make_options(order=kw.get("order", 1), integrator=kw.get("integrator", 0), t_end=kw.get("t_end", 1.0),
                           storage=kw.get("storage", 0))
    return rt.rt_create(mesh, mat, q, bc, opts)


@pytest.mark.parametrize("mutate,kw", [
    ({"mesh.nx": 0}, {}),
    ({"mesh.dx": -1.0}, {}),
    ({"mesh.kind": 7}, {}),
    ({"mat.n_mat": 0}, {}),
    ({"mat.n_mat": 65}, {}),
    ({"mat.n_regions": 0}, {}),
    ({"q.M": 0}, {}),
    ({"bc.side_kind": 2}, {}),        # periodic: not on the GPU path
    ({"bc.side_kind": 9}, {}),
    ({}, {"order": 3}),
    ({}, {"integrator": 5}),
    ({}, {"storage": 4}),
    ({}, {"t_end": -1.0}),
])
def test_create_rejects_invalid_arguments(rt, mutate, kw):
    p = si.lattice_problem(14)
    quad = rt.rt_quad_product(2, 4)
    with pytest.raises(rt.RTError) as e:
        _create(rt, p, quad, mutate=mutate, **kw)
    assert e.value.code == rt.RT_EINVAL
    assert rt.rt_last_error() != ""


def test_create_rejects_bad_cells_and_meshes(rt):
    quad = rt.rt_quad_product(2, 4)
    p = si.lattice_problem(14)
    p.materials.cell_mat = p.materials.cell_mat.copy()
    p.materials.cell_mat[5] = 3          # only 3 materials
    with pytest.raises(rt.RTError) as e:
        _create(rt, p, quad)
    assert e.value.code == rt.RT_EINVAL and "material id" in rt.rt_last_error()
    # clockwise triangle
    t = si.enclosure_problem(6, jitter=0.0)
    t.mesh.triangles = t.mesh.triangles.copy()
    t.mesh.triangles[0] = t.mesh.triangles[0][::-1]
    with pytest.raises(rt.RTError) as e:
        _create(rt, t, quad)
    assert e.value.code == rt.RT_EINVAL
    # second order on triangles: still validated (order 3 rejected)
    with pytest.raises(rt.RTError) as e:
        _create(rt, si.enclosure_problem(6), quad, order=3)
    assert e.value.code == rt.RT_EINVAL


def test_null_handles_are_rejected(rt):
    lib = rt.load_library()
    q = rt.rt_qoi_t()
    assert lib.rt_step(None, 1) == rt.RT_EINVAL
    assert lib.rt_qoi(None, C.byref(q)) == rt.RT_EINVAL
    assert lib.rt_batch_run(None, 1) == rt.RT_EINVAL
    lib.rt_destroy(None)
    lib.rt_batch_destroy(None)


@pytest.mark.parametrize("boxes,msg", [
    (((2.0, 5.0, 2.0, 5.05),), "grid line"),         # edge between grid lines
    (((0.0, 5.0, 2.0, 5.0),), "grid line"),          # on the domain boundary
    (((2.0, 7.0, 2.0, 5.0),), "grid line"),
    (((5.0, 2.0, 2.0, 5.0),), "x_lo < x_hi"),
    (((2.0, 5.0, 2.0, 5.0),) * 5, "n_boxes"),
    (((2.0, 5.0, float("nan"), 5.0),), "finite"),
])
def test_create_rejects_bad_qoi_boxes(rt, boxes, msg):
    p = si.lattice_problem(14)
    p.extra = {"boxes": boxes}
    with pytest.raises(rt.RTError) as e:
        _create(rt, p, rt.rt_quad_product(2, 4))
    assert e.value.code == rt.RT_EINVAL and msg in rt.rt_last_error()


def test_qoi_boxes_need_a_cartesian_mesh(rt):
    t = si.enclosure_problem(6)
    t.extra = {"boxes": ((0.2, 0.6, 0.2, 0.6),)}
    with pytest.raises(rt.RTError) as e:
        _create(rt, t, rt.rt_quad_product(2, 4))
    assert e.value.code == rt.RT_EINVAL and "Cartesian" in rt.rt_last_error()


def test_qoi_struct_layout(rt):
    # the header's rt_qoi_t: 392 bytes, box entries last
    assert C.sizeof(rt.rt_qoi_t) == 392
    assert rt.rt_qoi_t.box_out_int.offset == 392 - 8 * rt.RT_MAX_BOXES


def test_get_psi_cells_rejects_bad_arguments(rt):
    lib = rt.load_library()
    assert lib.rt_get_psi_cells(None, None, 0, None) == rt.RT_EINVAL

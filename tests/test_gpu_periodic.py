"""Periodic sides on Cartesian grids, on the GPU, against the FP64 oracle.

A periodic pair of sides (x-/x+ or y-/y+) has no boundary faces: the cell
across the side is the cell at the other end of the row or column, so the flux
form of Sec. 4.2 (Eq. sn_2d_eqn_fv) telescopes over the whole periodic axis.
With sigma_a = 0 and periodic sides only, the particle count sum_i A_i phi_i
is then conserved by every step of the scheme (the sharpest conservation check
of the flux form); the device reproduces that to FP32 rounding over 1000
steps. Element-wise parity against the oracle's periodic path covers both
orders, both integrators, both kernel families (chunk-uniform and per-lane
directions), 16- and 32-cell strips, ragged tiles, and one periodic axis
combined with inflow or vacuum sides on the other.
"""
import numpy as np
import pytest

import oracle
import sn_inputs as si

pytestmark = pytest.mark.gpu

PSI_TOL = 1e-5
QOI_TOL = 1e-4


@pytest.fixture(scope="module")
def rt():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2505_17284_gb300 import build, rt as rtmod
    build.build()
    rtmod.load_library()
    return rtmod


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def periodic_problem(n, kind, inflow=(0.0, 0.0, 0.0, 0.0), sigma_a=None):
    p = si.lattice_problem(n)
    p.extra = {}                       # no QoI squares
    p.boundary = si.Boundary(kind=kind, inflow=inflow)
    if sigma_a is not None:
        p.materials.sigma_a = np.full_like(p.materials.sigma_a, sigma_a)
    return p


P = si.PERIODIC


@pytest.mark.parametrize("kind,inflow", [((P, P, P, P), (0, 0, 0, 0)), ((P, P, 1, 1), (0, 0, 1.0, 0.5)),
                                         ((1, 0, P, P), (2.0, 0, 0, 0))])
@pytest.mark.parametrize("order,integrator", [(1, "euler"), (2, "heun"), (2, "euler")])
@pytest.mark.parametrize("variant,tile_x", [(0, 0), (1, 0), (2, 32)])
def test_periodic_parity_with_the_oracle(rt, kind, inflow, order, integrator, variant, tile_x):
    """84^2 grid (ragged tiles in x and y), 8x16 = 128 ordinates (8x32 with
    32-cell strips), a random state, 6 steps: psi element-wise and every QoI
    against the oracle."""
    p = periodic_problem(84, kind, inflow)
    n_p, n_phi, M = (8, 16, 128) if tile_x != 32 else (8, 32, 256)   # 32-cell strips: 64-ordinate quadrant chunks
    quad = rt.rt_quad_product(n_p, n_phi)
    integ = rt.RT_HEUN if integrator == "heun" else rt.RT_EULER
    s = rt.Solver(p, quad, order=order, integrator=integ, dt=0.5 * p.mesh.dx, tile_y=24, variant=variant,
                  tile_x=tile_x)
    psi0 = si.random_psi(p.mesh.n_cells, M, seed=7) + si.smooth_psi(p.mesh, M, seed=8)
    s.set_psi(psi0)
    start = s.psi()                    # the state the device starts from (FP32)
    s.step(6)
    got, q = s.psi(), s.qoi()
    dt = s.info.dt
    s.close()
    op = oracle.CartesianOracle(p, oracle.product_quadrature(n_p, n_phi), order=order)
    ref, acc, S = oracle.run(op, start, dt, 6, integrator)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) <= 4e-6 * scale
    assert rel_l2(got, ref) <= PSI_TOL
    m = S["mass"]
    assert abs(q["mass"] - m) <= QOI_TOL * m
    assert abs(q["outflow_now"] - S["outflow"]) <= QOI_TOL * max(abs(S["outflow"]), 1e-3 * m)
    assert abs(q["outflow_int"] - acc.outflow_int) <= QOI_TOL * max(abs(acc.outflow_int), 1e-3 * m)
    for r in range(len(S["abs"])):
        assert abs(q["abs_int"][r] - acc.abs_int[r]) <= QOI_TOL * max(abs(acc.abs_int[r]), 1e-3 * m)
    if all(k == P for k in kind):
        assert q["outflow_now"] == 0.0 and q["outflow_int"] == 0.0


@pytest.mark.parametrize("order,integrator", [(1, "euler"), (2, "heun")])
def test_periodic_box_conserves_particles_over_1000_steps(rt, order, integrator):
    """sigma_a = 0 and periodic on all sides: the particle count of a random
    non-negative state stays constant (FP32 rounding only) for 1000 steps,
    nothing leaves through the boundary and nothing is absorbed."""
    p = periodic_problem(56, (P, P, P, P), sigma_a=0.0)
    p.materials.Q = np.zeros_like(p.materials.Q)
    p.t_end = 1000 * 0.5 * p.mesh.dx
    quad = rt.rt_quad_product(4, 16)
    integ = rt.RT_HEUN if integrator == "heun" else rt.RT_EULER
    s = rt.Solver(p, quad, order=order, integrator=integ, dt=0.5 * p.mesh.dx)
    assert s.info.n_steps == 1000
    s.set_psi(si.random_psi(p.mesh.n_cells, 64, seed=11))
    m0 = s.qoi()["mass"]
    worst = 0.0
    for _ in range(10):
        s.step(100)
        q = s.qoi()
        worst = max(worst, abs(q["mass"] / m0 - 1.0))
        assert q["outflow_now"] == 0.0 and q["outflow_int"] == 0.0
        assert all(v == 0.0 for v in q["abs_int"])
    assert q["step"] == 1000
    assert worst <= 2e-5, worst
    s.close()


def test_periodic_on_triangles_is_rejected(rt):
    p = si.enclosure_problem(8)
    p.boundary = si.Boundary(kind=(P, P, 0, 0))
    with pytest.raises(rt.RTError) as e:
        rt.Solver(p, rt.rt_quad_product(2, 8))
    assert e.value.code == rt.RT_EINVAL
    assert "Cartesian" in rt.rt_last_error()


def test_unpaired_periodic_side_is_rejected(rt):
    p = periodic_problem(14, (P, 0, 0, 0))
    with pytest.raises(rt.RTError) as e:
        rt.Solver(p, rt.rt_quad_product(2, 8))
    assert e.value.code == rt.RT_EINVAL
    assert "pairs" in rt.rt_last_error()

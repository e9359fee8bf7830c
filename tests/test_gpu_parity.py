"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (FP32 storage and arithmetic against FP64): relative L2 error of
psi <= 1e-5 and relative error of every QoI <= 1e-4. Sizes are chosen so the
oracle finishes in seconds while the grids still span several tiles, ragged
tails in x and y, several ordinate chunks and both boundary kinds.
"""
import math

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


def rel(a, b, floor=1e-30):
    return abs(a - b) / max(abs(b), floor)


def oracle_op(problem, quad, order):
    if isinstance(problem.mesh, si.CartesianMesh):
        return oracle.CartesianOracle(problem, quad, order=order)
    return oracle.TriangleOracle(problem, quad, order=order)


def check_qoi(q, acc, S, n_regions, scale):
    for r in range(n_regions):
        assert abs(q["abs_int"][r] - acc.abs_int[r]) <= QOI_TOL * max(abs(acc.abs_int[r]), 1e-3 * scale), ("abs_int", r)
        assert abs(q["abs_now"][r] - S["abs"][r]) <= QOI_TOL * max(abs(S["abs"][r]), 1e-3 * scale), ("abs_now", r)
    assert rel(q["mass"], S["mass"]) <= QOI_TOL
    assert abs(q["outflow_int"] - acc.outflow_int) <= QOI_TOL * max(abs(acc.outflow_int), 1e-3 * scale)
    assert abs(q["outflow_now"] - S["outflow"]) <= QOI_TOL * max(abs(S["outflow"]), 1e-3 * scale)
    # QoI boxes (Sec. 3.1 QoI-1/2), when the problem has them
    nb = len(S.get("box_out", ()))
    assert len(q["box_out_now"]) == nb
    for b in range(nb):
        assert abs(q["box_out_now"][b] - S["box_out"][b]) <= QOI_TOL * max(abs(S["box_out"][b]), 1e-3 * scale), b
        assert abs(q["box_out_int"][b] - acc.box_out_int[b]) <= \
            QOI_TOL * max(abs(acc.box_out_int[b]), 1e-3 * scale), b


def run_pair(rt, problem, n_p, n_phi, order, integrator, steps, psi0=None, storage=0, dt=0.0, tile_y=0, tile_x=0):
    quad_lib = rt.rt_quad_product(n_p, n_phi)
    s = rt.Solver(problem, quad_lib, order=order, integrator=integrator, storage=storage, dt=dt,
                  tile_x=tile_x, tile_y=tile_y)
    M = n_p * n_phi
    if psi0 is not None:
        s.set_psi(psi0)
    s.step(steps)
    q = s.qoi()
    psi = s.psi()
    phi = s.phi()
    info = s.info
    s.close()
    op = oracle_op(problem, oracle.product_quadrature(n_p, n_phi), order)
    start = np.zeros((problem.mesh.n_cells, M)) if psi0 is None else psi0
    ref, acc, S = oracle.run(op, start, info.dt, steps, "euler" if integrator == rt.RT_EULER else "heun")
    return psi, phi, q, ref, acc, S, op, info


# ------------------------------------------------------------------ lattice, first order
def test_lattice_config1_full(rt):
    """70^2 lattice, 4x16 ordinates, first-order upwind + Euler, dt = dx/2, 64 steps."""
    p = si.lattice_problem(70)
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, p, 4, 16, 1, rt.RT_EULER, 64, dt=0.05)
    assert info.n_steps == 64 and q["step"] == 64 and abs(q["t"] - 3.2) < 1e-12
    assert rel_l2(psi, ref) <= PSI_TOL
    assert rel_l2(phi, op.phi(ref)) <= PSI_TOL
    check_qoi(q, acc, S, 3, scale=S["mass"])
    # discrete mass balance holds on the device to FP32 rounding
    bal = q["mass"] + sum(q["abs_int"]) + q["outflow_int"]
    assert abs(bal / q["source_int"] - 1) < 1e-5


@pytest.mark.parametrize("integrator", ["euler", "heun"])
@pytest.mark.parametrize("order", [1, 2])
def test_lattice_ragged_tiles(rt, order, integrator):
    """84^2 = 2*32 + 20 cells in x, segments of 24 rows (ragged in y),
    4x32 = 128 ordinates (4 chunks): every tile/segment/chunk boundary."""
    p = si.lattice_problem(84)
    integ = rt.RT_EULER if integrator == "euler" else rt.RT_HEUN
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, p, 4, 32, order, integ, 12, dt=0.5 * p.mesh.dx,
                                                  tile_y=24)
    assert info.tile_y == 24
    assert rel_l2(psi, ref) <= PSI_TOL
    check_qoi(q, acc, S, 3, scale=S["mass"])


@pytest.mark.parametrize("order,integrator", [(1, "euler"), (2, "heun"), (2, "euler"), (1, "heun")])
def test_random_state_one_step_elementwise(rt, order, integrator):
    """A random non-negative state on a 100 x 100 lattice (ragged: 100 = 3*32 + 4),
    one step: element-wise agreement with the oracle."""
    p = si.lattice_problem(100)
    M = 64
    psi0 = si.random_psi(p.mesh.n_cells, M, seed=21)
    integ = rt.RT_EULER if integrator == "euler" else rt.RT_HEUN
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, p, 4, 16, order, integ, 1, psi0=psi0, dt=0.5 * p.mesh.dx)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(psi - ref)) <= 2e-6 * scale
    assert rel_l2(psi, ref) <= PSI_TOL
    assert rel_l2(phi, op.phi(ref)) <= PSI_TOL
    check_qoi(q, acc, S, 3, scale=S["mass"])


@pytest.mark.parametrize("n_p,n_phi,variant,tile_x", [(4, 16, 0, 0), (8, 16, 0, 0), (2, 16, 0, 0), (8, 32, 1, 0),
                                                      (8, 32, 2, 16), (8, 32, 0, 32), (16, 32, 1, 0), (16, 32, 2, 16),
                                                      (16, 32, 2, 32), (4, 64, 2, 16), (4, 64, 0, 32)])
@pytest.mark.parametrize("order", [1, 2])
def test_kernel_variants(rt, n_p, n_phi, variant, tile_x, order):
    """Ordinates per lane (1, 2, 4), both direction families (per-lane and
    chunk-uniform) and both strip widths (16 and 32 cells) on a 91^2 grid (ragged
    tiles) from a smooth state, Heun."""
    p = si.lattice_problem(91)
    psi0 = si.smooth_psi(p.mesh, n_p * n_phi, seed=3)
    quad_lib = rt.rt_quad_product(n_p, n_phi)
    s = rt.Solver(p, quad_lib, order=order, integrator=rt.RT_HEUN, dt=0.5 * p.mesh.dx, variant=variant,
                  tile_x=tile_x)
    if tile_x:
        assert s.info.tile_x == tile_x
    s.set_psi(psi0)
    s.step(5)
    psi, q, dt = s.psi(), s.qoi(), s.info.dt
    s.close()
    op = oracle.CartesianOracle(p, oracle.product_quadrature(n_p, n_phi), order=order)
    ref, acc, S = oracle.run(op, psi0, dt, 5, "heun")
    assert rel_l2(psi, ref) <= PSI_TOL
    check_qoi(q, acc, S, 3, scale=S["mass"])


@pytest.mark.parametrize("n,variant,tile_x", [(63, 1, 16), (320, 2, 32)])
def test_library_kernel_choice_by_grid_size(rt, n, variant, tile_x):
    """256 ordinates (quadrants of 64): the library runs small grids (at most
    1e5 cells) on the per-lane kernel with 16-cell strips and larger ones on the
    32-cell chunk-uniform kernel; an explicit tile_x 32 asks for the latter at
    any size."""
    p = si.lattice_problem(n)
    quad = rt.rt_quad_product(8, 32)
    s = rt.Solver(p, quad, order=2, integrator=rt.RT_HEUN, dt=0.5 * p.mesh.dx)
    assert (s.info.variant, s.info.tile_x) == (variant, tile_x)
    s.close()
    s = rt.Solver(p, quad, order=2, integrator=rt.RT_HEUN, dt=0.5 * p.mesh.dx, tile_x=32)
    assert (s.info.variant, s.info.tile_x) == (2, 32)
    s.close()


def test_uniform_variant_rejected_for_mixed_chunks(rt):
    p = si.lattice_problem(14)
    xi = np.array([0.6, -0.6] * 32)
    eta = np.array([0.5] * 64)
    quad = (xi, eta, np.sqrt(1 - xi ** 2 - eta ** 2), np.full(64, 2 * math.pi / 64))
    with pytest.raises(rt.RTError) as e:
        rt.Solver(p, quad, order=2, integrator=rt.RT_HEUN, dt=0.25, variant=2)
    assert e.value.code == rt.RT_EINVAL


def test_wide_strips_need_uniform_pairs(rt):
    p = si.lattice_problem(14)
    with pytest.raises(rt.RTError) as e:
        rt.Solver(p, rt.rt_quad_product(4, 16), order=2, integrator=rt.RT_HEUN, dt=0.25, tile_x=32)
    assert e.value.code == rt.RT_EINVAL
    with pytest.raises(rt.RTError):
        rt.Solver(p, rt.rt_quad_product(16, 32), order=2, integrator=rt.RT_HEUN, dt=0.25, tile_x=24)


def test_mixed_sign_quadrature_groups(rt):
    """Ordinates whose consecutive groups mix signs of xi (one ordinate per lane
    then): alternate +xi/-xi ordinates."""
    p = si.lattice_problem(35)
    xi = np.array([0.6, -0.6, 0.3, -0.3] * 8)
    eta = np.array([0.5, 0.5, -0.7, -0.7] * 8)
    w = np.full(32, 2 * math.pi / 32)
    quad = (xi, eta, np.sqrt(1 - xi ** 2 - eta ** 2), w)
    s = rt.Solver(p, quad, order=2, integrator=rt.RT_HEUN, dt=0.5 * p.mesh.dx)
    psi0 = si.smooth_psi(p.mesh, 32, seed=8)
    s.set_psi(psi0)
    s.step(6)
    psi = s.psi()
    s.close()
    op = oracle.CartesianOracle(p, quad, order=2)
    ref, _, _ = oracle.run(op, psi0, 0.5 * p.mesh.dx, 6, "heun")
    assert rel_l2(psi, ref) <= PSI_TOL


def test_cartesian_inflow_boundary(rt):
    """Enclosure geometry on a 65^2 Cartesian grid: inflow psi^- = 1 on x = 0, MUSCL + Heun."""
    p = si.enclosure_cartesian_problem(65)
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, p, 2, 16, 2, rt.RT_HEUN, 30, dt=0.5 * p.mesh.dx)
    assert rel_l2(psi, ref) <= PSI_TOL
    check_qoi(q, acc, S, 4, scale=S["mass"])
    assert q["outflow_int"] < 0


def test_general_inflow_all_sides_and_odd_quadrature(rt):
    """Inflow of different strengths on every side and an ordinate count that is
    not a multiple of 32 (padding ordinates carry zero weight)."""
    p = si.lattice_problem(40)
    p.boundary = si.Boundary(kind=(1, 1, 1, 1), inflow=(1.0, 0.5, 0.25, 2.0))
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, p, 3, 10, 2, rt.RT_HEUN, 15, dt=0.5 * p.mesh.dx)
    assert info.M == 30 and info.M_pad == 32
    assert rel_l2(psi, ref) <= PSI_TOL
    check_qoi(q, acc, S, 3, scale=S["mass"])


def test_muscl_heun_lattice_mass_balance_and_symmetry(rt):
    p = si.lattice_problem(56)
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, p, 4, 16, 2, rt.RT_HEUN, 40, dt=0.5 * p.mesh.dx)
    assert rel_l2(psi, ref) <= PSI_TOL
    bal = q["mass"] + sum(q["abs_int"]) + q["outflow_int"]
    assert abs(bal / q["source_int"] - 1) < 1e-5
    ph = phi.reshape(56, 56)
    assert np.max(np.abs(ph - ph[:, ::-1])) <= 1e-5 * ph.max()


# ------------------------------------------------------------------ QoI boxes (Sec. 3.1 QoI-1/2)
BOXES = ((2.0, 5.0, 2.0, 5.0), (1.0, 6.0, 1.0, 6.0),      # the squares S_1.5, S_2.5
         (0.125, 0.25, 3.0, 6.875),                      # one cell wide, next to the x- boundary
         (4.5, 6.875, 0.125, 1.0))                       # next to two boundaries


@pytest.mark.parametrize("order,integrator,n_p,n_phi", [(1, "euler", 4, 16), (2, "heun", 4, 32), (2, "euler", 2, 16),
                                                        (1, "heun", 8, 16)])
def test_box_outflow_matches_the_oracle(rt, order, integrator, n_p, n_phi):
    """Outflow through four boxes (the paper's two squares, a one-cell-wide
    strip and a box one cell from two domain sides) from a random state: the
    per-box values at the final state and their time integrals, against the
    oracle; 56^2 cells (dx = 1/8), ragged tiles."""
    p = si.lattice_problem(56)
    p.extra = {"boxes": BOXES}
    integ = rt.RT_EULER if integrator == "euler" else rt.RT_HEUN
    psi0 = si.random_psi(p.mesh.n_cells, n_p * n_phi, seed=21)
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, p, n_p, n_phi, order, integ, 9, psi0=psi0,
                                                  dt=0.5 * p.mesh.dx, tile_y=24)
    assert rel_l2(psi, ref) <= PSI_TOL
    assert len(q["box_out_now"]) == 4 and np.all(q["box_out_now"] > 0) and np.all(q["box_out_int"] > 0)
    check_qoi(q, acc, S, 3, scale=S["mass"])


@pytest.mark.parametrize("quad", ["tess8", "prod12x40"])
def test_box_outflow_of_the_lattice_squares(rt, quad):
    """The lattice from psi = 0 with the squares S_1.5 and S_2.5 (QoI-1/2),
    MUSCL Heun; the tessellation rule of order 8, and a product rule whose
    ordinates are stored regrouped by quadrant (the box kernel reads the
    internal order)."""
    p = si.lattice_problem(42, t_end=2.0)
    if quad == "tess8":
        quad_lib, quad_or = rt.rt_quad_tessellation(8), oracle.tessellation_quadrature(8)
    else:
        quad_lib, quad_or = rt.rt_quad_product(12, 40), oracle.product_quadrature(12, 40)
    s = rt.Solver(p, quad_lib, order=2, integrator=rt.RT_HEUN, dt=0.5 * p.mesh.dx)
    s.step()
    q, info = s.qoi(), s.info
    s.close()
    assert info.regrouped == (quad != "tess8")
    op = oracle.CartesianOracle(p, quad_or, order=2)
    n = int(info.n_steps)
    _, acc, S = oracle.run(op, np.zeros((p.mesh.n_cells, len(quad_or[0]))), info.dt, n, "heun")
    check_qoi(q, acc, S, 3, scale=S["mass"])
    assert q["box_out_int"][0] > q["box_out_int"][1] > 0


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("mixed", [False, True])
def test_box_outflow_batched_equals_alone_bitwise(rt, storage, mixed):
    """Problems with and without boxes and with different N_t in one batch (so
    the box launches of finished problems are masked): every box value equals
    the problem solved alone, bit for bit. The mixed case puts Euler and Heun
    problems of both orders in one batch, so the box launch after a step covers
    several kernel-variant groups, split where the last stage differs."""
    probs = [si.lattice_problem(28, t_end=0.6), si.lattice_problem(30, t_end=1.0), si.lattice_problem(35, t_end=1.4)]
    probs[1].extra = {}
    quads = [rt.rt_quad_product(2, 16), rt.rt_quad_product(4, 16), rt.rt_quad_product(2, 32)]
    orders, integrators = [2, 2, 2], [rt.RT_HEUN] * 3
    if mixed:
        probs.append(si.lattice_problem(42, t_end=0.8))
        quads.append(rt.rt_quad_product(4, 16))
        orders, integrators = [1, 2, 2, 2], [rt.RT_EULER, rt.RT_HEUN, rt.RT_EULER, rt.RT_HEUN]
    dts = [0.5 * pr.mesh.dx for pr in probs]
    b = rt.Batch(probs, quads, dts=dts, storage=storage, orders=orders, integrators=integrators)
    b.run()
    for i, (pr, qd) in enumerate(zip(probs, quads)):
        s = rt.Solver(pr, qd, order=orders[i], integrator=integrators[i], dt=dts[i], storage=storage)
        s.step()
        a, c = b.qoi(i), s.qoi()
        s.close()
        assert len(a["box_out_now"]) == (0 if i == 1 else 2)
        for k in ("box_out_now", "box_out_int", "mass", "outflow_int"):
            assert np.array_equal(np.asarray(a[k]), np.asarray(c[k])), (i, k)
    b.close()


# ------------------------------------------------------------------ DP-2: per-block cross-sections
@pytest.mark.parametrize("integrator", ["euler", "heun"])
def test_lattice_dp2_per_block_parameters(rt, integrator):
    """DP-2 (Sec. 3.1.3): 49 block materials with drawn sigma_a, sigma_s, on an
    84^2 grid (ragged tiles) from a random state, so every block's
    cross-sections enter the first step; MUSCL, 4x32 ordinates."""
    d = si.dp2_instances(1, seed=11)[0]
    p = si.lattice_dp2_problem(84, d.sigma_a, d.sigma_s)
    integ = rt.RT_EULER if integrator == "euler" else rt.RT_HEUN
    psi0 = si.random_psi(p.mesh.n_cells, 128, seed=5)
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, p, 4, 32, 2, integ, 10, psi0=psi0, dt=0.5 * p.mesh.dx,
                                                  tile_y=24)
    assert rel_l2(psi, ref) <= PSI_TOL
    check_qoi(q, acc, S, 3, scale=S["mass"])


def test_lattice_dp2_nominal_equals_three_materials_bitwise(rt):
    """The nominal DP-2 point (49 materials carrying the three-material values)
    gives the checkerboard's result to the bit: material lookup is exact."""
    sa, ss = si.lattice_dp2_nominal()
    outs = []
    for p in (si.lattice_dp2_problem(70, sa, ss, t_end=1.0), si.lattice_problem(70, t_end=1.0)):
        s = rt.Solver(p, rt.rt_quad_product(4, 16), order=2, integrator=rt.RT_HEUN, dt=0.5 * p.mesh.dx)
        s.step()
        outs.append((s.psi(), s.qoi()))
        s.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    for k in ("mass", "abs_int", "outflow_int"):
        assert np.array_equal(np.asarray(outs[0][1][k]), np.asarray(outs[1][1][k])), k


def test_dp2_materials_on_triangles(rt):
    """Per-block materials (49 ids) through the triangle kernel's packed
    material/region word, against the oracle."""
    d = si.dp2_instances(1, seed=12)[0]
    t = si.lattice_triangle_problem(21, jitter=0.2, seed=3, t_end=0.5)
    xc, yc = t.mesh.centroids()
    bi, bj = np.floor(xc).astype(int), np.floor(yc).astype(int)
    t.materials = si.Materials(sigma_a=d.sigma_a.T.ravel().copy(), sigma_s=d.sigma_s.T.ravel().copy(),
                               Q=np.where(np.arange(49) == 24, 1.0, 0.0), cell_mat=(7 * bj + bi).astype(np.int32),
                               cell_region=si.lattice_block_material(bi, bj), region_names=si.LATTICE_REGIONS)
    psi0 = si.random_psi(t.mesh.n_cells, 64, seed=6)
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, t, 4, 16, 1, rt.RT_HEUN, 6, psi0=psi0)
    assert rel_l2(psi, ref) <= PSI_TOL
    check_qoi(q, acc, S, 3, scale=S["mass"])


# ------------------------------------------------------------------ triangles
# second order on triangles (Sec. 4.2): Green-Gauss gradient + Venkatakrishnan limiter
@pytest.mark.parametrize("integrator", ["euler", "heun"])
@pytest.mark.parametrize("n_p,n_phi", [(2, 16), (4, 16), (8, 16)])
def test_triangles_second_order_random_state(rt, integrator, n_p, n_phi):
    """Jittered enclosure mesh (2 * 26^2 triangles) from a random state, so the
    gradient, the limiter (extrema everywhere) and the reconstructed traces act
    on every cell and ordinate; 32, 64 and 128 ordinates (1 and 2 per lane)."""
    p = si.enclosure_problem(26, jitter=0.2, seed=1)
    integ = rt.RT_EULER if integrator == "euler" else rt.RT_HEUN
    psi0 = si.random_psi(p.mesh.n_cells, n_p * n_phi, seed=8)
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, p, n_p, n_phi, 2, integ, 6, psi0=psi0)
    assert rel_l2(psi, ref) <= PSI_TOL
    check_qoi(q, acc, S, 4, scale=S["mass"] + sum(acc.abs_int))


def test_triangles_second_order_enclosure_and_lattice(rt):
    """From psi = 0: the enclosure with its inflow (Heun, 40 steps) and the
    lattice on a jittered triangle mesh, against the oracle; the particle
    balance closes."""
    p = si.enclosure_problem(30, jitter=0.2, seed=0)
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, p, 4, 16, 2, rt.RT_HEUN, 40)
    assert rel_l2(psi, ref) <= PSI_TOL
    check_qoi(q, acc, S, 4, scale=S["mass"] + sum(acc.abs_int))
    bal = q["mass"] + sum(q["abs_int"]) + q["outflow_int"]
    assert abs(bal) <= 1e-5 * (q["mass"] + sum(q["abs_int"]))
    t = si.lattice_triangle_problem(21, jitter=0.2, seed=3, t_end=0.8)
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, t, 4, 16, 2, rt.RT_HEUN, 12)
    assert rel_l2(psi, ref) <= PSI_TOL
    check_qoi(q, acc, S, 3, scale=S["mass"])


def test_triangles_second_order_bf16_and_batch(rt):
    """BF16 storage stays within the measured bound of FP32 storage, and a
    second-order triangle problem batched with a first-order one and a
    Cartesian one equals the same problems alone, bit for bit."""
    p = si.enclosure_problem(30, jitter=0.2, seed=0, t_end=0.6)
    quad = rt.rt_quad_product(4, 16)
    outs = {}
    for storage in (0, 1):
        s = rt.Solver(p, quad, order=2, integrator=rt.RT_HEUN, storage=storage)
        s.step()
        outs[storage] = (s.psi(), s.qoi())
        s.close()
    assert rel_l2(outs[1][0], outs[0][0]) < 3e-2
    probs = [p, si.enclosure_problem(20, jitter=0.2, seed=4, t_end=0.6), si.lattice_problem(28, t_end=0.6)]
    orders = [2, 1, 2]
    quads = [quad, rt.rt_quad_product(2, 16), rt.rt_quad_product(4, 16)]
    b = rt.Batch(probs, quads, orders=orders, integrators=[rt.RT_HEUN] * 3)
    b.run()
    for i, (pr, qd, od) in enumerate(zip(probs, quads, orders)):
        s = rt.Solver(pr, qd, order=od, integrator=rt.RT_HEUN)
        s.step()
        a, c = b.qoi(i), s.qoi()
        assert np.array_equal(b.psi(i), s.psi()), i
        s.close()
        for k in ("mass", "abs_int", "outflow_int"):
            assert np.array_equal(np.asarray(a[k]), np.asarray(c[k])), (i, k)
    b.close()


@pytest.mark.parametrize("integrator", ["euler", "heun"])
def test_enclosure_triangles(rt, integrator):
    """Jittered split-square enclosure mesh (2*40^2 triangles), 4x16 ordinates."""
    p = si.enclosure_problem(40, jitter=0.2, seed=0)
    integ = rt.RT_EULER if integrator == "euler" else rt.RT_HEUN
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, p, 4, 16, 1, integ, 25)
    n_ref, dt_ref = oracle.triangle_dt(op, p.t_end)
    assert info.n_steps == n_ref and abs(info.dt - dt_ref) < 1e-15
    assert rel_l2(psi, ref) <= PSI_TOL
    check_qoi(q, acc, S, 4, scale=S["mass"] + sum(acc.abs_int))


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("integrator", ["euler", "heun"])
@pytest.mark.parametrize("n_p,n_phi", [(2, 16), (4, 16), (8, 32), (6, 16)])
def test_staged_triangle_kernel_matches_gathering_kernel(rt, n_p, n_phi, integrator, storage):
    """First order on triangles: the kernel that stages each 32-cell chunk's
    rows (own, halo, psi^n) in shared memory computes what the kernel that
    gathers neighbour rows from global memory computes (the same operations
    per element, some on FP32 pairs), and both match the oracle. 30^2 split
    mesh (57 chunks, ragged last chunk), 32 to 256 ordinates (1, 2 and 4
    ordinates per lane)."""
    p = si.enclosure_problem(30, jitter=0.2, seed=5)
    M = n_p * n_phi
    psi0 = si.random_psi(p.mesh.n_cells, M, seed=31)
    quad = rt.rt_quad_product(n_p, n_phi)
    integ = rt.RT_HEUN if integrator == "heun" else rt.RT_EULER
    out = {}
    for staged in (1, 0):
        s = rt.Solver(p, quad, order=1, integrator=integ, storage=storage)
        rt.rt_debug_set(s.h, "tri_staged", staged)
        assert rt.rt_info(s.h).variant == (3 if staged else 0)
        s.set_psi(psi0)
        s.step(5)
        out[staged] = (s.psi(), s.qoi(), s.info.dt)
        s.close()
    a, b = out[1][0], out[0][0]
    if storage == 0:
        assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(b))
    else:
        # Both kernels take the same stochastic-rounding bits per (cell, ordinate, step,
        # stage) but order some FP32 operations differently (scalar-flux sums, ordinate
        # pairs): rarely an element rounds to the other neighbouring BF16 value, and the
        # later steps carry that difference downstream. So the two agree nearly everywhere
        # bit for bit and to the BF16 level in L2; each is checked against the oracle below.
        assert np.mean(a != b) <= 1e-2
        assert rel_l2(a, b) <= 1e-3
    op = oracle.TriangleOracle(p, oracle.product_quadrature(n_p, n_phi), order=1)
    start = psi0.astype(np.float32).astype(np.float64)
    ref, acc, S = oracle.run(op, start, out[1][2], 5, integrator)
    if storage == 0:
        assert rel_l2(a, ref) <= PSI_TOL
        check_qoi(out[1][1], acc, S, len(S["abs"]), scale=S["mass"])
    else:
        # BF16 level: each of the 5 stores (10 with Heun) rounds by at most one unit
        # (2^-7 relative) with mean zero
        assert rel_l2(a, ref) <= 2e-2 and rel_l2(b, ref) <= 2e-2


def test_tri_staged_hook_rejects_other_solvers(rt):
    s = rt.Solver(si.lattice_problem(14), rt.rt_quad_product(2, 8), dt=0.25)
    with pytest.raises(rt.RTError) as e:
        rt.rt_debug_set(s.h, "tri_staged", 0)
    assert e.value.code == rt.RT_EINVAL
    s.close()


@pytest.mark.parametrize("n_p,n_phi", [(2, 16), (4, 16), (8, 32), (6, 16), (16, 32)])
def test_triangle_random_state_vector_widths(rt, n_p, n_phi):
    """Random state, one Euler step, ordinate counts 32/64/256/96/512 (1, 2 and
    4 ordinates per lane per access; 512 is gathered in several ordinate
    blocks per cell)."""
    p = si.enclosure_problem(18, jitter=0.2, seed=5)
    M = n_p * n_phi
    psi0 = si.random_psi(p.mesh.n_cells, M, seed=2)
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, p, n_p, n_phi, 1, rt.RT_EULER, 1, psi0=psi0)
    assert np.max(np.abs(psi - ref)) <= 2e-6 * np.max(np.abs(ref))
    check_qoi(q, acc, S, 4, scale=S["mass"])


@pytest.mark.parametrize("storage", [0, 1])
def test_triangle_heun_blocks_and_storage(rt, storage):
    """Heun (stage 2 gathers psi^n beside the neighbour rows) with 512
    ordinates in several blocks per cell, FP32 and BF16 storage, from a
    random state over 3 steps."""
    p = si.enclosure_problem(14, jitter=0.2, seed=9)
    psi0 = si.random_psi(p.mesh.n_cells, 512, seed=4)
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, p, 16, 32, 1, rt.RT_HEUN, 3, psi0=psi0, storage=storage)
    if storage == 0:
        assert rel_l2(psi, ref) <= PSI_TOL
        check_qoi(q, acc, S, 4, scale=S["mass"])
    else:
        assert rel_l2(psi, ref) <= 2e-2


def test_cartesian_ordinates_not_multiple_of_128(rt):
    """96 ordinates: the initial-state and conversion kernels take 1 ordinate
    per lane (32 divides 96, 64 and 128 do not)."""
    p = si.lattice_problem(21)
    psi0 = si.random_psi(p.mesh.n_cells, 96, seed=8)
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, p, 6, 16, 2, rt.RT_HEUN, 2, psi0=psi0, dt=0.5 * p.mesh.dx)
    assert rel_l2(psi, ref) <= PSI_TOL
    assert rel_l2(phi, op.phi(ref)) <= PSI_TOL
    check_qoi(q, acc, S, 3, scale=S["mass"])


def test_lattice_on_triangles(rt):
    p = si.lattice_triangle_problem(28, jitter=0.2, seed=1)
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, p, 2, 16, 1, rt.RT_EULER, 20)
    assert rel_l2(psi, ref) <= PSI_TOL
    bal = q["mass"] + sum(q["abs_int"]) + q["outflow_int"]
    assert abs(bal / q["source_int"] - 1) < 1e-5


# ------------------------------------------------------------------ BF16 storage
def test_bf16_storage_error_is_bounded(rt):
    """psi stored in bf16 (FP32 arithmetic): error against the FP64 oracle stays
    at the bf16 rounding level (2^-9 relative per store), measured here."""
    p = si.lattice_problem(70)
    psi, phi, q, ref, acc, S, op, info = run_pair(rt, p, 4, 16, 1, rt.RT_EULER, 64, dt=0.05, storage=rt.RT_BF16)
    e = rel_l2(psi, ref)
    assert e < 2e-2, e
    assert rel(q["abs_int"][1], acc.abs_int[1]) < 1e-2
    assert rel(q["mass"], S["mass"]) < 1e-2


@pytest.mark.parametrize("kind", ["enclosure", "lattice"])
def test_bf16_small_steps_keep_the_particle_balance(rt, kind):
    """Many small steps (the triangle time step comes from the smallest cells,
    so most cells change by a small fraction of a BF16 unit per step): BF16
    stores round stochastically, so the state keeps moving and the particle
    balance mass + absorbed + outflow = emitted holds at the BF16 level, and
    the QoIs stay close to the FP32 run's."""
    if kind == "enclosure":
        p = si.enclosure_problem(100, jitter=0.2, seed=2, t_end=0.6)
        quad, order, integ, dt = rt.rt_quad_product(4, 16), 1, rt.RT_EULER, 0.0
    else:
        p = si.lattice_problem(56, t_end=1.6)
        quad, order, integ, dt = rt.rt_quad_product(4, 16), 2, rt.RT_HEUN, 0.05 * 7.0 / 56
    res = {}
    for storage in (rt.RT_FP32, rt.RT_BF16):
        s = rt.Solver(p, quad, order=order, integrator=integ, storage=storage, dt=dt)
        s.step()
        res[storage] = (s.qoi(), s.info.n_steps)
        s.close()
    q32, n = res[rt.RT_FP32]
    q16, _ = res[rt.RT_BF16]
    assert n >= 100
    budget = abs(q32["mass"]) + float(np.sum(np.abs(q32["abs_int"]))) + abs(q32["outflow_int"])
    for q, tol in ((q32, 1e-5), (q16, 2e-3)):
        bal = q["mass"] + float(np.sum(q["abs_int"])) + q["outflow_int"] - q["source_int"]
        assert abs(bal) <= tol * budget, (bal, budget)
    assert rel(q16["mass"], q32["mass"]) < 2e-2
    assert abs(float(np.sum(q16["abs_int"])) - float(np.sum(q32["abs_int"]))) < 2e-2 * budget


# ------------------------------------------------------------------ execution paths
def test_graph_replay_matches_direct_launches_bitwise(rt):
    p = si.lattice_problem(49)
    quad = rt.rt_quad_product(2, 16)
    a = rt.Solver(p, quad, order=2, integrator=rt.RT_HEUN, dt=0.5 * p.mesh.dx)
    b = rt.Solver(p, quad, order=2, integrator=rt.RT_HEUN, dt=0.5 * p.mesh.dx)
    a.step(40)               # graph path (16-step graphs) + 8 direct steps
    for _ in range(40):
        b.step(1)            # direct launches only
    assert np.array_equal(a.psi(), b.psi())
    qa, qb = a.qoi(), b.qoi()
    for k in qa:
        assert np.array_equal(np.asarray(qa[k]), np.asarray(qb[k])), k
    a.close()
    b.close()


def test_checkpoint_resume_is_bitwise(rt):
    p = si.lattice_problem(42)
    quad = rt.rt_quad_product(2, 16)
    a = rt.Solver(p, quad, order=1, integrator=rt.RT_EULER, dt=0.5 * p.mesh.dx)
    a.step(11)
    blob = rt.rt_get_state(a.h)
    a.step(9)
    qa, pa = a.qoi(), a.psi()
    b = rt.Solver(p, quad, order=1, integrator=rt.RT_EULER, dt=0.5 * p.mesh.dx)
    rt.rt_set_state(b.h, blob)
    b.step(9)
    qb, pb = b.qoi(), b.psi()
    assert np.array_equal(pa, pb)
    for k in qa:
        assert np.array_equal(np.asarray(qa[k]), np.asarray(qb[k])), k
    a.close()
    b.close()


def test_step_clamps_at_final_time(rt):
    p = si.lattice_problem(14)
    s = rt.Solver(p, rt.rt_quad_product(2, 4), dt=0.25)
    s.step(1000)
    q = s.qoi()
    assert q["step"] == s.info.n_steps and abs(q["t"] - p.t_end) < 1e-12
    s.close()


def test_timeout_reports_status_and_context_survives(rt):
    """A wait with a tiny limit on a load that is never issued: the kernel gives
    up, reports RT_ETIMEOUT, and the GPU stays usable."""
    p = si.lattice_problem(35)
    quad = rt.rt_quad_product(2, 16)
    s = rt.Solver(p, quad, dt=0.1)
    rt.rt_debug_set(s.h, "wait_limit_cycles", 2_000_000)
    rt.rt_debug_set(s.h, "drop_load", 3)
    s.step(1)
    with pytest.raises(rt.RTError) as e:
        s.qoi()
    assert e.value.code == rt.RT_ETIMEOUT
    with pytest.raises(rt.RTError) as e:
        s.step(1)
    assert e.value.code == rt.RT_ESTATE
    s.close()
    # a fresh solver on the same context works
    t = rt.Solver(p, quad, dt=0.1)
    t.step(3)
    assert t.qoi()["step"] == 3
    t.close()


def test_nonfinite_is_detected(rt):
    p = si.lattice_problem(14)
    p.materials.sigma_a = np.array([0.0, 3.0e38, 0.0])
    s = rt.Solver(p, rt.rt_quad_product(2, 4), dt=0.25)
    s.step(6)
    with pytest.raises(rt.RTError) as e:
        s.qoi()
    assert e.value.code == rt.RT_ENONFINITE
    s.close()


def test_set_psi_roundtrip_and_device_view(rt):
    import torch
    p = si.lattice_problem(21)
    s = rt.Solver(p, rt.rt_quad_product(2, 8), dt=0.1)
    psi0 = si.random_psi(p.mesh.n_cells, 16, seed=4)
    s.set_psi(psi0)
    back = s.psi()
    assert np.max(np.abs(back - psi0)) <= 1e-7 * np.max(psi0)     # FP32 rounding
    q = s.qoi()
    op = oracle.CartesianOracle(p, oracle.product_quadrature(2, 8))
    assert rel(q["mass"], op.integrands(psi0)["mass"]) < 1e-6
    ptr, phiptr, storage = rt.rt_device_state(s.h)
    assert ptr and phiptr and storage == rt.RT_FP32
    s.close()


def test_psi_cells_equals_rows_of_the_whole_state(rt):
    """rt_get_psi_cells returns the caller's rows on both mesh kinds (triangles
    are stored in a different order on the device), for repeated and unsorted
    ids; an id out of range is rejected and changes nothing."""
    for p, order in ((si.lattice_problem(28, t_end=0.3), 2), (si.enclosure_problem(12, t_end=0.3), 2)):
        s = rt.Solver(p, rt.rt_quad_product(2, 16), order=order, integrator=rt.RT_HEUN)
        s.set_psi(si.random_psi(p.mesh.n_cells, 32, seed=2))
        s.step(3)
        full = s.psi()
        cells = np.array([5, 0, p.mesh.n_cells - 1, 5, 17, 3])
        assert np.array_equal(s.psi_cells(cells), full[cells])
        assert s.psi_cells(np.array([], dtype=np.int64)).shape == (0, 32)
        with pytest.raises(rt.RTError) as e:
            s.psi_cells(np.array([0, p.mesh.n_cells]))
        assert e.value.code == rt.RT_EINVAL
        assert np.array_equal(s.psi(), full)
        s.close()


# ------------------------------------------------------------------ batches
def test_batch_results_equal_single_solves_bitwise(rt):
    """Mixed grid sizes and ordinate counts in one batch: each problem's result is
    bit-identical to solving it alone (same kernels, same work split, fixed
    reduction order)."""
    inst = [(28, 2, 16, 8.0, 1.2), (35, 4, 16, 12.0, 0.7), (21, 2, 32, 5.5, 1.4)]
    probs, quads = [], []
    for n, n_p, n_phi, sa, ss in inst:
        pr = si.lattice_problem(n, sigma_a_blue=sa, sigma_s_scatter=ss)
        pr.t_end = 1.0
        probs.append(pr)
        quads.append(rt.rt_quad_product(n_p, n_phi))
    dts = [0.5 * pr.mesh.dx for pr in probs]
    b = rt.Batch(probs, quads, order=2, integrator=rt.RT_HEUN, dts=dts)
    b.run()
    for i, (pr, qd) in enumerate(zip(probs, quads)):
        s = rt.Solver(pr, qd, order=2, integrator=rt.RT_HEUN, dt=dts[i])
        s.step()
        assert np.array_equal(b.psi(i), s.psi())
        qa, qb = b.qoi(i), s.qoi()
        assert qa["step"] == qb["step"] == s.info.n_steps
        for k in qa:
            assert np.array_equal(np.asarray(qa[k]), np.asarray(qb[k])), k
        s.close()
    b.close()


def test_batch_against_oracle(rt):
    probs = [si.lattice_problem(21, sigma_a_blue=7.0), si.lattice_problem(14, sigma_a_blue=13.0)]
    for pr in probs:
        pr.t_end = 0.8
    quads = [rt.rt_quad_product(2, 8), rt.rt_quad_product(2, 16)]
    b = rt.Batch(probs, quads, order=2, integrator=rt.RT_HEUN, dts=[0.5 * pr.mesh.dx for pr in probs])
    b.run()
    for i, pr in enumerate(probs):
        n_p, n_phi = (2, 8) if i == 0 else (2, 16)
        op = oracle.CartesianOracle(pr, oracle.product_quadrature(n_p, n_phi), order=2)
        n = oracle.n_steps_for(pr.t_end, 0.5 * pr.mesh.dx)
        ref, acc, S = oracle.run(op, np.zeros((pr.mesh.n_cells, n_p * n_phi)), pr.t_end / n, n, "heun")
        assert rel_l2(b.psi(i), ref) <= PSI_TOL
        check_qoi(b.qoi(i), acc, S, 3, scale=S["mass"])
    b.close()


def _solo(rt, pr, qd, order, integrator, dt, n=None):
    s = rt.Solver(pr, qd, order=order, integrator=integrator, dt=dt)
    s.step(n)
    out = (s.psi(), s.qoi())
    s.close()
    return out


def test_batch_mixed_kinds_and_integrators_bitwise(rt):
    """Cartesian MUSCL-Heun, Cartesian first-order Euler and a triangle mesh in
    one batch: each result is bit-identical to its solve alone."""
    a = si.lattice_problem(28, sigma_a_blue=9.0)
    a.t_end = 0.9
    c = si.enclosure_problem(12, seed=3, t_end=0.5)
    e = si.lattice_problem(35, sigma_s_scatter=0.8)
    e.t_end = 0.6
    probs = [a, c, e]
    quads = [rt.rt_quad_product(2, 16), rt.rt_quad_product(2, 8), rt.rt_quad_product(4, 16)]
    orders = [2, 1, 1]
    integ = [rt.RT_HEUN, rt.RT_EULER, rt.RT_EULER]
    dts = [0.5 * a.mesh.dx, 0.0, 0.5 * e.mesh.dx]
    b = rt.Batch(probs, quads, dts=dts, orders=orders, integrators=integ)
    b.run()
    for i in range(3):
        ref_psi, ref_q = _solo(rt, probs[i], quads[i], orders[i], integ[i], dts[i])
        assert np.array_equal(b.psi(i), ref_psi), i
        q = b.qoi(i)
        for k in q:
            assert np.array_equal(np.asarray(q[k]), np.asarray(ref_q[k])), (i, k)
    b.close()


def test_batch_add_remove_between_steps(rt):
    """Continuous batching: problems join and leave between steps; every
    problem's result still equals its solve alone, and progress counts the
    steps each one has taken."""
    p0 = si.lattice_problem(21, sigma_a_blue=6.0)
    p0.t_end = 2.0                      # 12 steps
    p1 = si.lattice_problem(28, sigma_s_scatter=1.1)
    p1.t_end = 2.0                      # 16 steps
    p2 = si.enclosure_problem(10, seed=7, t_end=0.4)
    q0, q1, q2 = rt.rt_quad_product(2, 8), rt.rt_quad_product(2, 16), rt.rt_quad_product(2, 8)
    dt0, dt1 = 0.5 * p0.mesh.dx, 0.5 * p1.mesh.dx
    b = rt.Batch([p0], [q0], dts=[dt0], capacity=3)
    b.step(3)
    s1 = b.add(p1, q1, order=2, integrator=rt.RT_HEUN, dt=dt1)
    assert s1 == 1
    b.step(5)
    assert b.progress(0)[0] == 8 and b.progress(1)[0] == 5
    psi0_after_8 = b.psi(0)
    b.remove(0)
    with pytest.raises(rt.RTError):
        b.progress(0)
    s2 = b.add(p2, q2, order=1, integrator=rt.RT_EULER)
    assert s2 == 0                      # the freed slot is reused
    b.step(4)
    assert b.progress(1)[0] == 9 and b.progress(0)[0] == 4
    b.run()
    for slot, (pr, qd, o, ig, dt) in ((1, (p1, q1, 2, rt.RT_HEUN, dt1)), (0, (p2, q2, 1, rt.RT_EULER, 0.0))):
        done, total = b.progress(slot)
        assert done == total
        ref_psi, ref_q = _solo(rt, pr, qd, o, ig, dt)
        assert np.array_equal(b.psi(slot), ref_psi), slot
        assert b.qoi(slot)["mass"] == ref_q["mass"]
    # p0 left after 8 of its steps: its state then equals 8 steps alone
    s = rt.Solver(p0, q0, order=2, integrator=rt.RT_HEUN, dt=dt0)
    s.step(8)
    assert np.array_equal(psi0_after_8, s.psi())
    s.close()
    b.close()


def test_batch_launch_count(rt):
    """rt_batch_launches counts what the batch enqueues: two Heun problems of one
    kernel variant, one with the QoI squares (2 + 1 initial launches), then per
    step 2 stage launches and 1 box launch, the same whether a call launches
    directly (the first after a membership change) or replays a graph."""
    probs = [si.lattice_problem(28, t_end=3.2), si.lattice_problem(30, t_end=3.2)]
    probs[1].extra = {}
    quads = [rt.rt_quad_product(4, 16), rt.rt_quad_product(4, 16)]
    b = rt.Batch(probs, quads, order=2, integrator=rt.RT_HEUN, dts=[0.5 * pr.mesh.dx for pr in probs])
    assert b.launches() == 3
    b.step(1)             # rebuilt work list: direct launches
    assert b.launches() == 3 + 3
    b.step(4)             # captured graph
    b.step(4)             # replayed graph
    assert b.launches() == 3 + 3 + 2 * 4 * 3
    b.close()


def test_batch_capacity_and_empty_slots(rt):
    p = si.lattice_problem(14)
    p.t_end = 0.3
    q = rt.rt_quad_product(2, 8)
    b = rt.Batch([], [], capacity=1)
    b.step(2)                           # nothing to do
    slot = b.add(p, q, order=1, integrator=rt.RT_EULER)
    with pytest.raises(rt.RTError) as e:
        b.add(p, q, order=1, integrator=rt.RT_EULER)
    assert e.value.code == rt.RT_EINVAL and "no free slot" in rt.rt_last_error()
    with pytest.raises(rt.RTError):
        b.qoi(slot + 1)
    b.run()
    done, total = b.progress(slot)
    assert done == total > 0
    b.step(3)                           # finished problems do not step further
    assert b.progress(slot)[0] == total
    b.close()


# ------------------------------------------------------------------ autotuner
def test_autotune_picks_a_buildable_config_that_matches_the_oracle(rt):
    p = si.lattice_problem(63)
    p.t_end = 0.6
    quad = rt.rt_quad_product(8, 32)
    cfg, ms = rt.rt_autotune(p, quad, order=2, integrator=rt.RT_HEUN, dt=0.5 * p.mesh.dx, steps=3)
    assert ms > 0
    assert cfg["tile_x"] in (16, 32) and 1 <= cfg["tile_y"] <= 64 and cfg["variant"] in (1, 2)
    s = rt.Solver(p, quad, order=2, integrator=rt.RT_HEUN, dt=0.5 * p.mesh.dx, tile_x=cfg["tile_x"],
                  tile_y=cfg["tile_y"], variant=cfg["variant"], vec=cfg["vec"])
    assert (s.info.tile_x, s.info.tile_y, s.info.variant, s.info.vec) == \
        (cfg["tile_x"], cfg["tile_y"], cfg["variant"], cfg["vec"])
    s.step()
    psi, q, dt, n = s.psi(), s.qoi(), s.info.dt, s.info.n_steps
    s.close()
    op = oracle.CartesianOracle(p, oracle.product_quadrature(8, 32), order=2)
    ref, acc, S = oracle.run(op, np.zeros((p.mesh.n_cells, 256)), dt, n, "heun")
    assert rel_l2(psi, ref) <= PSI_TOL
    check_qoi(q, acc, S, 3, scale=S["mass"])


def test_autotune_cache_and_solver_flag(rt, tmp_path, monkeypatch):
    from paper_2505_17284_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE_PATH", str(tmp_path / "tune.json"))
    monkeypatch.setattr(autotune, "_mem", None)
    p = si.lattice_problem(42)
    quad = rt.rt_quad_product(4, 16)
    a = autotune.tuned_config(p, quad, 1, rt.RT_EULER, dt=0.5 * p.mesh.dx)
    assert (tmp_path / "tune.json").exists()
    b = autotune.tuned_config(p, quad, 1, rt.RT_EULER, dt=0.5 * p.mesh.dx)
    assert a == b                         # second call from the cache
    s = rt.Solver(p, quad, order=1, integrator=rt.RT_EULER, dt=0.5 * p.mesh.dx, tune=True)
    assert (s.info.tile_x, s.info.tile_y) == (a["tile_x"], a["tile_y"])
    s.close()


def test_autotune_rejects_triangles(rt):
    p = si.enclosure_problem(8, seed=1, t_end=0.2)
    with pytest.raises(rt.RTError) as e:
        rt.rt_autotune(p, rt.rt_quad_product(2, 8), order=1, integrator=rt.RT_EULER)
    assert e.value.code == rt.RT_EINVAL


# ------------------------------------------------------------------ tessellation quadrature (Sec. 5.1.1)
@pytest.mark.parametrize("N,n", [(4, 63), (8, 63), (22, 28)])
def test_tessellation_quadrature_cartesian(rt, N, n):
    """The paper's tessellation rule (64, 256 and 1936 ordinates: per-lane,
    32-cell chunk-uniform (asked for with tile_x 32: on a grid this small the
    library picks the per-lane kernel) and chunk-uniform kernels), MUSCL Heun
    from a smooth state against the oracle."""
    p = si.lattice_problem(n)
    M = 4 * N * N
    psi0 = si.smooth_psi(p.mesh, M, seed=6)
    quad = rt.rt_quad_tessellation(N)
    s = rt.Solver(p, quad, order=2, integrator=rt.RT_HEUN, dt=0.5 * p.mesh.dx, tile_x=32 if N == 8 else 0)
    assert N != 8 or (s.info.variant == 2 and s.info.tile_x == 32)
    # 484 ordinates per quadrant: stored regrouped, each quadrant padded to 512
    assert s.info.regrouped == (N == 22) and (N != 22 or (s.info.M_pad == 2048 and s.info.variant == 2))
    s.set_psi(psi0)
    assert np.array_equal(s.psi(), psi0.astype(np.float32).astype(np.float64))   # caller's order both ways
    steps = 4
    s.step(steps)
    psi, q, dt = s.psi(), s.qoi(), s.info.dt
    s.close()
    op = oracle.CartesianOracle(p, oracle.tessellation_quadrature(N), order=2)
    ref, acc, S = oracle.run(op, psi0, dt, steps, "heun")
    assert rel_l2(psi, ref) <= PSI_TOL
    check_qoi(q, acc, S, 3, scale=S["mass"])


def test_tessellation_quadrature_triangles(rt):
    p = si.enclosure_problem(20, jitter=0.2, seed=3)
    quad = rt.rt_quad_tessellation(4)
    psi0 = si.random_psi(p.mesh.n_cells, 64, seed=9)
    s = rt.Solver(p, quad, order=1, integrator=rt.RT_EULER)
    s.set_psi(psi0)
    s.step(5)
    psi, q, dt = s.psi(), s.qoi(), s.info.dt
    s.close()
    op = oracle.TriangleOracle(p, oracle.tessellation_quadrature(4))
    ref, acc, S = oracle.run(op, psi0, dt, 5, "euler")
    assert rel_l2(psi, ref) <= PSI_TOL
    check_qoi(q, acc, S, 4, scale=S["mass"])


def test_regrouped_product_quadrature(rt):
    """12 x 40 product rule: 120 ordinates per quadrant, so chunks of the
    caller's order mix signs; stored regrouped (quadrants padded to 128) and
    run on the chunk-uniform kernel, against the oracle; psi round-trips in the
    caller's order and a checkpoint resumes bit for bit."""
    p = si.lattice_problem(28)
    quad = rt.rt_quad_product(12, 40)
    psi0 = si.smooth_psi(p.mesh, 480, seed=2)
    s = rt.Solver(p, quad, order=2, integrator=rt.RT_HEUN, dt=0.5 * p.mesh.dx)
    assert s.info.regrouped == 1 and s.info.M_pad == 512 and s.info.variant == 2
    s.set_psi(psi0)
    s.step(2)
    blob = rt.rt_get_state(s.h)
    s.step(2)
    psi, q, dt = s.psi(), s.qoi(), s.info.dt
    s.close()
    b = rt.Solver(p, quad, order=2, integrator=rt.RT_HEUN, dt=0.5 * p.mesh.dx)
    rt.rt_set_state(b.h, blob)
    b.step(2)
    assert np.array_equal(b.psi(), psi)
    b.close()
    op = oracle.CartesianOracle(p, oracle.product_quadrature(12, 40), order=2)
    ref, acc, S = oracle.run(op, psi0, dt, 4, "heun")
    assert rel_l2(psi, ref) <= PSI_TOL
    check_qoi(q, acc, S, 3, scale=S["mass"])
    lane = rt.Solver(p, quad, order=2, integrator=rt.RT_HEUN, dt=0.5 * p.mesh.dx, variant=1)
    assert lane.info.regrouped == 0          # the per-lane kernel keeps the caller's order
    lane.close()

"""GPU parity at the production sizes, in the launch configuration the bench
times: the lattice at 1400^2 x 512 ordinates (MUSCL, Heun, FP32, autotuned
tiles, QoI squares attached) and the enclosure at 1300^2 split (3.38e6
triangles) x 256 ordinates (first order, Euler, FP32; and the paper's second
order scheme with Heun).

The whole state is too large for the oracle, so sampled cells are checked one
by one: the value of a cell after K steps depends only on the cells within the
scheme's domain of dependence (4 cells per Heun step with MUSCL, one triangle
per Euler step at first order, four per Heun step at second order on
triangles), so the oracle solves a patch around the cell,
wide enough that its artificial edges cannot reach the centre in K steps, from
the same initial state (psi = 0) with the same dt. Properties that hold at any
size are checked on the whole state: the particle balance and, for the
lattice, the mirror symmetry about x = 3.5.
"""
import numpy as np
import pytest

import oracle
import sn_inputs as si

pytestmark = pytest.mark.gpu

PSI_TOL = 1e-5


@pytest.fixture(scope="module")
def rt():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2505_17284_gb300 import build, rt as rtmod
    build.build()
    rtmod.load_library()
    return rtmod


def lattice_patch(p, ci, cj, R):
    """The cells of lattice problem p within R cells of (ci, cj), clipped to the
    domain (its sides stay vacuum), as a problem of its own; returns it and the
    patch index of (ci, cj)."""
    n = p.mesh.nx
    i0, i1, j0, j1 = max(0, ci - R), min(n, ci + R + 1), max(0, cj - R), min(n, cj + R + 1)
    m = p.mesh
    mesh = si.CartesianMesh(nx=i1 - i0, ny=j1 - j0, x0=m.x0 + i0 * m.dx, y0=m.y0 + j0 * m.dy, dx=m.dx, dy=m.dy)
    idx = (np.arange(j0, j1)[:, None] * n + np.arange(i0, i1)[None, :]).ravel()
    mt = p.materials
    mats = si.Materials(sigma_a=mt.sigma_a, sigma_s=mt.sigma_s, Q=mt.Q, cell_mat=mt.cell_mat[idx],
                        cell_region=mt.cell_region[idx], region_names=mt.region_names)
    return si.Problem(mesh=mesh, materials=mats, boundary=si.Boundary(), t_end=p.t_end), \
        (cj - j0) * (i1 - i0) + (ci - i0)


def triangle_patch(p, n, ci, cj, R):
    """The triangles of the squares within R squares of square (ci, cj) of the
    n x n split mesh of p (same vertices), with p's inflow side only where the
    patch touches x = 0; returns the problem and the patch ids of the two
    triangles of square (ci, cj)."""
    i0, i1, j0, j1 = max(0, ci - R), min(n, ci + R + 1), max(0, cj - R), min(n, cj + R + 1)
    sq = (np.arange(j0, j1)[:, None] * n + np.arange(i0, i1)[None, :]).ravel()
    tri_ids = np.stack([2 * sq, 2 * sq + 1], axis=1).ravel()
    T = p.mesh.triangles[tri_ids]
    vids, inv = np.unique(T.ravel(), return_inverse=True)
    V = p.mesh.vertices[vids]
    mesh = si.TriangleMesh(vertices=V, triangles=inv.reshape(-1, 3).astype(np.int32),
                           box=(V[:, 0].min(), V[:, 1].min(), V[:, 0].max(), V[:, 1].max()))
    mt = p.materials
    mats = si.Materials(sigma_a=mt.sigma_a, sigma_s=mt.sigma_s, Q=mt.Q, cell_mat=mt.cell_mat[tri_ids],
                        cell_region=mt.cell_region[tri_ids], region_names=mt.region_names)
    b = p.boundary
    bc = si.Boundary(kind=(b.kind[0] if i0 == 0 else si.VACUUM, si.VACUUM, si.VACUUM, si.VACUUM),
                     inflow=(b.inflow[0] if i0 == 0 else 0.0, 0.0, 0.0, 0.0))
    local_sq = (cj - j0) * (i1 - i0) + (ci - i0)
    return si.Problem(mesh=mesh, materials=mats, boundary=bc, t_end=p.t_end), (2 * local_sq, 2 * local_sq + 1)


def test_lattice_1400_production_sampled_parity(rt):
    n, K = 1400, 4
    p = si.lattice_problem(n)
    s = rt.Solver(p, rt.rt_quad_product(16, 32), order=2, integrator=rt.RT_HEUN, dt=0.5 * p.mesh.dx, tune=True)
    s.step(K)
    info, q = s.info, s.qoi()
    rng = np.random.default_rng(7)
    # the source block [3,4]^2 is cells 600..799; after K steps the state is
    # nonzero there and within a few cells of it; far cells stay exactly 0
    inside = rng.integers(600, 800, size=(24, 2))
    band = np.concatenate([rng.integers(584, 600, size=(8, 2)), rng.integers(800, 816, size=(8, 2))])
    band[::2, 0] = rng.integers(600, 800, size=8)       # edge bands in x and in y
    far = np.stack([rng.integers(0, n, size=8), rng.integers(0, 400, size=8)], axis=1)
    cells_ij = np.concatenate([inside, band, far])
    cells = cells_ij[:, 1] * n + cells_ij[:, 0]
    gpu = s.psi_cells(cells)
    phi = s.phi()
    s.close()
    quad = oracle.product_quadrature(16, 32)
    ref = np.empty_like(gpu)
    for r, (ci, cj) in enumerate(cells_ij):
        pp, c = lattice_patch(p, int(ci), int(cj), 4 * K + 1)
        op = oracle.CartesianOracle(pp, quad, order=2)
        psi, _, _ = oracle.run(op, np.zeros((pp.mesh.n_cells, 512)), info.dt, K, "heun")
        ref[r] = psi[c]
    scale = np.abs(ref).max()
    assert scale > 0
    assert float(np.linalg.norm(gpu - ref) / np.linalg.norm(ref)) <= PSI_TOL
    assert np.max(np.abs(gpu - ref)) <= 10 * PSI_TOL * scale
    assert np.all(gpu[-8:] == 0.0)
    # whole state: particle balance and mirror symmetry about x = 3.5
    bal = q["mass"] + sum(q["abs_int"]) + q["outflow_int"]
    assert abs(bal / q["source_int"] - 1) <= 1e-5
    ph = phi.reshape(n, n)
    assert np.max(np.abs(ph - ph[:, ::-1])) <= 1e-5 * ph.max()


def test_enclosure_1300_production_sampled_parity(rt):
    n, K = 1300, 6
    p = si.enclosure_problem(n, jitter=0.2, seed=0)
    s = rt.Solver(p, rt.rt_quad_product(8, 32), order=1, integrator=rt.RT_EULER)
    s.step(K)
    info, q = s.info, s.qoi()
    rng = np.random.default_rng(9)
    # inflow enters through the opening of the left wall, y in [0.4, 0.9]
    # (squares 400..692); after K steps the state is nonzero within a few
    # squares of x = 0 there
    near = np.stack([rng.integers(0, 5, size=24), rng.integers(400, 693, size=24)], axis=1)
    wall = np.stack([rng.integers(0, 5, size=6), rng.integers(0, 380, size=6)], axis=1)
    far = np.stack([rng.integers(200, n, size=6), rng.integers(0, n, size=6)], axis=1)
    sq_ij = np.concatenate([near, wall, far])
    cells = np.concatenate([[2 * (j * n + i), 2 * (j * n + i) + 1] for i, j in sq_ij])
    gpu = s.psi_cells(cells)
    s.close()
    quad = oracle.product_quadrature(8, 32)
    ref = np.empty_like(gpu)
    for r, (ci, cj) in enumerate(sq_ij):
        pp, (c0, c1) = triangle_patch(p, n, int(ci), int(cj), K + 2)
        op = oracle.TriangleOracle(pp, quad, order=1)
        psi, _, _ = oracle.run(op, np.zeros((pp.mesh.n_cells, 256)), info.dt, K, "euler")
        ref[2 * r], ref[2 * r + 1] = psi[c0], psi[c1]
    scale = np.abs(ref).max()
    assert scale > 0
    assert float(np.linalg.norm(gpu - ref) / np.linalg.norm(ref)) <= PSI_TOL
    assert np.max(np.abs(gpu - ref)) <= 10 * PSI_TOL * scale
    assert np.all(gpu[-12:] == 0.0)
    # whole state: particle balance (no source: mass + absorbed + outflow = 0)
    bal = q["mass"] + sum(q["abs_int"]) + q["outflow_int"]
    assert abs(bal) <= 1e-5 * (q["mass"] + sum(q["abs_int"]))


def test_enclosure_1300_second_order_sampled_parity(rt):
    """The paper's production scheme (Green-Gauss + Venkatakrishnan, Heun) at
    1300^2 split x 256: each stage reaches two triangles, so a step reaches
    four and the patch has half-width 4K + 2 squares."""
    n, K = 1300, 3
    p = si.enclosure_problem(n, jitter=0.2, seed=0)
    s = rt.Solver(p, rt.rt_quad_product(8, 32), order=2, integrator=rt.RT_HEUN)
    s.step(K)
    info, q = s.info, s.qoi()
    rng = np.random.default_rng(11)
    near = np.stack([rng.integers(0, 6, size=16), rng.integers(400, 693, size=16)], axis=1)
    far = np.stack([rng.integers(200, n, size=4), rng.integers(0, n, size=4)], axis=1)
    sq_ij = np.concatenate([near, far])
    cells = np.concatenate([[2 * (j * n + i), 2 * (j * n + i) + 1] for i, j in sq_ij])
    gpu = s.psi_cells(cells)
    s.close()
    quad = oracle.product_quadrature(8, 32)
    ref = np.empty_like(gpu)
    for r, (ci, cj) in enumerate(sq_ij):
        pp, (c0, c1) = triangle_patch(p, n, int(ci), int(cj), 4 * K + 2)
        op = oracle.TriangleOracle(pp, quad, order=2)
        psi, _, _ = oracle.run(op, np.zeros((pp.mesh.n_cells, 256)), info.dt, K, "heun")
        ref[2 * r], ref[2 * r + 1] = psi[c0], psi[c1]
    assert np.abs(ref).max() > 0
    assert float(np.linalg.norm(gpu - ref) / np.linalg.norm(ref)) <= PSI_TOL
    assert np.all(gpu[-8:] == 0.0)
    bal = q["mass"] + sum(q["abs_int"]) + q["outflow_int"]
    assert abs(bal) <= 1e-5 * (q["mass"] + sum(q["abs_int"]))

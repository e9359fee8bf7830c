"""Checks of the seeded input generators: RNG test vector, lattice and
enclosure geometry, split-square meshes and the sweep draws."""
import numpy as np

import sn_inputs as si


def test_splitmix64_published_vector():
    # splitmix64 seeded with 1234567: the first five outputs of the reference generator
    out = si.splitmix64(1234567, np.arange(5, dtype=np.uint64))
    assert [int(v) for v in out] == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                     4593380528125082431, 16408922859458223821]
    u = si.uniform01(0, np.arange(100000, dtype=np.uint64))
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.01


def test_lattice_geometry():
    # Sec. 3.1: 11 blue blocks, red centre block, the rest white; 100 cells per block at n = 70
    p = si.lattice_problem(70)
    mat = p.materials.cell_mat.reshape(70, 70)
    assert (mat == si.MAT_BLUE).sum() == 1100
    assert (mat == si.MAT_RED).sum() == 100
    assert np.all(mat[30:40, 30:40] == si.MAT_RED)
    # mirror symmetric about x = 3.5, not about y = 3.5
    assert np.array_equal(mat, mat[:, ::-1])
    assert not np.array_equal(mat, mat[::-1, :])
    # paper's C_{4,6} (0-based block (3,5)) is white
    assert np.all(mat[50:60, 30:40] == si.MAT_WHITE)
    assert p.mesh.dx == 0.1


def test_enclosure_geometry_areas():
    n = 260
    p = si.enclosure_cartesian_problem(n)
    mat = p.materials.cell_mat
    A = (1.3 / n) ** 2
    wall = (mat == si.ENC_WALL).sum() * A
    rim = (mat == si.ENC_RIM).sum() * A
    core = (mat == si.ENC_CORE).sum() * A
    # core 0.3 x 0.7; rim 0.4 x 0.8 minus core; walls: 2 x 1.3 x 0.05 + 2 x 1.2 x 0.05 - opening 0.5 x 0.05
    assert abs(core - 0.21) < 1e-9
    assert abs(rim - (0.32 - 0.21)) < 1e-9
    assert abs(wall - (0.13 + 0.12 - 0.025)) < 1e-9


def test_split_mesh_jitter_bounds():
    n, L = 30, 1.3
    m0 = si.split_grid_mesh(n, L)
    m = si.split_grid_mesh(n, L, jitter=0.2, seed=0)
    d = np.abs(m.vertices - m0.vertices)
    assert d.max() <= 0.2 * L / n + 1e-15
    on_bnd = (m0.vertices[:, 0] == 0) | (m0.vertices[:, 0] == L) | (m0.vertices[:, 1] == 0) | (m0.vertices[:, 1] == L)
    assert np.all(d[on_bnd] == 0)
    assert d[~on_bnd].max() > 0.15 * L / n
    # same seed, same mesh; triangles stay counter-clockwise
    assert np.array_equal(m.vertices, si.split_grid_mesh(n, L, jitter=0.2, seed=0).vertices)
    v = m.vertices[m.triangles]
    cr = (v[:, 1, 0] - v[:, 0, 0]) * (v[:, 2, 1] - v[:, 0, 1]) - (v[:, 1, 1] - v[:, 0, 1]) * (v[:, 2, 0] - v[:, 0, 0])
    assert cr.min() > 0.2 * (L / n) ** 2


def test_sweep_draws():
    inst = si.sweep_instances(256, seed=0)
    assert len(inst) == 256
    assert {i.n for i in inst} == {70, 140, 280, 560}
    assert {i.M for i in inst} == {64, 128, 256}
    assert all(5 <= i.sigma_a <= 15 and 0.5 <= i.sigma_s <= 1.5 for i in inst)
    assert inst[3].n == si.sweep_instances(4, seed=0)[3].n
    t = si.poisson_arrivals(2000, rate=10.0, seed=0)
    assert np.all(np.diff(t) > 0) and abs(t[-1] / 2000 - 0.1) < 0.01


def test_dp2_nominal_is_the_lattice():
    """At the nominal per-block values the DP-2 lattice (49 materials, Sec.
    3.1.3) gives every cell the cross-sections and source of the three-material
    checkerboard, and the oracle's solution is the same to the bit."""
    import oracle
    sa, ss = si.lattice_dp2_nominal()
    assert sa.shape == (7, 7) and sa[1, 1] == 10.0 and ss[1, 1] == 0.0 and ss[0, 0] == 1.0
    p, q = si.lattice_dp2_problem(14, sa, ss, t_end=0.4), si.lattice_problem(14, t_end=0.4)
    P, Q = p.materials, q.materials
    assert len(P.sigma_a) == 49 and P.cell_mat.max() == 48
    for f in ("sigma_a", "sigma_s", "Q"):
        assert np.array_equal(getattr(P, f)[P.cell_mat], getattr(Q, f)[Q.cell_mat]), f
    assert np.array_equal(P.cell_region, Q.cell_region)
    # material id is the block index 7 j + i of the cell's block
    xc, yc = p.mesh.centres()
    assert np.array_equal(P.cell_mat, 7 * np.floor(yc).astype(int) + np.floor(xc).astype(int))
    quad = oracle.product_quadrature(2, 8)
    outs = []
    for pr in (p, q):
        op = oracle.CartesianOracle(pr, quad, order=2)
        outs.append(oracle.run(op, np.zeros((pr.mesh.n_cells, 16)), 0.25, 8, "heun"))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1].abs_int, outs[1][1].abs_int)


def test_dp2_draws():
    inst = si.dp2_instances(64, seed=3)
    bi, bj = np.meshgrid(np.arange(7), np.arange(7), indexing="ij")
    blue = si.lattice_block_material(bi, bj) == si.MAT_BLUE
    assert blue.sum() == 11
    for d in inst:
        assert d.sigma_a.shape == (7, 7) and d.sigma_s.shape == (7, 7)
        assert np.all((d.sigma_a[blue] >= 5) & (d.sigma_a[blue] <= 15))
        assert np.all((d.sigma_s[blue] >= 0) & (d.sigma_s[blue] <= 0.5))
        assert np.all((d.sigma_a[~blue] >= 0) & (d.sigma_a[~blue] <= 0.5))
        assert np.all((d.sigma_s[~blue] >= 0.5) & (d.sigma_s[~blue] <= 1.5))
        assert len(np.unique(d.sigma_a)) == 49 and len(np.unique(d.sigma_s)) == 49
    assert {d.n for d in inst} == {70, 140, 280, 560} and {d.M for d in inst} == {64, 128, 256}
    again = si.dp2_instances(8, seed=3)
    assert all(np.array_equal(a.sigma_a, b.sigma_a) and a.n == b.n for a, b in zip(inst[:8], again))
    # draw order: block (i, j) takes draw 2 + 7 j + i of its instance
    u = si.uniform01(3, np.arange(100, 200, dtype=np.uint64))
    assert inst[1].sigma_a[2, 0] == 0.5 * u[2 + 2]
    assert inst[1].sigma_a[1, 1] == 5.0 + 10.0 * u[2 + 7 + 1]


def test_serving_memory_estimate_covers_second_order_triangles():
    """The admission estimate grows by the limited gradient (8 B per cell and
    ordinate) for second-order triangle problems, and is exact in its psi term."""
    from paper_2505_17284_gb300 import serve, rt
    n, M = 1000, 100                       # M_pad = 128
    base = serve.estimate_bytes(n, M, triangles=True)
    two = serve.estimate_bytes(n, M, triangles=True, order=2)
    assert two - base == n * (2 * 128 * 4 + 48)
    assert serve.estimate_bytes(n, M) - serve.estimate_bytes(n, M, storage=rt.RT_BF16) == n * 2 * 128 * 2

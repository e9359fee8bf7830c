"""The full-size GPU parity tests check sampled cells against the oracle run
on a patch around each cell. This checks that reduction on the CPU: a patch of
half-width 4K + 1 cells (MUSCL, Heun) or K + 2 squares (first order on
triangles, Euler) reproduces the whole-domain oracle at its centre after K
steps exactly, including cells at the domain boundary and at the inflow."""
import numpy as np

import oracle
import sn_inputs as si
from test_gpu_full_size import lattice_patch, triangle_patch


def test_lattice_patch_equals_whole_domain():
    n, K = 140, 4
    p = si.lattice_problem(n)
    q = oracle.product_quadrature(2, 8)
    dt = 0.5 * p.mesh.dx
    full, _, _ = oracle.run(oracle.CartesianOracle(p, q, order=2), np.zeros((n * n, 16)), dt, K, "heun")
    for ci, cj in [(60, 60), (59, 71), (75, 55), (0, 0), (139, 70), (70, 80)]:
        pp, c = lattice_patch(p, ci, cj, 4 * K + 1)
        ps, _, _ = oracle.run(oracle.CartesianOracle(pp, q, order=2), np.zeros((pp.mesh.n_cells, 16)), dt, K, "heun")
        assert np.array_equal(ps[c], full[cj * n + ci]), (ci, cj)
    assert np.abs(full).max() > 0


def test_triangle_patch_equals_whole_domain():
    n, K = 130, 6
    p = si.enclosure_problem(n, jitter=0.2, seed=0)
    q = oracle.product_quadrature(2, 8)
    op = oracle.TriangleOracle(p, q, order=1)
    _, dt = oracle.triangle_dt(op, p.t_end)
    full, _, _ = oracle.run(op, np.zeros((p.mesh.n_cells, 16)), dt, K, "euler")
    for ci, cj in [(0, 50), (1, 60), (3, 45), (0, 10), (60, 60)]:
        pp, (c0, c1) = triangle_patch(p, n, ci, cj, K + 2)
        ps, _, _ = oracle.run(oracle.TriangleOracle(pp, q, order=1), np.zeros((pp.mesh.n_cells, 16)), dt, K, "euler")
        t0 = 2 * (cj * n + ci)
        assert np.array_equal(ps[c0], full[t0]) and np.array_equal(ps[c1], full[t0 + 1]), (ci, cj)
    assert np.abs(full).max() > 0


def test_second_order_triangle_patch_equals_whole_domain():
    n, K = 130, 3
    p = si.enclosure_problem(n, jitter=0.2, seed=0)
    q = oracle.product_quadrature(2, 8)
    op = oracle.TriangleOracle(p, q, order=2)
    _, dt = oracle.triangle_dt(op, p.t_end)
    full, _, _ = oracle.run(op, np.zeros((p.mesh.n_cells, 16)), dt, K, "heun")
    for ci, cj in [(0, 50), (2, 60), (5, 45), (1, 85)]:
        pp, (c0, c1) = triangle_patch(p, n, ci, cj, 4 * K + 2)
        ps, _, _ = oracle.run(oracle.TriangleOracle(pp, q, order=2), np.zeros((pp.mesh.n_cells, 16)), dt, K, "heun")
        t0 = 2 * (cj * n + ci)
        assert np.array_equal(ps[c0], full[t0]) and np.array_equal(ps[c1], full[t0 + 1]), (ci, cj)
    assert np.abs(full).max() > 0

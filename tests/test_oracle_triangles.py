"""Pins for the triangle-mesh oracle (Sec. 4.2 on triangles, first order):
mesh-metric invariants, an exact discrete attenuation chain, steadiness of a
uniform state under matching inflow, exact conservation, exact infinite-medium
decay inside the domain of dependence, and the discrete mass balance."""
import math

import numpy as np
import pytest

import sn_inputs as si
from oracle import TriangleOracle, product_quadrature, run, triangle_dt
from oracle.triangles import triangle_metrics


def quad_custom(xis, etas):
    xis, etas = np.asarray(xis, float), np.asarray(etas, float)
    mu = np.sqrt(np.clip(1 - xis ** 2 - etas ** 2, 0, None))
    return xis, etas, mu, np.full(xis.size, 2 * math.pi / xis.size)


def uniform_tri_problem(n, L, sigma_a, sigma_s, Q=0.0, jitter=0.0, seed=0, kind=(0, 0, 0, 0),
                        inflow=(0, 0, 0, 0), ny=None, Ly=None):
    mesh = si.split_grid_mesh(n, L, jitter=jitter, seed=seed, ny=ny, Ly=Ly)
    nc = mesh.n_cells
    mats = si.Materials(sigma_a=np.array([sigma_a]), sigma_s=np.array([sigma_s]), Q=np.array([Q]),
                        cell_mat=np.zeros(nc, np.int32), cell_region=np.zeros(nc, np.int32),
                        region_names=("all",))
    return si.Problem(mesh=mesh, materials=mats, boundary=si.Boundary(kind=kind, inflow=inflow), t_end=1.0)


@pytest.mark.parametrize("jitter", [0.0, 0.2])
def test_metrics(jitter):
    n, L = 9, 1.3
    m = si.split_grid_mesh(n, L, jitter=jitter, seed=4)
    area, nl, nbr, side = triangle_metrics(m.vertices, m.triangles, m.box)
    assert np.all(area > 0)
    assert abs(area.sum() - L * L) < 1e-13
    # closed polygons: sum of outward n*l vanishes
    assert np.max(np.abs(nl.sum(axis=1))) < 1e-14
    # neighbour symmetry: the shared edge has opposite n*l on the two sides
    for t in range(area.size):
        for e in range(3):
            j = nbr[t, e]
            if j < 0:
                continue
            back = np.where(nbr[j] == t)[0]
            assert back.size == 1
            assert np.allclose(nl[j, back[0]], -nl[t, e], atol=1e-15)
    # boundary: 4n edges, n per side, total length 4L, normals point outward
    b = nbr < 0
    assert b.sum() == 4 * n
    for s, (nx_, ny_) in enumerate(((-1, 0), (1, 0), (0, -1), (0, 1))):
        sel = b & (side == s)
        assert sel.sum() == n
        v = nl[sel]
        assert np.allclose(v[:, 0] * nx_ + v[:, 1] * ny_, np.linalg.norm(v, axis=1))
        assert abs(np.linalg.norm(v, axis=1).sum() - L) < 1e-13


def test_exact_discrete_attenuation_chain():
    """Ordinates with eta = 0 on the unjittered split grid: the flow passes the
    triangles of a row as a chain upper_0, lower_0, upper_1, ..., each entered
    through one edge with (omega . n) l = -xi dx and of area dx^2/2, so the steady
    state multiplies by 1/(1 + sigma dx/(2 xi)) per triangle."""
    n, L, sigma = 12, 1.5, 2.3
    q = quad_custom([0.9, 0.4, -0.7], [0.0, 0.0, 0.0])
    p = uniform_tri_problem(n, L, sigma, 0.0, kind=(si.INFLOW, 0, 0, 0), inflow=(1.0, 0, 0, 0), ny=3, Ly=0.4)
    op = TriangleOracle(p, q)
    dx = L / n
    psi = np.zeros((p.mesh.n_cells, 3))
    for k in range(2):
        r = 1.0 / (1.0 + sigma * dx / (2 * q[0][k]))
        for c in range(p.mesh.n_cells):
            sq, upper = divmod(c, 2)
            i = sq % n
            m = 2 * i + (0 if upper else 1)      # position in the chain
            psi[c, k] = r ** (m + 1)
    assert np.max(np.abs(op.F(psi))) < 1e-12


@pytest.mark.parametrize("jitter", [0.0, 0.2])
def test_uniform_state_with_matching_inflow_is_steady(jitter):
    """sigma_a = 0 and psi = c everywhere with inflow c on every side: the fluxes of
    a constant close around each triangle and scattering is in balance, F = 0."""
    q = product_quadrature(2, 8)
    c = 0.7
    p = uniform_tri_problem(8, 1.0, 0.0, 1.3, jitter=jitter, seed=2, kind=(1, 1, 1, 1), inflow=(c, c, c, c))
    op = TriangleOracle(p, q)
    assert np.max(np.abs(op.F(np.full((p.mesh.n_cells, 16), c)))) < 1e-12


def test_conservation_compact_support():
    """sigma_a = 0 and a state supported far from the boundary: no particle reaches
    the boundary in k steps (one cell per step at most), so the mass is constant."""
    n = 24
    q = product_quadrature(2, 8)
    p = uniform_tri_problem(n, 1.0, 0.0, 0.8, jitter=0.2, seed=7)
    op = TriangleOracle(p, q)
    xc, yc = p.mesh.centroids()
    rng = np.random.default_rng(1)
    inside = (np.abs(xc - 0.5) < 0.15) & (np.abs(yc - 0.5) < 0.15)
    psi0 = np.where(inside[:, None], rng.uniform(0.5, 1.5, (p.mesh.n_cells, 16)), 0.0)
    m0 = op.integrands(psi0)["mass"]
    _, dt = triangle_dt(op, 1.0)
    psi, acc, S = run(op, psi0, dt, 6, "euler")
    assert abs(S["mass"] / m0 - 1) < 1e-13
    assert acc.outflow_int == 0.0


@pytest.mark.parametrize("integrator", ["euler", "heun"])
def test_interior_infinite_medium_decay(integrator):
    """Uniform isotropic psi^0 = 1 with vacuum sides: the boundary influence moves
    one cell layer per stage, so cells far inside follow the infinite-medium
    recurrence phi^{n+1} = g phi^n exactly."""
    n, k = 40, 4
    sa, ss = 0.8, 0.5
    q = product_quadrature(2, 8)
    p = uniform_tri_problem(n, 1.0, sa, ss, jitter=0.2, seed=3)
    op = TriangleOracle(p, q)
    _, dt = triangle_dt(op, 1.0)
    psi, _, _ = run(op, np.ones((p.mesh.n_cells, 16)), dt, k, integrator)
    xc, yc = p.mesh.centroids()
    dist = np.minimum.reduce([xc, 1 - xc, yc, 1 - yc])
    far = dist > (2 * k + 3) * (1.0 / n)
    assert far.sum() > 10
    g = 1 - sa * dt if integrator == "euler" else 1 - sa * dt + 0.5 * (sa * dt) ** 2
    phi = op.phi(psi)
    assert np.max(np.abs(phi[far] / (2 * math.pi * g ** k) - 1)) < 1e-13
    assert np.min(phi) < 0.99 * 2 * math.pi * g ** k   # the boundary did act


def test_enclosure_mass_balance():
    """mass(T) + absorbed + outflow = 0 with psi^0 = 0, Q = 0 and inflow on x = 0."""
    p = si.enclosure_problem(26, jitter=0.2, seed=0)
    q = product_quadrature(2, 8)
    op = TriangleOracle(p, q)
    _, dt = triangle_dt(op, 2.6)
    psi, acc, S = run(op, np.zeros((p.mesh.n_cells, 16)), dt, 30, "euler")
    lhs = S["mass"] + acc.abs_int.sum() + acc.outflow_int
    assert acc.outflow_int < 0
    assert abs(lhs) < 1e-12 * (S["mass"] + acc.abs_int.sum())


def test_triangle_dt_rule():
    p = si.enclosure_problem(10, jitter=0.0)
    op = TriangleOracle(p, product_quadrature(2, 4))
    dx = 0.13
    # right isosceles triangle with legs dx: 2A/P = dx^2 / (dx (2 + sqrt 2))
    assert abs(op.min_2A_over_P() - dx / (2 + math.sqrt(2))) < 1e-15
    n, dt = triangle_dt(op, 2.6)
    assert dt <= 0.9 * dx / (2 + math.sqrt(2)) and abs(n * dt - 2.6) < 1e-12


# ---------------------------------------------------------------- second order (Sec. 4.2)
from oracle.triangles import venkatakrishnan


def _phi_venkat(y):
    """The textbook Venkatakrishnan function (eps = 0) of y = beta / Delta."""
    return (y * y + 2 * y) / (y * y + y + 2)


def test_venkatakrishnan_special_values():
    """With eps = 0 the printed limiter is the textbook function of y = beta/Delta
    (beta_max for Delta > 0, beta_min for Delta < 0); Delta = 0 gives 1; a flat
    side (beta = 0) with eps > 0 gives eps^2 / (2 Delta^2 + eps^2)."""
    d = np.array([0.3, 0.3, -0.2, 1.0, 0.0, 2.0])
    bmax = np.array([0.3, 1.2, 5.0, 2.0, 0.0, 0.0])
    bmin = np.array([-9.0, -9.0, -0.6, -1.0, -1.0, -1.0])
    L = venkatakrishnan(d, bmax, bmin, 0.0)
    y = np.where(d > 0, bmax, bmin)[:5] / np.where(d == 0, 1, d)[:5]
    assert np.allclose(L[:4], _phi_venkat(y[:4]), rtol=1e-14)
    assert L[4] == 1.0                                   # Delta = 0
    assert abs(L[0] - 0.75) < 1e-15 and abs(L[1] - 12 / 11) < 1e-15   # y = 1 and y = 4
    eps = 0.5
    assert abs(venkatakrishnan(np.array([2.0]), np.array([0.0]), np.array([-1.0]), eps)[0]
               - eps ** 2 / (2 * 4.0 + eps ** 2)) < 1e-15
    assert abs(_phi_venkat(2.0) - 1.0) < 1e-15 and abs(_phi_venkat(4.0) - 12 / 11) < 1e-15


def test_green_gauss_gradient_and_limiter_on_a_linear_field():
    """psi = a + b.x on the unjittered split mesh: the two cells of every
    interior edge are point-symmetric about its midpoint, so the Green-Gauss
    gradient with face averages is exact; the neighbour differences are
    2 b.r_e, so y = beta/Delta per edge follows from the geometry alone and
    L = min_e phi(y_e) (Delta = (1/2) g.r as printed)."""
    n = 8
    p = uniform_tri_problem(n, 1.0, 0.0, 0.0)
    q = product_quadrature(1, 4)
    op = TriangleOracle(p, q, order=2)
    xc, yc = p.mesh.centroids()
    b = np.array([1.0, 0.3])
    psi = (2.0 + b[0] * xc + b[1] * yc)[:, None] * np.ones((1, 4))
    gx, gy = op.gradient(psi)
    interior = np.all(op.nbr >= 0, axis=1)
    assert interior.sum() > 50
    assert np.max(np.abs(gx[interior] - b[0])) < 1e-12 and np.max(np.abs(gy[interior] - b[1])) < 1e-12
    L = op.limiter(psi, gx, gy)[:, 0]
    for c in np.nonzero(interior)[0]:
        gr = op.r[c] @ b                        # b . r_e for the three edges
        bmax, bmin = max(0.0, 2 * gr.max()), min(0.0, 2 * gr.min())
        ys = [(bmax if v > 0 else bmin) / (0.5 * v) for v in gr if v != 0]
        expect = min(_phi_venkat(y) for y in ys)
        assert abs(L[c] - expect) < 1e-9, c
    assert L[interior].max() > 1.0               # the printed limiter exceeds 1 on smooth data


def _bump_problem(n, jitter=0.2):
    return uniform_tri_problem(n, 1.0, 0.0, 0.0, jitter=jitter, seed=5)


def _bump_error(order, n):
    """L1 error of pure advection of a Gaussian bump over t = 0.2 (Heun)."""
    q = quad_custom([0.6, -0.5], [0.3, 0.45])
    p = _bump_problem(n)
    op = TriangleOracle(p, q, order=order)
    xc, yc = p.mesh.centroids()
    bump = lambda x, y: np.exp(-((x - 0.4) ** 2 + (y - 0.4) ** 2) / (2 * 0.08 ** 2))
    T = 0.2
    N = int(math.ceil(T / (0.5 * op.min_2A_over_P())))
    psi, _, _ = run(op, np.stack([bump(xc, yc)] * 2, 1), T / N, N, "heun")
    ex = np.stack([bump(xc - q[0][k] * T, yc - q[1][k] * T) for k in range(2)], 1)
    return float(np.sum(op.area[:, None] * np.abs(psi - ex)))


def test_second_order_converges_faster_than_first():
    """On jittered meshes the limited second-order scheme converges at well
    above first order on a smooth bump (ratio > 2.3 per halving of h, against
    < 2 for first order) and is several times more accurate."""
    e1 = [_bump_error(1, n) for n in (16, 32)]
    e2 = [_bump_error(2, n) for n in (16, 32)]
    assert e1[0] / e1[1] < 2.0
    assert e2[0] / e2[1] > 2.3
    assert e2[1] < 0.25 * e1[1]


def test_second_order_conservation_and_uniform_state():
    """Fluxes telescope with the reconstructed traces (mass constant for a
    compactly supported state), and a uniform state with matching inflow
    stays steady (zero gradient, L = 1)."""
    n = 24
    q = product_quadrature(2, 8)
    p = uniform_tri_problem(n, 1.0, 0.0, 0.8, jitter=0.2, seed=7)
    op = TriangleOracle(p, q, order=2)
    xc, yc = p.mesh.centroids()
    rng = np.random.default_rng(1)
    inside = (np.abs(xc - 0.5) < 0.15) & (np.abs(yc - 0.5) < 0.15)
    psi0 = np.where(inside[:, None], rng.uniform(0.5, 1.5, (p.mesh.n_cells, 16)), 0.0)
    m0 = op.integrands(psi0)["mass"]
    _, dt = triangle_dt(op, 1.0)
    psi, acc, S = run(op, psi0, dt, 4, "heun")
    assert abs(S["mass"] / m0 - 1) < 1e-13
    # (leaving ordinates see the ghost value 0 in a boundary cell's gradient;
    # the limiter then keeps only eps^2/(2 Delta^2) ~ 1e-12 of that slope)
    c = 0.7
    pu = uniform_tri_problem(8, 1.0, 0.0, 1.3, jitter=0.2, seed=2, kind=(1, 1, 1, 1), inflow=(c, c, c, c))
    opu = TriangleOracle(pu, q, order=2)
    Fu = opu.F(np.full((pu.mesh.n_cells, 16), c))
    assert np.max(np.abs(Fu)) < 1e-8

"""Pins for the Cartesian oracle (Sec. 4.2-4.3) against closed forms,
invariants and the paper's printed lattice QoIs.

Each test names the property it checks; together they fail on a dropped term,
a wrong sign, a wrong index or a transposed operand anywhere in F, the traces,
the limiter, the boundary ghosts, the time integrators or the QoIs.
"""
import json
import math
import os

import numpy as np
import pytest

import sn_inputs as si
from oracle import CartesianOracle, product_quadrature, run, n_steps_for
from oracle.cartesian import minmod

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def quad_custom(xis, etas, weights=None):
    xis = np.asarray(xis, float)
    etas = np.asarray(etas, float)
    mu = np.sqrt(np.clip(1.0 - xis ** 2 - etas ** 2, 0.0, None))
    if weights is None:
        weights = np.full(xis.size, 2 * math.pi / xis.size)
    return xis, etas, mu, np.asarray(weights, float)


def uniform_problem(nx, ny, L, sigma_a, sigma_s, Q=0.0, kind=(0, 0, 0, 0), inflow=(0, 0, 0, 0), Ly=None):
    Ly = L if Ly is None else Ly
    mesh = si.CartesianMesh(nx=nx, ny=ny, x0=0.0, y0=0.0, dx=L / nx, dy=Ly / ny)
    n = nx * ny
    mats = si.Materials(sigma_a=np.array([sigma_a]), sigma_s=np.array([sigma_s]), Q=np.array([Q]),
                        cell_mat=np.zeros(n, np.int32), cell_region=np.zeros(n, np.int32),
                        region_names=("all",))
    return si.Problem(mesh=mesh, materials=mats, boundary=si.Boundary(kind=kind, inflow=inflow), t_end=1.0)


def test_minmod_definition():
    a = np.array([1.0, -1.0, 2.0, -3.0, 0.0, 1.0, -2.0])
    b = np.array([2.0, -0.5, -1.0, 1.0, 5.0, 0.0, -2.0])
    assert np.array_equal(minmod(a, b), [1.0, -0.5, 0.0, 0.0, 0.0, 0.0, -2.0])


# ---------------------------------------------------------------- P2
@pytest.mark.parametrize("ny,periodic_y", [(1, False), (3, False), (2, True)])
def test_exact_discrete_attenuation_first_order(ny, periodic_y):
    """Steady first-order upwind slab: xi (psi_i - psi_{i-1})/dx + sigma psi_i = 0 with
    psi_{-1} = 1 gives psi_i = (xi/(xi + sigma dx))^(i+1) exactly, for every
    ordinate entering through x = 0; ordinates with xi < 0 see vacuum and stay 0."""
    nx, L, sigma = 25, 2.0, 1.7
    if periodic_y:
        q = quad_custom([1.0, 0.6, 0.3, -0.5], [0.0, 0.5, -0.8, 0.3])
        kind = (si.INFLOW, si.VACUUM, si.PERIODIC, si.PERIODIC)
    else:
        q = quad_custom([1.0, 0.6, 0.3, -0.5], [0.0, 0.0, 0.0, 0.0])
        kind = (si.INFLOW, si.VACUUM, si.VACUUM, si.VACUUM)
    p = uniform_problem(nx, ny, L, sigma, 0.0, kind=kind, inflow=(1.0, 0, 0, 0), Ly=0.3 * ny)
    op = CartesianOracle(p, q, order=1)
    dx = L / nx
    i = np.arange(nx)
    prof = np.zeros((nx, 4))
    for k in range(4):
        if q[0][k] > 0:
            prof[:, k] = (q[0][k] / (q[0][k] + sigma * dx)) ** (i + 1)
    psi = np.tile(prof[None, :, :], (ny, 1, 1)).reshape(nx * ny, 4)
    F = op.F(psi)
    assert np.max(np.abs(F)) < 1e-13
    # marching reaches the same state
    dt = 0.4 * dx
    psi_t, _, _ = run(op, np.zeros_like(psi), dt, int(12.0 / dt), "euler")
    assert np.max(np.abs(psi_t - psi)) < 1e-12


def _attenuation_error(nx, order, integrator, sigma=1.0, xi=0.8):
    L = 1.0
    q = quad_custom([xi], [0.0])
    p = uniform_problem(nx, 1, L, sigma, 0.0, kind=(si.INFLOW, 0, 0, 0), inflow=(1.0, 0, 0, 0), Ly=0.1)
    op = CartesianOracle(p, q, order=order)
    dx = L / nx
    dt = 0.3 * dx / xi
    psi, _, _ = run(op, np.zeros((nx, 1)), dt, int(6.0 / dt), integrator)
    xl = np.arange(nx) * dx
    exact = (xi / sigma) * (np.exp(-sigma * xl / xi) - np.exp(-sigma * (xl + dx) / xi)) / dx
    return np.sum(np.abs(psi[:, 0] - exact)) * dx


@pytest.mark.parametrize("order,integrator,lo,hi", [(1, "euler", 0.9, 1.15), (2, "heun", 1.8, 2.3)])
def test_attenuation_convergence_order(order, integrator, lo, hi):
    """Steady attenuation under constant inflow converges to the cell averages of
    exp(-sigma x / xi): first order for upwind, second order for MUSCL-minmod."""
    e = [_attenuation_error(n, order, integrator) for n in (20, 40, 80)]
    rates = [math.log2(e[0] / e[1]), math.log2(e[1] / e[2])]
    assert lo < rates[-1] < hi, (e, rates)


# ---------------------------------------------------------------- linear exactness
@pytest.mark.parametrize("order", [1, 2])
def test_linear_field_divergence_exact(order):
    """For psi_k = a_k + b_k x + c_k y both upwind and MUSCL (equal one-sided
    slopes, so minmod returns them) give flux divergence xi b + eta c in cells
    two layers away from the boundary."""
    nx, ny = 12, 9
    q = product_quadrature(2, 8)
    p = uniform_problem(nx, ny, 1.2, 0.0, 0.0, Ly=0.9)
    op = CartesianOracle(p, q, order=order)
    xc, yc = p.mesh.centres()
    rng = np.random.default_rng(3)
    a, b, c = rng.uniform(1, 2, 16), rng.uniform(-1, 1, 16), rng.uniform(-1, 1, 16)
    psi = a[None, :] + b[None, :] * xc[:, None] + c[None, :] * yc[:, None]
    div = op.flux_sum(psi) / op.area
    expect = np.broadcast_to(q[0] * b + q[1] * c, div.shape)
    inner = ((xc > 2 * p.mesh.dx + 1e-9) & (xc < 1.2 - 2 * p.mesh.dx) &
             (yc > 2 * p.mesh.dy + 1e-9) & (yc < 0.9 - 2 * p.mesh.dy))
    assert np.max(np.abs(div[inner] - expect[inner])) < 1e-11


# ---------------------------------------------------------------- P3 / P4 / P5 / P6
@pytest.mark.parametrize("order,integrator", [(1, "euler"), (2, "heun"), (2, "euler"), (1, "heun")])
def test_conservation_periodic(order, integrator):
    """sigma_a = 0 on a periodic box: the mass sum_i A_i phi_i is constant."""
    q = product_quadrature(2, 8)
    p = uniform_problem(16, 12, 1.0, 0.0, 0.7, kind=(2, 2, 2, 2), Ly=0.75)
    op = CartesianOracle(p, q, order=order)
    psi0 = si.random_psi(p.mesh.n_cells, 16, seed=11)
    m0 = op.integrands(psi0)["mass"]
    dt = 0.25 * p.mesh.dx
    psi, acc, S = run(op, psi0, dt, 200, integrator)
    assert abs(S["mass"] / m0 - 1.0) < 1e-13
    assert acc.outflow_int == 0.0


@pytest.mark.parametrize("integrator", ["euler", "heun"])
def test_infinite_medium_decay(integrator):
    """Uniform isotropic psi on a periodic box: phi^n = phi^0 g^n + source part, with
    g = 1 - s dt (Euler) or 1 - s dt + (s dt)^2/2 (Heun), s = sigma_a."""
    sa, ss, Q = 0.9, 0.6, 0.25
    q = product_quadrature(4, 8)
    p = uniform_problem(6, 5, 1.0, sa, ss, Q=Q, kind=(2, 2, 2, 2))
    op = CartesianOracle(p, q, order=2)
    psi0 = np.full((30, 32), 0.8)
    dt, n = 0.05, 40
    psi, acc, S = run(op, psi0, dt, n, integrator)
    phi = op.phi(psi)
    phi0, src = 0.8 * 2 * math.pi, 2 * math.pi * Q
    # phi' = -sa phi + src: exact discrete recurrence of each scheme
    ph = phi0
    for _ in range(n):
        if integrator == "euler":
            ph = ph + dt * (-sa * ph + src)
        else:
            p1 = ph + dt * (-sa * ph + src)
            ph = 0.5 * (ph + p1 + dt * (-sa * p1 + src))
    assert np.max(np.abs(phi / ph - 1.0)) < 1e-13
    g = 1 - sa * dt if integrator == "euler" else 1 - sa * dt + 0.5 * (sa * dt) ** 2
    ph_closed = (phi0 - src / sa) * g ** n + src / sa
    assert abs(ph / ph_closed - 1.0) < 1e-12
    # continuum limit exp(-sa t) is approached
    assert abs(ph_closed - ((phi0 - src / sa) * math.exp(-sa * n * dt) + src / sa)) < 0.02 * phi0


def test_scattering_relaxation_euler():
    """sigma_a = 0, uniform anisotropic psi: phi is constant and the anisotropic
    part psi_k - phi/(2 pi) decays by exactly (1 - sigma_s dt) per Euler step."""
    ss, dt, n = 1.5, 0.1, 25
    q = product_quadrature(2, 8)
    p = uniform_problem(4, 4, 1.0, 0.0, ss, kind=(2, 2, 2, 2))
    op = CartesianOracle(p, q, order=1)
    prof = si.random_psi(1, 16, seed=5)[0]
    psi0 = np.tile(prof, (16, 1))
    psi, _, _ = run(op, psi0, dt, n, "euler")
    phi0 = prof @ q[3]
    assert np.allclose(op.phi(psi), phi0, rtol=1e-13)
    expect = phi0 / (2 * math.pi) + (prof - phi0 / (2 * math.pi)) * (1 - ss * dt) ** n
    assert np.max(np.abs(psi - expect[None, :])) < 1e-13


@pytest.mark.parametrize("xi,eta", [(1.0, 0.0), (-1.0, 0.0), (0.0, 1.0), (0.0, -1.0)])
def test_exact_shift(xi, eta):
    """One ordinate along an axis, sigma = 0, first-order Euler with dt = dx: the
    state moves by exactly one cell per step (up to a few ulp of rounding in
    psi_i - (psi_i - psi_{i-1}))."""
    n = 10
    q = quad_custom([xi], [eta], [2 * math.pi])
    p = uniform_problem(n, n, 1.0, 0.0, 0.0, kind=(2, 2, 2, 2))
    op = CartesianOracle(p, q, order=1)
    psi = si.random_psi(n * n, 1, seed=9) + 0.5
    cur = psi.reshape(n, n)
    for _ in range(7):
        psi, _, _ = run(op, psi, 0.1, 1, "euler")
        cur = np.roll(cur, (int(eta), int(xi)), axis=(0, 1))
        assert np.max(np.abs(psi.reshape(n, n) - cur) / cur) < 8 * np.finfo(float).eps


# ---------------------------------------------------------------- limiter: max principle
@pytest.mark.parametrize("integrator", ["euler", "heun"])
def test_muscl_minmod_max_principle(integrator):
    """Pure advection of step data on a periodic box with (|xi|/dx + |eta|/dy) dt <= 0.6:
    MUSCL-minmod keeps every ordinate inside [min, max] of its initial data
    (each stage is a convex combination). An unlimited central slope overshoots."""
    n = 16
    q = product_quadrature(2, 8)
    p = uniform_problem(n, n, 1.0, 0.0, 0.0, kind=(2, 2, 2, 2))
    op = CartesianOracle(p, q, order=2)
    xc, yc = p.mesh.centres()
    psi0 = np.where((np.abs(xc - 0.5) < 0.2) & (np.abs(yc - 0.5) < 0.25), 2.0, 0.5)[:, None] * np.ones(16)[None, :]
    dt = 0.6 / (np.max(np.abs(q[0]) + np.abs(q[1])) * n)
    psi, _, _ = run(op, psi0, dt, 40, integrator)
    assert psi.min() >= 0.5 - 1e-13 and psi.max() <= 2.0 + 1e-13
    assert psi.min() < 1.999 and np.ptp(psi) > 0.5   # it did move


# ---------------------------------------------------------------- P7 / P8 / golden
@pytest.mark.parametrize("order,integrator", [(1, "euler"), (2, "heun")])
def test_lattice_mass_balance(order, integrator):
    """mass(T) + absorbed + outflow = mass(0) + emitted: an exact identity of the
    scheme (interior fluxes telescope, weights sum to 2 pi)."""
    p = si.lattice_problem(35)
    q = product_quadrature(2, 8)
    op = CartesianOracle(p, q, order=order)
    dt = 0.5 * p.mesh.dx
    psi, acc, S = run(op, np.zeros((p.mesh.n_cells, 16)), dt, 30, integrator)
    lhs = S["mass"] + acc.abs_int.sum() + acc.outflow_int
    rhs = op.source_rate() * 30 * dt
    assert abs(lhs / rhs - 1.0) < 1e-12
    assert acc.outflow_int > 0


def test_enclosure_cartesian_mass_balance_with_inflow():
    p = si.enclosure_cartesian_problem(26)
    q = product_quadrature(2, 8)
    op = CartesianOracle(p, q, order=2)
    dt = 0.5 * p.mesh.dx
    psi, acc, S = run(op, np.zeros((p.mesh.n_cells, 16)), dt, 40, "heun")
    lhs = S["mass"] + acc.abs_int.sum() + acc.outflow_int
    scale = S["mass"] + acc.abs_int.sum()
    assert acc.outflow_int < 0           # net inflow through x = 0
    assert abs(lhs) < 1e-12 * scale


@pytest.mark.parametrize("order,integrator", [(1, "euler"), (2, "heun")])
def test_lattice_mirror_symmetry(order, integrator):
    """B, R and W are symmetric about x = 3.5 and the quadrature is closed under
    varphi -> pi - varphi, so phi(x, y) = phi(7 - x, y)."""
    n = 28
    p = si.lattice_problem(n)
    q = product_quadrature(4, 8)
    op = CartesianOracle(p, q, order=order)
    psi, _, _ = run(op, np.zeros((n * n, 32)), 0.5 * p.mesh.dx, 20, integrator)
    phi = op.phi(psi).reshape(n, n)
    assert np.max(np.abs(phi - phi[:, ::-1])) < 1e-12 * phi.max()
    # and not symmetric in y (block C_{4,6} of the paper is white)
    assert np.max(np.abs(phi - phi[::-1, :])) > 1e-6 * phi.max()


def test_lattice_qoi_against_paper_table():
    """At 70^2 with 4x16 ordinates (first-order Euler, dt = dx/2, T = 3.2) the
    oracle lands within 2 % of the paper's reference QoI-3/4/5 (a different,
    much finer discretisation), and QoI-4 + QoI-5 of the paper's table equal
    2 pi T up to its outflow, as the scheme's mass balance requires."""
    g = json.load(open(os.path.join(GOLDEN, "lattice_qoi_table.json")))
    T = g["T"]
    assert abs(g["qoi4_absorption_time_integrated"]["mean"] + g["qoi5_mass_at_T"]["mean"]
               - 2 * math.pi * T) < 0.01
    p = si.lattice_problem(70)
    q = product_quadrature(4, 16)
    op = CartesianOracle(p, q, order=1)
    n = n_steps_for(T, 0.5 * p.mesh.dx)
    assert n == 64
    psi, acc, S = run(op, np.zeros((4900, 64)), T / n, n, "euler")
    blue = si.LATTICE_REGIONS.index("blue")
    assert abs(S["abs"][blue] / g["qoi3_absorption_at_T"]["mean"] - 1) < 0.02
    assert abs(acc.abs_int[blue] / g["qoi4_absorption_time_integrated"]["mean"] - 1) < 0.02
    assert abs(S["mass"] / g["qoi5_mass_at_T"]["mean"] - 1) < 0.02


# ---------------------------------------------------------------- QoI boxes (Sec. 3.1 QoI-1/2)
def _box_cells(p, box):
    xc, yc = p.mesh.centres()
    return (xc > box[0]) & (xc < box[1]) & (yc > box[2]) & (yc < box[3])


@pytest.mark.parametrize("order", [1, 2])
def test_box_flow_closes_the_box_balance(order):
    """Finite-volume conservation on the union of the cells inside a box: over
    one Euler step, the change of the box's particle content equals dt times
    (emission - absorption - outflow + inflow) through its boundary, with the
    flows of box_flow. Any wrong face, side, sign, normal, length or trace in
    box_flow breaks the identity."""
    p = si.lattice_problem(28)
    p.extra = {"boxes": ((2.0, 5.0, 2.0, 5.0), (1.0, 6.0, 1.0, 6.0), (0.25, 3.0, 4.5, 6.75))}
    q = product_quadrature(4, 8)
    op = CartesianOracle(p, q, order=order)
    psi0 = si.random_psi(p.mesh.n_cells, 32, seed=3)
    dt = 0.4 * p.mesh.dx
    psi1 = psi0 + dt * op.F(psi0)
    out, inn = op.box_flow(psi0)
    assert np.all(out > 0) and np.all(inn > 0)
    A = p.mesh.dx * p.mesh.dy
    phi0, phi1 = psi0 @ q[3], psi1 @ q[3]
    for b, box in enumerate(p.extra["boxes"]):
        m = _box_cells(p, box)
        change = A * (phi1[m].sum() - phi0[m].sum())
        emitted = A * 2 * math.pi * op.Q[m].sum()
        absorbed = A * (op.sigma_a[m] * phi0[m]).sum()
        rhs = dt * (emitted - absorbed - out[b] + inn[b])
        assert abs(change - rhs) <= 1e-12 * (abs(change) + dt * (out[b] + inn[b])), b


def test_box_flow_of_the_whole_domain_is_the_boundary_outflow():
    """With vacuum sides nothing enters the domain, so the flow out of a box
    equal to the whole domain is the domain's boundary outflow."""
    p = si.lattice_problem(21)
    p.extra = {"boxes": ((0.0, 7.0, 0.0, 7.0),)}
    op = CartesianOracle(p, product_quadrature(2, 8), order=2)
    psi = si.random_psi(p.mesh.n_cells, 16, seed=4)
    out, inn = op.box_flow(psi)
    assert abs(out[0] - op.outflow(psi)) <= 1e-13 * out[0]
    assert inn[0] == 0.0


def test_box_flow_uniform_state_closed_form():
    """A uniform state psi = c in every cell and ordinate (first order): the
    flow out of a W x H box is c (H sum_k w_k |xi_k| + W sum_k w_k |eta_k|),
    and sum_k w_k |xi_k| tends to the hemisphere integral of |xi|, pi."""
    p = uniform_problem(20, 20, 2.0, 0.0, 0.0)
    p.extra = {"boxes": ((0.4, 1.5, 0.2, 1.0),)}
    q = product_quadrature(16, 64)
    op = CartesianOracle(p, q, order=1)
    c = 0.75
    out, inn = op.box_flow(np.full((400, q[0].size), c))
    W, H = 1.1, 0.8
    assert abs(out[0] - inn[0]) <= 1e-13 * out[0]
    assert abs(out[0] / (c * math.pi * (W + H)) - 1) < 2e-3
    assert si.lattice_problem(70).extra["boxes"] == si.LATTICE_QOI_SQUARES
    assert si.lattice_problem(64).extra == {}

"""The pins catch plausible mistakes: each test plants one mistake in a copy of
the oracle (on the CPU) and checks that the matching closed form no longer holds."""
import math

import numpy as np
import pytest

import sn_inputs as si
from oracle import CartesianOracle, product_quadrature, run
from oracle import cartesian as cart
from test_oracle_cartesian import uniform_problem, quad_custom


def _decay_error(op, dt=0.05, n=20, sa=0.9, Q=0.25):
    psi, _, _ = run(op, np.full((op.nx * op.ny, op.M), 0.8), dt, n, "euler")
    ph = 0.8 * 2 * math.pi
    for _ in range(n):
        ph = ph + dt * (-sa * ph + 2 * math.pi * Q)
    return np.max(np.abs(op.phi(psi) / ph - 1))


def test_dropped_scattering_term_is_caught():
    q = product_quadrature(2, 8)
    p = uniform_problem(4, 4, 1.0, 0.9, 0.6, Q=0.25, kind=(2, 2, 2, 2))
    good = CartesianOracle(p, q, order=1)
    assert _decay_error(good) < 1e-13

    class NoScatter(CartesianOracle):
        def F(self, psi):
            return -self.flux_sum(psi) / self.area - self.sigma_t[:, None] * psi + self.Q[:, None]
    assert _decay_error(NoScatter(p, q, order=1)) > 1e-3


def test_downwind_trace_is_caught():
    nx, sigma = 20, 1.5
    q = quad_custom([0.8], [0.0])
    p = uniform_problem(nx, 1, 1.0, sigma, 0.0, kind=(si.INFLOW, 0, 0, 0), inflow=(1.0, 0, 0, 0), Ly=0.1)
    dx = 1.0 / nx
    prof = ((0.8 / (0.8 + sigma * dx)) ** (np.arange(nx) + 1))[:, None]

    class Downwind(CartesianOracle):
        def _face_traces(self, P, vel, g_lo, g_hi, periodic):
            return super()._face_traces(P, -vel, g_lo, g_hi, periodic)
    assert np.max(np.abs(CartesianOracle(p, q).F(prof))) < 1e-13
    assert np.max(np.abs(Downwind(p, q).F(prof))) > 1e-2


def test_unlimited_slope_is_caught(monkeypatch):
    n = 16
    q = product_quadrature(2, 8)
    p = uniform_problem(n, n, 1.0, 0.0, 0.0, kind=(2, 2, 2, 2))
    xc, yc = p.mesh.centres()
    psi0 = np.where((np.abs(xc - 0.5) < 0.2) & (np.abs(yc - 0.5) < 0.25), 2.0, 0.5)[:, None] * np.ones(16)[None, :]
    dt = 0.6 / (np.max(np.abs(q[0]) + np.abs(q[1])) * n)
    monkeypatch.setattr(cart, "minmod", lambda a, b: 0.5 * (a + b))
    psi, _, _ = run(CartesianOracle(p, q, order=2), psi0, dt, 40, "heun")
    assert psi.max() > 2.0 + 1e-3 or psi.min() < 0.5 - 1e-3


def test_wrong_heun_average_is_caught():
    q = product_quadrature(2, 8)
    p = uniform_problem(4, 4, 1.0, 0.9, 0.6, Q=0.0, kind=(2, 2, 2, 2))
    op = CartesianOracle(p, q, order=1)
    psi = np.full((16, 16), 1.0)
    dt, sa = 0.1, 0.9
    # Heun as printed: (psi + psi2)/2; a variant that returns psi2 is first order and fails the recurrence
    psi1 = psi + dt * op.F(psi)
    psi2 = psi1 + dt * op.F(psi1)
    g_heun = 1 - sa * dt + 0.5 * (sa * dt) ** 2
    assert np.allclose(op.phi(0.5 * (psi + psi2)), 2 * math.pi * g_heun, rtol=1e-14)
    assert not np.allclose(op.phi(psi2), 2 * math.pi * g_heun, rtol=1e-6)


def test_box_flow_from_the_outside_cell_is_caught():
    """Taking the trace of a leaving ordinate from the cell outside the box
    (instead of the upwind inside cell) breaks the box balance."""
    p = si.lattice_problem(14)
    p.extra = {"boxes": ((2.0, 5.0, 1.0, 6.0),)}
    q = product_quadrature(2, 8)
    psi0 = si.random_psi(p.mesh.n_cells, 16, seed=9)
    dt = 0.4 * p.mesh.dx
    A = p.mesh.dx * p.mesh.dy
    xc, yc = p.mesh.centres()
    m = (xc > 2) & (xc < 5) & (yc > 1) & (yc < 6)

    class OutsideTrace(CartesianOracle):
        def traces(self, psi):
            Tx, Ty = super().traces(psi)
            P = psi.reshape(self.ny, self.nx, self.M)
            Tx = Tx.copy()
            Tx[:, 10, :] = np.where(self.xi > 0, P[:, 10, :], Tx[:, 10, :])   # x+ side (face 10 at x = 5)
            return Tx, Ty

        def F(self, psi):
            return CartesianOracle.F(self, psi)

    def residual(op):
        good = CartesianOracle(p, q, order=1)
        psi1 = psi0 + dt * good.F(psi0)
        out, inn = op.box_flow(psi0)
        phi0, phi1 = psi0 @ q[3], psi1 @ q[3]
        change = A * (phi1[m].sum() - phi0[m].sum())
        rhs = dt * (A * 2 * math.pi * good.Q[m].sum() - A * (good.sigma_a[m] * phi0[m]).sum() - out[0] + inn[0])
        return abs(change - rhs) / abs(change)

    assert residual(CartesianOracle(p, q, order=1)) < 1e-12
    assert residual(OutsideTrace(p, q, order=1)) > 1e-3


def test_limiter_without_the_half_is_caught():
    """Delta = g.r instead of the printed (1/2) g.r changes the limiter on a
    linear field away from the textbook values the pin derives."""
    from oracle import TriangleOracle
    from oracle.triangles import venkatakrishnan
    from test_oracle_triangles import uniform_tri_problem, _phi_venkat

    class NoHalf(TriangleOracle):
        def limiter(self, psi, gx, gy):
            nb = [self.neighbour_values(psi, e) for e in range(3)]
            pmax = np.maximum(psi, np.maximum(np.maximum(nb[0], nb[1]), nb[2]))
            pmin = np.minimum(psi, np.minimum(np.minimum(nb[0], nb[1]), nb[2]))
            L = None
            for e in range(3):
                delta = gx * self.r[:, e, 0:1] + gy * self.r[:, e, 1:2]
                Le = venkatakrishnan(delta, pmax - psi, pmin - psi, self.eps[:, None])
                L = Le if L is None else np.minimum(L, Le)
            return L

    p = uniform_tri_problem(8, 1.0, 0.0, 0.0)
    q = product_quadrature(1, 4)
    xc, yc = p.mesh.centroids()
    psi = (2.0 + xc + 0.3 * yc)[:, None] * np.ones((1, 4))

    def worst(op):
        gx, gy = op.gradient(psi)
        L = op.limiter(psi, gx, gy)[:, 0]
        err = 0.0
        for c in np.nonzero(np.all(op.nbr >= 0, axis=1))[0]:
            gr = op.r[c] @ np.array([1.0, 0.3])
            bmax, bmin = max(0.0, 2 * gr.max()), min(0.0, 2 * gr.min())
            expect = min(_phi_venkat((bmax if v > 0 else bmin) / (0.5 * v)) for v in gr if v != 0)
            err = max(err, abs(L[c] - expect))
        return err

    assert worst(TriangleOracle(p, q, order=2)) < 1e-9
    assert worst(NoHalf(p, q, order=2)) > 1e-2

"""Pins for the oracle's product quadrature (Sec. 4.1, Eq. sn_2d and Eq.
polar_coordinates): weights sum to 2 pi and the rule integrates low-degree
polynomials of (xi, eta, mu) over the upper hemisphere exactly. The closed
forms are integrals over [0,1] x [0, 2 pi) in (mu, varphi) computed by hand.
The tessellation rule (Sec. 5.1.1) is pinned by its order-1 closed form, the
tiling of the hemisphere, weights from direct area integration, symmetry and
moment convergence."""
import math

import numpy as np
import pytest

import oracle
from oracle import product_quadrature, gauss_legendre_01

pytestmark = pytest.mark.filterwarnings("ignore")

SHAPES = [(4, 16), (8, 16), (8, 32), (16, 32), (2, 8)]


@pytest.mark.parametrize("n_p,n_phi", SHAPES)
def test_moments(n_p, n_phi):
    xi, eta, mu, w = product_quadrature(n_p, n_phi)
    assert xi.size == n_p * n_phi
    two_pi = 2 * math.pi
    assert abs(w.sum() - two_pi) < 1e-13
    assert abs(np.sum(w * mu) - math.pi) < 1e-13
    # int (1-mu^2) cos^2 = (2/3) * pi
    assert abs(np.sum(w * xi ** 2) - two_pi / 3) < 1e-13
    assert abs(np.sum(w * eta ** 2) - two_pi / 3) < 1e-13
    if n_p >= 3 and n_phi >= 8:
        # int (1-mu^2)^2 cos^2 sin^2 = (8/15)(pi/4);  int (1-mu^2)^2 cos^4 = (8/15)(3 pi/4)
        assert abs(np.sum(w * xi ** 2 * eta ** 2) - two_pi / 15) < 1e-13
        assert abs(np.sum(w * xi ** 4) - two_pi / 5) < 1e-13
    for odd in (xi, eta, xi * eta, xi ** 3, xi * eta ** 2):
        assert abs(np.sum(w * odd)) < 1e-13
    # unit directions on the upper hemisphere
    assert np.allclose(xi ** 2 + eta ** 2 + mu ** 2, 1.0, atol=1e-14)
    assert np.all(mu > 0) and np.all(mu < 1)
    # midpoint azimuths: no ordinate grazes an axis-aligned face
    assert np.all(np.abs(xi) > 1e-8) and np.all(np.abs(eta) > 1e-8)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16])
def test_gauss_legendre_exact_degree(n):
    x, w = gauss_legendre_01(n)
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14
    # and not exact one degree higher (guards against a wrong rule that happens to be better)
    if n <= 4:
        k = 2 * n
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) > 1e-8


def test_ordinate_ordering_and_mirror_closure():
    # k = a * n_p + p: polar index fastest; the set is closed under varphi -> pi - varphi
    n_p, n_phi = 4, 16
    xi, eta, mu, w = product_quadrature(n_p, n_phi)
    mu_p, _ = gauss_legendre_01(n_p)
    for a in range(n_phi):
        assert np.allclose(mu[a * n_p:(a + 1) * n_p], mu_p)
        b = n_phi // 2 - 1 - a
        b %= n_phi
        assert np.allclose(xi[b * n_p:(b + 1) * n_p], -xi[a * n_p:(a + 1) * n_p], atol=1e-15)
        assert np.allclose(eta[b * n_p:(b + 1) * n_p], eta[a * n_p:(a + 1) * n_p], atol=1e-15)


# ------------------------------------------------------------------ tessellation rule (Sec. 5.1.1)
def test_tessellation_order_one_is_the_octant_centroids():
    """N = 1: one point per face, the face centre (+-1, +-1, 1)/sqrt(3), with
    weight the octant's area pi/2."""
    xi, eta, mu, w = oracle.tessellation_quadrature(1)
    s = 1.0 / np.sqrt(3.0)
    assert np.allclose(np.abs(xi), s) and np.allclose(np.abs(eta), s) and np.allclose(mu, s)
    assert np.allclose(w, np.pi / 2)
    # quadrants in azimuth order
    assert list(np.sign(xi)) == [1, -1, -1, 1] and list(np.sign(eta)) == [1, 1, -1, -1]


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 12])
def test_tessellation_size_tiling_and_quadrant_blocks(N):
    xi, eta, mu, w = oracle.tessellation_quadrature(N)
    assert len(w) == 4 * N * N
    assert abs(w.sum() - 2 * np.pi) < 1e-12          # the spherical triangles tile the hemisphere
    assert np.all(w > 0) and np.all(mu > 0)
    assert np.allclose(xi ** 2 + eta ** 2 + mu ** 2, 1.0)
    sx, sy = np.sign(xi).reshape(4, N * N), np.sign(eta).reshape(4, N * N)
    for q, (a, b) in enumerate([(1, 1), (-1, 1), (-1, -1), (1, -1)]):
        assert np.all(sx[q] == a) and np.all(sy[q] == b)


def _projected_area(p, q, r, levels=6):
    """Area on the unit sphere of the central projection of the flat triangle
    (p, q, r): the integral over the flat triangle of (n . x) / |x|^3 (n the
    unit normal of its plane), by the midpoint rule on 4^levels sub-triangles."""
    n = np.cross(q - p, r - p)
    area2 = np.linalg.norm(n)
    n = n / area2
    tris = [(p, q, r)]
    for _ in range(levels):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        tris = nxt
    cent = np.array([(a + b + c) / 3 for a, b, c in tris])
    f = np.abs(cent @ n) / np.linalg.norm(cent, axis=1) ** 3
    return f.sum() * (area2 / 2) / len(tris)


@pytest.mark.parametrize("N", [2, 3])
def test_tessellation_weights_are_projected_areas(N):
    """Each weight equals the area of the projected small triangle computed by
    direct integration (independent of the spherical-excess formula)."""
    _, _, _, w = oracle.tessellation_quadrature(N)
    tris = oracle.quadrature.tessellation_triangles(N)
    ref = np.array([_projected_area(*t) for t in tris])
    assert np.max(np.abs(w - ref) / ref) < 2e-4


def test_tessellation_symmetry_and_moments():
    """Mirror and swap symmetries of the point set; second moments exact (the
    face is symmetric under cyclic permutation of the axes); the fourth moment
    of mu converges at second order to 2 pi / 5."""
    for N in (3, 6):
        xi, eta, mu, w = oracle.tessellation_quadrature(N)
        P = np.round(np.stack([xi, eta, mu, w], 1), 12)
        key = lambda A: sorted(map(tuple, A))
        assert key(P) == key(P[:, [1, 0, 2, 3]])
        assert key(P) == key(P * np.array([-1, 1, 1, 1]))
        for v in (xi, eta, mu):
            assert abs((w * v * v).sum() - 2 * np.pi / 3) < 1e-12
    err = []
    for N in (4, 8, 16):
        xi, eta, mu, w = oracle.tessellation_quadrature(N)
        err.append(abs((w * mu ** 4).sum() - 2 * np.pi / 5))
    assert 3.0 < err[0] / err[1] < 5.0 and 3.0 < err[1] / err[2] < 5.0


def test_tessellation_order_22_has_the_papers_1936_angles():
    """The paper's reference runs use the tessellation rule of order N = 22
    with 1936 angles (Sec. 3.1, caption of the lattice figure): 4 N^2 = 1936."""
    xi, eta, mu, w = oracle.tessellation_quadrature(22)
    assert len(w) == 1936
    assert abs(w.sum() - 2 * np.pi) < 1e-12

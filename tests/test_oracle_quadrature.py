"""Pins for the oracle's product quadrature (Sec. 4.1, Eq. sn_2d and Eq.
polar_coordinates): weights sum to 2 pi and the rule integrates low-degree
polynomials of (xi, eta, mu) over the upper hemisphere exactly. The closed
forms are integrals over [0,1] x [0, 2 pi) in (mu, varphi) computed by hand."""
import math

import numpy as np
import pytest

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

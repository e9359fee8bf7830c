"""Angular quadrature on the upper hemisphere (oracle, test infrastructure).

Sec. 4.1 (Eq. sn_2d): ordinates Omega_k = (xi_k, eta_k, mu_k) with mu_k in
[0, 1], xi = sqrt(1-mu^2) cos(varphi), eta = sqrt(1-mu^2) sin(varphi)
(Eq. polar_coordinates), weights normalised to sum to 2*pi.

Tensorised Gauss-Legendre product rule (Sec. 5.1.1 names it as the
alternative to the tessellation rule): an n_p-point Gauss-Legendre rule on
mu in [0, 1] times n_phi equally spaced azimuths at the midpoints
varphi_a = (a + 1/2) 2 pi / n_phi. Ordinate index k = a * n_p + p (azimuth
major, polar fastest). The Gauss-Legendre nodes come from numpy's library
routine (a library primitive used as one step).
"""
import numpy as np


def gauss_legendre_01(n: int):
    """n-point Gauss-Legendre nodes and weights mapped from [-1,1] to [0,1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def product_quadrature(n_p: int, n_phi: int):
    """Return (xi, eta, mu, w), each of length M = n_p * n_phi, sum(w) = 2*pi."""
    mu_p, w_p = gauss_legendre_01(n_p)
    phis = (np.arange(n_phi) + 0.5) * (2.0 * np.pi / n_phi)
    xi = np.empty(n_p * n_phi)
    eta = np.empty_like(xi)
    mu = np.empty_like(xi)
    w = np.empty_like(xi)
    for a, ph in enumerate(phis):
        for p in range(n_p):
            k = a * n_p + p
            s = np.sqrt(1.0 - mu_p[p] ** 2)
            xi[k] = s * np.cos(ph)
            eta[k] = s * np.sin(ph)
            mu[k] = mu_p[p]
            w[k] = w_p[p] * (2.0 * np.pi / n_phi)
    return xi, eta, mu, w

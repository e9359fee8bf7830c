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

Tessellation rule (Sec. 5.1.1, the paper's own choice): the four upper faces
of the octahedron with vertices on the unit sphere, each triangulated into N^2
congruent triangles by dividing its edges into N parts; the quadrature point of
a small triangle is its centroid pushed out to the sphere, its weight the area
of the spherical triangle spanned by its pushed-out vertices (the spherical
excess). M = 4 N^2 points; the spherical triangles tile the hemisphere, so the
weights sum to 2*pi.
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


# upper faces of the octahedron, one per quadrant of azimuth (xi>0,eta>0;
# xi<0,eta>0; xi<0,eta<0; xi>0,eta<0): corners A, B and the pole
_FACES = (((1.0, 0.0, 0.0), (0.0, 1.0, 0.0)), ((0.0, 1.0, 0.0), (-1.0, 0.0, 0.0)),
          ((-1.0, 0.0, 0.0), (0.0, -1.0, 0.0)), ((0.0, -1.0, 0.0), (1.0, 0.0, 0.0)))


def spherical_excess(a, b, c):
    """Area of the spherical triangle with unit-vector corners a, b, c, from
    the triple product form tan(E/2) = |a.(b x c)| / (1 + a.b + b.c + c.a)."""
    num = abs(np.dot(a, np.cross(b, c)))
    den = 1.0 + np.dot(a, b) + np.dot(b, c) + np.dot(c, a)
    return 2.0 * np.arctan2(num, den)


def tessellation_triangles(N: int):
    """Flat small triangles of the tessellation, in quadrature order: face by
    face, rows j = 0..N-1 from the equator up, in each row i = 0..N-1-j the
    upward triangle (i, j) and then, if i < N-1-j, the downward one."""
    pole = np.array([0.0, 0.0, 1.0])
    out = []
    for A, B in _FACES:
        A, B = np.array(A), np.array(B)
        P = lambda i, j: A + (B - A) * (i / N) + (pole - A) * (j / N)
        for j in range(N):
            for i in range(N - j):
                out.append((P(i, j), P(i + 1, j), P(i, j + 1)))
                if i < N - 1 - j:
                    out.append((P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)))
    return out


def tessellation_quadrature(N: int):
    """Return (xi, eta, mu, w) of the tessellation rule of order N (M = 4 N^2)."""
    tris = tessellation_triangles(N)
    M = len(tris)
    xi, eta, mu, w = (np.empty(M) for _ in range(4))
    for k, (p, q, r) in enumerate(tris):
        c = (p + q + r) / 3.0
        c = c / np.linalg.norm(c)
        xi[k], eta[k], mu[k] = c
        w[k] = spherical_excess(p / np.linalg.norm(p), q / np.linalg.norm(q), r / np.linalg.norm(r))
    return xi, eta, mu, w

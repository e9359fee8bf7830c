"""Finite-volume S_N operator on triangle meshes in FP64 (oracle, test infrastructure).

Sec. 4.2 on a mesh of triangles C_i with area A_i. Each edge e_ij has length
l_ij and unit normal n_ij pointing from C_i into C_j. The semi-discrete form
(Eq. sn_2d_eqn_fv, with the area factor on the reaction terms restored) is

  A_i d/dt psi_{k,i} = - sum_{j in S_i} (omega_k . n_ij) l_ij psi_hat_{k,i,j}
                       - A_i sigma_t,i psi_{k,i}
                       + A_i sigma_s,i/(2 pi) sum_l w_l psi_{l,i} + A_i Q_i

with the upwind trace of Eq. upwind1stOrder: psi_hat = R_i where
omega . n_ij > 0, else R_j, both evaluated at the edge midpoint x_ij.
First order: R = psi. Second order (the paper's production scheme, Sec. 4.2):
R_i = psi_i + L_i g_i . r_ij with r_ij = x_ij - x_i (x_i the centroid),
the Green-Gauss gradient g_i = (1/A_i) sum_j l_ij n_ij (psi_i + psi_j)/2 and
the Venkatakrishnan limiter L_i = min_j L_ij of Eq. V_limiter, written as
printed: Delta = (1/2) g_i . r_ij; for Delta > 0
L_ij = (1/Delta) ((b^2 + e^2) Delta + 2 Delta^2 b) / (b^2 + 2 Delta^2 + b Delta + e^2)
with b = beta_max = max_{j in S_i and i} psi_j - psi_i, for Delta < 0 the same
with b = beta_min (the min), and L_ij = 1 for Delta = 0; e = K A_i^3, K = 1.
Boundary edges use a ghost cell holding psi^- (the side's inflow value for
entering ordinates, 0 otherwise): it enters the gradient and the max/min as a
neighbour value, and fluxes through boundary edges are first order (Sec.
4.2, last paragraph).

The mesh metrics (areas, outward normals times lengths, neighbours, boundary
sides) are derived here from the vertex list alone.
"""
import numpy as np

from sn_inputs import INFLOW, PERIODIC


def triangle_metrics(vertices, triangles, box):
    """Areas, outward (n*l) per local edge, neighbour per local edge (-1 on the
    boundary) and boundary side per local edge (0..3 for x-, x+, y-, y+; -1 inside).

    Local edge e of triangle (a, b, c) runs from vertex e to vertex (e+1) % 3.
    For a counter-clockwise triangle the outward normal of edge p->q scaled by
    its length is (q_y - p_y, -(q_x - p_x)).
    """
    V = np.asarray(vertices, dtype=np.float64)
    T = np.asarray(triangles, dtype=np.int64)
    n_t = T.shape[0]
    P = V[T]                                   # [n_t, 3, 2]
    a, b, c = P[:, 0], P[:, 1], P[:, 2]
    area = 0.5 * ((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]))
    Pn = np.roll(P, -1, axis=1)                # q of each edge p->q
    nl = np.stack([Pn[:, :, 1] - P[:, :, 1], -(Pn[:, :, 0] - P[:, :, 0])], axis=2)   # [n_t, 3, 2]
    owner = {}
    for t in range(n_t):
        for e in range(3):
            owner[(int(T[t, e]), int(T[t, (e + 1) % 3]))] = t
    nbr = np.full((n_t, 3), -1, dtype=np.int64)
    for t in range(n_t):
        for e in range(3):
            nbr[t, e] = owner.get((int(T[t, (e + 1) % 3]), int(T[t, e])), -1)
    side = np.full((n_t, 3), -1, dtype=np.int64)
    xmin, ymin, xmax, ymax = box
    mid = 0.5 * (P + Pn)                       # edge midpoints
    bnd = nbr < 0
    d = np.stack([np.abs(mid[:, :, 0] - xmin), np.abs(mid[:, :, 0] - xmax),
                  np.abs(mid[:, :, 1] - ymin), np.abs(mid[:, :, 1] - ymax)], axis=2)
    side[bnd] = np.argmin(d[bnd], axis=1)
    return area, nl, nbr, side


def venkatakrishnan(delta, beta_max, beta_min, eps):
    """Limiter value of one edge (Eq. V_limiter as printed), elementwise."""
    eps2 = eps * eps
    with np.errstate(divide="ignore", invalid="ignore"):
        up = ((beta_max ** 2 + eps2) * delta + 2 * delta ** 2 * beta_max) / \
            (beta_max ** 2 + 2 * delta ** 2 + beta_max * delta + eps2) / delta
        dn = ((beta_min ** 2 + eps2) * delta + 2 * delta ** 2 * beta_min) / \
            (beta_min ** 2 + 2 * delta ** 2 + beta_min * delta + eps2) / delta
    return np.where(delta > 0, up, np.where(delta < 0, dn, 1.0))


class TriangleOracle:
    def __init__(self, problem, quad, order=1, K=1.0):
        if order not in (1, 2):
            raise ValueError("order must be 1 or 2")
        self.order = order
        mesh = problem.mesh
        self.xi, self.eta, _, self.w = [np.asarray(q, dtype=np.float64) for q in quad]
        self.M = self.xi.size
        self.area, self.nl, self.nbr, self.side = triangle_metrics(mesh.vertices, mesh.triangles, mesh.box)
        self.n_cells = self.area.size
        # second order: centroid-to-edge-midpoint vectors, the neighbour's local
        # index of each shared edge, and the limiter's epsilon = K A^3
        P = np.asarray(mesh.vertices, dtype=np.float64)[np.asarray(mesh.triangles)]
        self.r = 0.5 * (P + np.roll(P, -1, axis=1)) - P.mean(axis=1)[:, None, :]     # [n, 3, 2]
        self.nbr_edge = np.full((self.n_cells, 3), -1, dtype=np.int64)
        for e in range(3):
            for f in range(3):
                j = self.nbr[:, e]
                hit = (j >= 0)
                hit[hit] = self.nbr[j[hit], f] == np.nonzero(hit)[0]
                self.nbr_edge[hit, e] = f
        self.eps = K * self.area ** 3
        m = problem.materials
        mat = np.asarray(m.cell_mat)
        self.sigma_a = np.asarray(m.sigma_a, dtype=np.float64)[mat]
        self.sigma_s = np.asarray(m.sigma_s, dtype=np.float64)[mat]
        self.sigma_t = self.sigma_a + self.sigma_s
        self.Q = np.asarray(m.Q, dtype=np.float64)[mat]
        self.region = np.asarray(m.cell_region)
        self.n_regions = max(m.n_regions, int(self.region.max()) + 1 if self.region.size else 0)
        bc = problem.boundary
        if any(k == PERIODIC for k in bc.kind):
            raise NotImplementedError("triangle meshes: no periodic sides")
        normals = ((-1.0, 0.0), (1.0, 0.0), (0.0, -1.0), (0.0, 1.0))
        self.ghost = np.zeros((4, self.M))
        for s in range(4):
            on = normals[s][0] * self.xi + normals[s][1] * self.eta
            val = bc.inflow[s] if bc.kind[s] == INFLOW else 0.0
            self.ghost[s] = np.where(on < 0.0, val, 0.0)

    def phi(self, psi):
        """Scalar flux phi_i = sum_k w_k psi_{k,i} (Eq. sn_2d)."""
        return psi @ self.w

    def neighbour_values(self, psi, e):
        """psi of the cell across local edge e, or the ghost value psi^-: [n_cells, M]."""
        j = self.nbr[:, e]
        inside = j >= 0
        other = np.empty_like(psi)
        other[inside] = psi[j[inside]]
        other[~inside] = self.ghost[self.side[~inside, e]]
        return other

    def gradient(self, psi):
        """Green-Gauss gradient (gx, gy), each [n_cells, M]."""
        gx = np.zeros_like(psi)
        gy = np.zeros_like(psi)
        for e in range(3):
            avg = 0.5 * (psi + self.neighbour_values(psi, e))
            gx += self.nl[:, e, 0:1] * avg
            gy += self.nl[:, e, 1:2] * avg
        return gx / self.area[:, None], gy / self.area[:, None]

    def limiter(self, psi, gx, gy):
        """Venkatakrishnan limiter L_i per cell and ordinate: [n_cells, M]."""
        nb = [self.neighbour_values(psi, e) for e in range(3)]
        pmax = np.maximum(psi, np.maximum(np.maximum(nb[0], nb[1]), nb[2]))
        pmin = np.minimum(psi, np.minimum(np.minimum(nb[0], nb[1]), nb[2]))
        L = None
        for e in range(3):
            delta = 0.5 * (gx * self.r[:, e, 0:1] + gy * self.r[:, e, 1:2])
            Le = venkatakrishnan(delta, pmax - psi, pmin - psi, self.eps[:, None])
            L = Le if L is None else np.minimum(L, Le)
        return L

    def reconstruct(self, psi):
        """R_i at the three edge midpoints: [3][n_cells, M] (first order: psi)."""
        if self.order == 1:
            return [psi, psi, psi]
        gx, gy = self.gradient(psi)
        L = self.limiter(psi, gx, gy)
        return [psi + L * (gx * self.r[:, e, 0:1] + gy * self.r[:, e, 1:2]) for e in range(3)]

    def edge_trace(self, psi, e, R=None):
        """Upwind trace on local edge e of every cell: [n_cells, M]. Boundary
        edges are first order (cell value or ghost)."""
        on = self.nl[:, e, 0:1] * self.xi[None, :] + self.nl[:, e, 1:2] * self.eta[None, :]
        j = self.nbr[:, e]
        inside = j >= 0
        if R is None or self.order == 1:
            return np.where(on > 0.0, psi, self.neighbour_values(psi, e)), on
        mine = np.where(inside[:, None], R[e], psi)
        other = np.empty_like(psi)
        for f in range(3):
            sel = inside & (self.nbr_edge[:, e] == f)
            other[sel] = R[f][j[sel]]
        other[~inside] = self.ghost[self.side[~inside, e]]
        return np.where(on > 0.0, mine, other), on

    def flux_sum(self, psi):
        R = self.reconstruct(psi)
        s = np.zeros_like(psi)
        for e in range(3):
            tr, on = self.edge_trace(psi, e, R)
            s += on * tr
        return s

    def F(self, psi):
        phi = self.phi(psi)
        collide = -self.sigma_t[:, None] * psi + (self.sigma_s * phi / (2.0 * np.pi))[:, None] \
            + self.Q[:, None]
        return -self.flux_sum(psi) / self.area[:, None] + collide

    def outflow(self, psi):
        tot = 0.0
        for e in range(3):
            b = self.nbr[:, e] < 0
            if not b.any():
                continue
            tr, on = self.edge_trace(psi, e)
            tot += float(np.sum((on[b] * tr[b]) @ self.w))
        return tot

    def integrands(self, psi):
        phi = self.phi(psi)
        a = self.area * self.sigma_a * phi
        absr = np.array([a[self.region == r].sum() for r in range(self.n_regions)])
        return {"abs": absr, "mass": float(np.sum(self.area * phi)), "outflow": self.outflow(psi)}

    def source_rate(self):
        return float(np.sum(self.area * self.Q) * self.w.sum())

    def min_2A_over_P(self):
        """min_i 2 A_i / P_i, P_i the perimeter (bounds the outflow speed of a cell)."""
        perim = np.linalg.norm(self.nl, axis=2).sum(axis=1)
        return float(np.min(2.0 * self.area / perim))

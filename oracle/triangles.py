"""Finite-volume S_N operator on triangle meshes in FP64 (oracle, test infrastructure).

Sec. 4.2 on a mesh of triangles C_i with area A_i. Each edge e_ij has length
l_ij and unit normal n_ij pointing from C_i into C_j. The semi-discrete form
(Eq. sn_2d_eqn_fv, with the area factor on the reaction terms restored) is

  A_i d/dt psi_{k,i} = - sum_{j in S_i} (omega_k . n_ij) l_ij psi_hat_{k,i,j}
                       - A_i sigma_t,i psi_{k,i}
                       + A_i sigma_s,i/(2 pi) sum_l w_l psi_{l,i} + A_i Q_i

with the first-order upwind trace (Eq. upwind1stOrder with R = psi):
psi_hat = psi_i where omega . n_ij > 0, else psi_j. Boundary edges use a ghost
cell holding psi^- (the side's inflow value for entering ordinates, 0
otherwise), with first-order fluxes (Sec. 4.2, last paragraph).

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


class TriangleOracle:
    def __init__(self, problem, quad, order=1):
        if order != 1:
            raise NotImplementedError("triangle meshes: first order only")
        mesh = problem.mesh
        self.xi, self.eta, _, self.w = [np.asarray(q, dtype=np.float64) for q in quad]
        self.M = self.xi.size
        self.area, self.nl, self.nbr, self.side = triangle_metrics(mesh.vertices, mesh.triangles, mesh.box)
        self.n_cells = self.area.size
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

    def edge_trace(self, psi, e):
        """Upwind trace on local edge e of every cell: [n_cells, M]."""
        on = self.nl[:, e, 0:1] * self.xi[None, :] + self.nl[:, e, 1:2] * self.eta[None, :]
        j = self.nbr[:, e]
        inside = j >= 0
        other = np.empty_like(psi)
        other[inside] = psi[j[inside]]
        other[~inside] = self.ghost[self.side[~inside, e]]
        return np.where(on > 0.0, psi, other), on

    def flux_sum(self, psi):
        s = np.zeros_like(psi)
        for e in range(3):
            tr, on = self.edge_trace(psi, e)
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

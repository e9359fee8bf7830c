"""Cartesian finite-volume S_N operator F(psi) in FP64 (oracle, test infrastructure).

Follows Sec. 4.2 on a uniform nx x ny grid of rectangles (cell id j*nx + i):

  A_i d/dt psi_{k,i} + sum_faces (omega_k . n) l psi_hat_{k,face}
      + A_i sigma_t,i psi_{k,i} = A_i sigma_s,i/(2 pi) sum_l w_l psi_{l,i} + A_i Q_i

(Eq. sn_2d_eqn_fv, with the area factor on the reaction terms restored). The
trace psi_hat on a face is the reconstruction R from the upwind cell (Eq.
upwind1stOrder): the cell on the side the ordinate comes from. First order:
R = psi_i. Second order (MUSCL): R = psi_i +/- slope_i / 2 with the minmod
slope per dimension, slope_i = minmod(psi_{i+1} - psi_i, psi_i - psi_{i-1}),
minmod(a, b) = 0 if a b <= 0 else the argument of smaller magnitude.

Boundaries (Sec. 4.2, last paragraph): a ghost cell across each boundary face
holds psi^-: the side's inflow value for ordinates entering through that side,
0 otherwise. Fluxes through boundary faces are first order (the trace is the
ghost value for entering ordinates, the cell value for leaving ones). A slope
next to the boundary uses the ghost value as the missing neighbour. Periodic
sides wrap instead and have no boundary faces.

QoI integrands of a state (Sec. 3.1 QoI-3..5 and the mass balance):
  abs[r]  = sum_{i in region r} A_i sigma_a,i phi_i
  mass    = sum_i A_i phi_i
  outflow = sum_{boundary faces} l sum_k w_k (omega_k . n) psi_hat_k
and, for each QoI box b (problem.extra["boxes"], rectangles (x_lo, x_hi, y_lo,
y_hi) with edges on grid lines; the squares S_l of Sec. 3.1 QoI-1/2):
  box_out[b] = sum_{faces f of the box boundary} l_f sum_k w_k max(omega_k . n_f, 0) psi_hat_k,f
with n_f pointing out of the box and psi_hat the same upwind trace the fluxes
use, i.e. the outflow through the box boundary of Sec. 3.1 QoI-1 evaluated with
the scheme's own traces (reading: the paper defines the integral for the
continuous solution and leaves the discrete trace open).
"""
import numpy as np

from sn_inputs import VACUUM, INFLOW, PERIODIC


def minmod(a, b):
    """0 where a and b differ in sign (or one is 0), else the one of smaller magnitude."""
    return np.where(a * b > 0.0, np.where(np.abs(a) < np.abs(b), a, b), 0.0)


class CartesianOracle:
    def __init__(self, problem, quad, order=1):
        mesh = problem.mesh
        self.nx, self.ny = mesh.nx, mesh.ny
        self.dx, self.dy = mesh.dx, mesh.dy
        self.area = mesh.dx * mesh.dy
        self.xi, self.eta, _, self.w = [np.asarray(q, dtype=np.float64) for q in quad]
        self.M = self.xi.size
        self.order = order
        m = problem.materials
        mat = np.asarray(m.cell_mat)
        self.sigma_a = np.asarray(m.sigma_a, dtype=np.float64)[mat]
        self.sigma_s = np.asarray(m.sigma_s, dtype=np.float64)[mat]
        self.sigma_t = self.sigma_a + self.sigma_s
        self.Q = np.asarray(m.Q, dtype=np.float64)[mat]
        self.region = np.asarray(m.cell_region)
        self.n_regions = max(m.n_regions, int(self.region.max()) + 1 if self.region.size else 0)
        bc = problem.boundary
        self.kind = tuple(bc.kind)
        if (self.kind[0] == PERIODIC) != (self.kind[1] == PERIODIC) or \
           (self.kind[2] == PERIODIC) != (self.kind[3] == PERIODIC):
            raise ValueError("periodic sides come in pairs")
        # psi^- per side and ordinate: inflow value for entering ordinates, else 0
        # outward normals: x- (-1,0), x+ (1,0), y- (0,-1), y+ (0,1)
        normals = ((-1.0, 0.0), (1.0, 0.0), (0.0, -1.0), (0.0, 1.0))
        self.ghost = []
        for s in range(4):
            on = normals[s][0] * self.xi + normals[s][1] * self.eta
            val = bc.inflow[s] if self.kind[s] == INFLOW else 0.0
            self.ghost.append(np.where(on < 0.0, val, 0.0))
        # QoI boxes as cell index ranges [i0, i1) x [j0, j1)
        self.boxes = []
        for box in problem.extra.get("boxes", ()):
            lim = []
            for e, v in enumerate(box):
                o, h = (mesh.x0, mesh.dx) if e < 2 else (mesh.y0, mesh.dy)
                r = int(round((v - o) / h))
                if abs(o + r * h - v) > 1e-9 * max(1.0, abs(v)):
                    raise ValueError(f"box edge {v} is not a grid line")
                lim.append(r)
            self.boxes.append(tuple(lim))

    # ------------------------------------------------------------------
    def phi(self, psi):
        """Scalar flux phi_i = sum_k w_k psi_{k,i} (Eq. sn_2d)."""
        return psi @ self.w

    def _face_traces(self, P, vel, g_lo, g_hi, periodic):
        """Upwind traces on the faces normal to the last spatial axis.

        P: [..., L, M] cell values along the axis; vel: [M] velocity component
        along the axis. Returns T with T[..., f, :] the trace on the face
        between cell f-1 and cell f: faces 0..L (L+1 faces) when bounded,
        faces 0..L-1 (face 0 joins cell L-1 and cell 0) when periodic.
        """
        L = P.shape[-2]
        if periodic:
            lo = np.roll(P, 1, axis=-2)      # cell i-1
            hi = np.roll(P, -1, axis=-2)     # cell i+1
        else:
            glo = np.broadcast_to(g_lo, P[..., :1, :].shape)
            ghi = np.broadcast_to(g_hi, P[..., :1, :].shape)
            lo = np.concatenate([glo, P[..., :-1, :]], axis=-2)
            hi = np.concatenate([P[..., 1:, :], ghi], axis=-2)
        if self.order == 2:
            slope = minmod(hi - P, P - lo)
        else:
            slope = np.zeros_like(P)
        R_plus = P + 0.5 * slope             # value of cell i at its upper face
        R_minus = P - 0.5 * slope            # value of cell i at its lower face
        if periodic:
            left_state = np.roll(R_plus, 1, axis=-2)    # from cell f-1 (mod L)
            right_state = R_minus                       # from cell f
        else:
            left_state = np.concatenate([glo, R_plus], axis=-2)     # faces 0..L
            right_state = np.concatenate([R_minus, ghi], axis=-2)
            # boundary faces are first order: cell value, not the reconstruction
            left_state[..., L, :] = P[..., L - 1, :]
            right_state[..., 0, :] = P[..., 0, :]
        return np.where(vel > 0.0, left_state, right_state)

    def traces(self, psi):
        """(Tx, Ty): traces on x-faces [ny, nx(+1), M] and y-faces [ny(+1), nx, M]."""
        P = psi.reshape(self.ny, self.nx, self.M)
        px = self.kind[0] == PERIODIC
        py = self.kind[2] == PERIODIC
        Tx = self._face_traces(P, self.xi, self.ghost[0], self.ghost[1], px)
        Py = np.swapaxes(P, 0, 1)            # [nx, ny, M]: y along axis -2
        Ty = np.swapaxes(self._face_traces(Py, self.eta, self.ghost[2], self.ghost[3], py), 0, 1)
        return Tx, Ty

    def flux_sum(self, psi):
        """sum over the four faces of (omega . n) l psi_hat, per cell and ordinate."""
        Tx, Ty = self.traces(psi)
        nx, ny = self.nx, self.ny
        if self.kind[0] == PERIODIC:
            Tx_lo, Tx_hi = Tx, np.roll(Tx, -1, axis=1)
        else:
            Tx_lo, Tx_hi = Tx[:, :nx, :], Tx[:, 1:, :]
        if self.kind[2] == PERIODIC:
            Ty_lo, Ty_hi = Ty, np.roll(Ty, -1, axis=0)
        else:
            Ty_lo, Ty_hi = Ty[:ny, :, :], Ty[1:, :, :]
        # faces: x+ n=(1,0) l=dy; x- n=(-1,0) l=dy; y+ n=(0,1) l=dx; y- n=(0,-1) l=dx
        s = (self.xi * self.dy) * Tx_hi + (-self.xi * self.dy) * Tx_lo \
            + (self.eta * self.dx) * Ty_hi + (-self.eta * self.dx) * Ty_lo
        return s.reshape(nx * ny, self.M)

    def F(self, psi):
        """Right-hand side of the semi-discrete system d psi/dt = F(psi) (Eq. ODE)."""
        phi = self.phi(psi)
        collide = -self.sigma_t[:, None] * psi + (self.sigma_s * phi / (2.0 * np.pi))[:, None] \
            + self.Q[:, None]
        return -self.flux_sum(psi) / self.area + collide

    # ------------------------------------------------------------------
    def outflow(self, psi):
        """Net particle flow out through the domain boundary at state psi."""
        if all(k == PERIODIC for k in self.kind):
            return 0.0
        Tx, Ty = self.traces(psi)
        tot = 0.0
        if self.kind[0] != PERIODIC:
            tot += self.dy * np.sum((Tx[:, 0, :] * (-self.xi)) @ self.w)
            tot += self.dy * np.sum((Tx[:, self.nx, :] * self.xi) @ self.w)
        if self.kind[2] != PERIODIC:
            tot += self.dx * np.sum((Ty[0, :, :] * (-self.eta)) @ self.w)
            tot += self.dx * np.sum((Ty[self.ny, :, :] * self.eta) @ self.w)
        return float(tot)

    def box_flow(self, psi):
        """(out, in) per QoI box: particle flow leaving and entering through the
        box boundary, sum over its faces of l sum_k w_k max(+-omega_k . n, 0)
        psi_hat_k with the upwind traces of the fluxes (n out of the box)."""
        Tx, Ty = self.traces(psi)
        fx, fy = Tx.shape[1], Ty.shape[0]       # faces per row / column (nx+1 bounded, nx periodic)
        out, inn = [], []
        for (i0, i1, j0, j1) in self.boxes:
            sides = ((Tx[j0:j1, i0 % fx, :], -self.xi, self.dy), (Tx[j0:j1, i1 % fx, :], self.xi, self.dy),
                     (Ty[j0 % fy, i0:i1, :], -self.eta, self.dx), (Ty[j1 % fy, i0:i1, :], self.eta, self.dx))
            o = n = 0.0
            for T, on, l in sides:
                o += l * float(np.sum(T @ (self.w * np.maximum(on, 0.0))))
                n += l * float(np.sum(T @ (self.w * np.maximum(-on, 0.0))))
            out.append(o)
            inn.append(n)
        return np.array(out), np.array(inn)

    def integrands(self, psi):
        """QoI integrands at state psi: abs per region, mass, outflow (and the
        outflow of each QoI box, if any)."""
        phi = self.phi(psi)
        a = self.area * self.sigma_a * phi
        absr = np.array([a[self.region == r].sum() for r in range(self.n_regions)])
        S = {"abs": absr, "mass": float(self.area * phi.sum()), "outflow": self.outflow(psi)}
        if self.boxes:
            S["box_out"] = self.box_flow(psi)[0]
        return S

    def source_rate(self):
        """Particles emitted per unit time: sum_i A_i Q_i sum_k w_k = 2 pi sum_i A_i Q_i."""
        return float(self.area * self.Q.sum() * self.w.sum())

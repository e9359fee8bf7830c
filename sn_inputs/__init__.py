"""Seeded, synthetic inputs for the 2-D S_N benchmarks (lattice and enclosure).

This module is shared by the FP64 oracle, the tests and the benchmark. It holds
problem *definitions* only: geometry, material tables, meshes, random states and
parameter draws. It contains none of the method's arithmetic (no quadrature, no
fluxes, no collision term, no time stepping, no mesh metrics).

Problem sources:
  * Lattice benchmark, Sec. 3.1 (blocks C_ij, the blue set B, the red source R,
    material table of Fig. "lattice"), translated from [-3.5,3.5]^2 to [0,7]^2.
  * Enclosure (cavity) benchmark: a one-sided variant of the Hohlraum of Sec. 3.2
    (walls of sigma_a = 100, an inner block with an absorbing rim, inflow on
    x = 0 only), with the rim scattering taken from the paper's green material.
  * Random numbers: splitmix64 (Steele, Lea and Flood, "Fast splittable
    pseudorandom number generators", OOPSLA 2014) used as a counter-based
    generator: draw number i of stream `seed` is the splitmix64 output after
    i+1 increments of the state `seed`.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------
# counter-based RNG (splitmix64)
# ----------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter) -> np.ndarray:
    """Return splitmix64 output number `counter` (0-based) of the stream started at `seed`.

    The state after counter+1 increments is seed + (counter+1)*golden (mod 2^64);
    the output is the splitmix64 finaliser applied to that state.
    """
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counter) -> np.ndarray:
    """Uniform doubles in [0,1): top 53 bits of splitmix64 output times 2^-53."""
    return (splitmix64(seed, counter) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ----------------------------------------------------------------------------
# problem containers
# ----------------------------------------------------------------------------
VACUUM, INFLOW, PERIODIC = 0, 1, 2
SIDES = ("x-", "x+", "y-", "y+")


@dataclass
class Materials:
    """Piecewise-constant material table plus per-cell material and QoI-region ids."""
    sigma_a: np.ndarray          # [n_mat] float64
    sigma_s: np.ndarray          # [n_mat] float64
    Q: np.ndarray                # [n_mat] float64, isotropic source density
    cell_mat: np.ndarray         # [n_cells] int32
    cell_region: np.ndarray      # [n_cells] int32
    region_names: tuple = ()

    @property
    def n_regions(self) -> int:
        return len(self.region_names)


@dataclass
class Boundary:
    """Per side (x-, x+, y-, y+): kind (VACUUM | INFLOW | PERIODIC) and the
    isotropic inflow value psi^- used for ordinates entering through that side."""
    kind: tuple = (VACUUM, VACUUM, VACUUM, VACUUM)
    inflow: tuple = (0.0, 0.0, 0.0, 0.0)


@dataclass
class CartesianMesh:
    nx: int
    ny: int
    x0: float
    y0: float
    dx: float
    dy: float

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny

    def centres(self):
        """Cell centres, cell id = j*nx + i (x fastest)."""
        xc = self.x0 + (np.arange(self.nx) + 0.5) * self.dx
        yc = self.y0 + (np.arange(self.ny) + 0.5) * self.dy
        X, Y = np.meshgrid(xc, yc)          # [ny, nx]
        return X.ravel(), Y.ravel()


@dataclass
class TriangleMesh:
    vertices: np.ndarray         # [n_vert, 2] float64
    triangles: np.ndarray        # [n_tri, 3] int32, counter-clockwise
    box: tuple = (0.0, 0.0, 1.0, 1.0)   # (xmin, ymin, xmax, ymax) of the domain

    @property
    def n_cells(self) -> int:
        return int(self.triangles.shape[0])

    def centroids(self):
        v = self.vertices[self.triangles]   # [n_tri, 3, 2]
        c = v.mean(axis=1)
        return c[:, 0], c[:, 1]


@dataclass
class Problem:
    mesh: object                 # CartesianMesh | TriangleMesh
    materials: Materials
    boundary: Boundary
    t_end: float
    name: str = ""
    extra: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# lattice benchmark (Sec. 3.1) on [0,7]^2
# ----------------------------------------------------------------------------
# block (i, j), 0-based, i = x index, j = y index, block = [i,i+1] x [j,j+1].
# Blue set B of Sec. 3.1 (paper's 1-based C_{i,j} minus one in each index).
LATTICE_ABSORBERS = ((1, 1), (3, 1), (5, 1), (2, 2), (4, 2), (1, 3), (5, 3),
                     (2, 4), (4, 4), (1, 5), (5, 5))
LATTICE_SOURCE = (3, 3)
MAT_WHITE, MAT_BLUE, MAT_RED = 0, 1, 2
LATTICE_REGIONS = ("white", "blue", "red")
# squares S_l = [-l, l]^2 of QoI-1/2 (Sec. 3.1), l = 1.5 and 2.5, in [0,7]^2:
# (x_lo, x_hi, y_lo, y_hi); their edges are grid lines when n is a multiple of 7
LATTICE_QOI_SQUARES = ((2.0, 5.0, 2.0, 5.0), (1.0, 6.0, 1.0, 6.0))


def lattice_extra(n: int) -> dict:
    """The QoI squares, on grids where they follow cell faces (n multiple of 7)."""
    return {"boxes": LATTICE_QOI_SQUARES} if n % 7 == 0 else {}


def lattice_block_material(bi: np.ndarray, bj: np.ndarray) -> np.ndarray:
    mat = np.full(np.shape(bi), MAT_WHITE, dtype=np.int32)
    for (i, j) in LATTICE_ABSORBERS:
        mat[(bi == i) & (bj == j)] = MAT_BLUE
    mat[(bi == LATTICE_SOURCE[0]) & (bj == LATTICE_SOURCE[1])] = MAT_RED
    return mat


def lattice_materials_table(sigma_a_blue=10.0, sigma_s_white=1.0, sigma_s_red=1.0, q_red=1.0):
    """Material table of the lattice (Sec. 3.1): white (sigma_s = 1), blue
    (sigma_a = 10), red (sigma_s = 1, Q = 1). DP-1 varies sigma_a_blue and the
    scattering of the white blocks."""
    sigma_a = np.array([0.0, sigma_a_blue, 0.0])
    sigma_s = np.array([sigma_s_white, 0.0, sigma_s_red])
    Q = np.array([0.0, 0.0, q_red])
    return sigma_a, sigma_s, Q


def lattice_problem(n: int, sigma_a_blue=10.0, sigma_s_scatter=1.0, t_end=3.2) -> Problem:
    """Lattice checkerboard on an n x n Cartesian grid over [0,7]^2, vacuum
    boundaries, psi0 = 0, T = 3.2. Cells are classified by their centre. When n
    is a multiple of 7 the QoI squares S_1.5, S_2.5 are attached as boxes."""
    mesh = CartesianMesh(nx=n, ny=n, x0=0.0, y0=0.0, dx=7.0 / n, dy=7.0 / n)
    xc, yc = mesh.centres()
    mat = lattice_block_material(np.floor(xc).astype(int), np.floor(yc).astype(int))
    sa, ss, q = lattice_materials_table(sigma_a_blue, sigma_s_scatter, sigma_s_scatter)
    m = Materials(sigma_a=sa, sigma_s=ss, Q=q, cell_mat=mat,
                  cell_region=mat.copy(), region_names=LATTICE_REGIONS)
    return Problem(mesh=mesh, materials=m, boundary=Boundary(), t_end=t_end, name=f"lattice{n}",
                   extra=lattice_extra(n))


def lattice_dp2_nominal():
    """Per-block cross-sections [7, 7] (index [i, j], i along x) equal to the
    nominal table of Sec. 3.1: the DP-2 point at which the lattice is the
    three-material checkerboard."""
    bi, bj = np.meshgrid(np.arange(7), np.arange(7), indexing="ij")
    cls = lattice_block_material(bi, bj)
    sa, ss, _ = lattice_materials_table()
    return sa[cls], ss[cls]


def lattice_dp2_problem(n: int, sigma_a_blocks, sigma_s_blocks, q_red=1.0, t_end=3.2) -> Problem:
    """Lattice with the DP-2 design parameters of Sec. 3.1.3: one absorption and
    one scattering cross-section per block C_ij (arrays [7, 7], index [i, j], i
    along x). Material id = 7 j + i (49 materials); the source Q = q_red sits in
    the red centre block only; the QoI regions stay the white / blue / red
    classes of the nominal layout."""
    sa = np.asarray(sigma_a_blocks, dtype=np.float64)
    ss = np.asarray(sigma_s_blocks, dtype=np.float64)
    assert sa.shape == (7, 7) and ss.shape == (7, 7)
    mesh = CartesianMesh(nx=n, ny=n, x0=0.0, y0=0.0, dx=7.0 / n, dy=7.0 / n)
    xc, yc = mesh.centres()
    bi, bj = np.floor(xc).astype(int), np.floor(yc).astype(int)
    mat = (7 * bj + bi).astype(np.int32)
    region = lattice_block_material(bi, bj)
    # material m = 7 j + i: flatten [i, j] with j slowest
    Q = np.zeros(49)
    Q[7 * LATTICE_SOURCE[1] + LATTICE_SOURCE[0]] = q_red
    m = Materials(sigma_a=sa.T.ravel().copy(), sigma_s=ss.T.ravel().copy(), Q=Q, cell_mat=mat,
                  cell_region=region, region_names=LATTICE_REGIONS)
    return Problem(mesh=mesh, materials=m, boundary=Boundary(), t_end=t_end, name=f"lattice{n}_dp2",
                   extra=lattice_extra(n))


def lattice_triangle_problem(n: int, jitter=0.0, seed=0, t_end=3.2) -> Problem:
    """Lattice geometry on the split-square triangle mesh (material by centroid)."""
    mesh = split_grid_mesh(n, 7.0, jitter=jitter, seed=seed)
    xc, yc = mesh.centroids()
    mat = lattice_block_material(np.floor(xc).astype(int), np.floor(yc).astype(int))
    sa, ss, q = lattice_materials_table()
    m = Materials(sigma_a=sa, sigma_s=ss, Q=q, cell_mat=mat,
                  cell_region=mat.copy(), region_names=LATTICE_REGIONS)
    return Problem(mesh=mesh, materials=m, boundary=Boundary(), t_end=t_end, name=f"lattice_tri{n}")


# ----------------------------------------------------------------------------
# enclosure (cavity) benchmark on [0,1.3]^2
# ----------------------------------------------------------------------------
ENC_VOID, ENC_WALL, ENC_RIM, ENC_CORE = 0, 1, 2, 3
ENCLOSURE_REGIONS = ("void", "wall", "rim", "core")


def enclosure_material_at(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Material id of the enclosure at points (x, y).

    walls (sigma_a=100, sigma_s=0.1), 0.05 thick: bottom, top, right, and the
    left wall except its opening y in [0.4, 0.9]; the inner block
    [0.45,0.85]x[0.25,1.05] is a rim of 0.05 around the core [0.5,0.8]x[0.3,1.0];
    void elsewhere.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    mat = np.full(x.shape, ENC_VOID, dtype=np.int32)
    wall = (y < 0.05) | (y > 1.25) | (x > 1.25) | ((x < 0.05) & ((y < 0.4) | (y > 0.9)))
    block = (x > 0.45) & (x < 0.85) & (y > 0.25) & (y < 1.05)
    core = (x > 0.5) & (x < 0.8) & (y > 0.3) & (y < 1.0)
    mat[block] = ENC_RIM
    mat[core] = ENC_CORE
    mat[wall] = ENC_WALL
    return mat


def enclosure_materials_table(rim_sigma_s=90.0):
    sigma_a = np.array([0.0, 100.0, 10.0, 0.1])
    sigma_s = np.array([0.0, 0.1, rim_sigma_s, 0.9])
    Q = np.zeros(4)
    return sigma_a, sigma_s, Q


def enclosure_problem(n: int, jitter=0.2, seed=0, t_end=2.6, rim_sigma_s=90.0) -> Problem:
    """Enclosure on the n x n split-square triangle mesh with interior vertices
    jittered by U[-jitter*dx, jitter*dx]; isotropic inflow psi^- = 1 on x = 0."""
    mesh = split_grid_mesh(n, 1.3, jitter=jitter, seed=seed)
    xc, yc = mesh.centroids()
    mat = enclosure_material_at(xc, yc)
    sa, ss, q = enclosure_materials_table(rim_sigma_s)
    m = Materials(sigma_a=sa, sigma_s=ss, Q=q, cell_mat=mat, cell_region=mat.copy(),
                  region_names=ENCLOSURE_REGIONS)
    bc = Boundary(kind=(INFLOW, VACUUM, VACUUM, VACUUM), inflow=(1.0, 0.0, 0.0, 0.0))
    return Problem(mesh=mesh, materials=m, boundary=bc, t_end=t_end, name=f"enclosure{n}")


def enclosure_cartesian_problem(n: int, t_end=2.6, rim_sigma_s=90.0) -> Problem:
    """Enclosure geometry on an (unjittered) n x n Cartesian grid."""
    mesh = CartesianMesh(nx=n, ny=n, x0=0.0, y0=0.0, dx=1.3 / n, dy=1.3 / n)
    xc, yc = mesh.centres()
    mat = enclosure_material_at(xc, yc)
    sa, ss, q = enclosure_materials_table(rim_sigma_s)
    m = Materials(sigma_a=sa, sigma_s=ss, Q=q, cell_mat=mat, cell_region=mat.copy(),
                  region_names=ENCLOSURE_REGIONS)
    bc = Boundary(kind=(INFLOW, VACUUM, VACUUM, VACUUM), inflow=(1.0, 0.0, 0.0, 0.0))
    return Problem(mesh=mesh, materials=m, boundary=bc, t_end=t_end, name=f"enclosure_cart{n}")


# ----------------------------------------------------------------------------
# split-square triangle meshes
# ----------------------------------------------------------------------------
def split_grid_mesh(n: int, L: float, jitter: float = 0.0, seed: int = 0, ny: int | None = None,
                    Ly: float | None = None) -> TriangleMesh:
    """n x ny squares over [0,L]x[0,Ly], each split along its (i,j)->(i+1,j+1)
    diagonal into two counter-clockwise triangles: lower id 2c with vertices
    (i,j),(i+1,j),(i+1,j+1) and upper id 2c+1 with (i,j),(i+1,j+1),(i,j+1),
    where c = j*n + i. Vertex id v = j*(n+1) + i. Interior vertices move by
    U[-jitter*dx, jitter*dx] in each coordinate; draws 2v and 2v+1 of the
    splitmix64 stream `seed`. Boundary vertices stay on the boundary."""
    ny = n if ny is None else ny
    Ly = L if Ly is None else Ly
    dx, dy = L / n, Ly / ny
    iv, jv = np.meshgrid(np.arange(n + 1), np.arange(ny + 1))
    iv, jv = iv.ravel(), jv.ravel()
    vx = iv * dx
    vy = jv * dy
    if jitter > 0.0:
        vid = (jv * (n + 1) + iv).astype(np.uint64)
        ux = uniform01(seed, 2 * vid)
        uy = uniform01(seed, 2 * vid + 1)
        interior = (iv > 0) & (iv < n) & (jv > 0) & (jv < ny)
        vx = np.where(interior, vx + (2.0 * ux - 1.0) * jitter * dx, vx)
        vy = np.where(interior, vy + (2.0 * uy - 1.0) * jitter * dy, vy)
    verts = np.stack([vx, vy], axis=1)
    ic, jc = np.meshgrid(np.arange(n), np.arange(ny))
    ic, jc = ic.ravel(), jc.ravel()
    v00 = jc * (n + 1) + ic
    v10 = v00 + 1
    v01 = v00 + (n + 1)
    v11 = v01 + 1
    tri = np.empty((2 * n * ny, 3), dtype=np.int32)
    tri[0::2] = np.stack([v00, v10, v11], axis=1)
    tri[1::2] = np.stack([v00, v11, v01], axis=1)
    return TriangleMesh(vertices=verts, triangles=tri, box=(0.0, 0.0, L, Ly))


# ----------------------------------------------------------------------------
# random states and parameter draws
# ----------------------------------------------------------------------------
def random_psi(n_cells: int, M: int, seed: int, low=0.0, high=1.0) -> np.ndarray:
    """A non-negative random angular flux psi[cell][k] (float64)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(low, high, size=(n_cells, M))


def smooth_psi(mesh, M: int, seed: int) -> np.ndarray:
    """A smooth, positive angular flux: a Gaussian bump in space times a random
    positive angular profile (exercises the limiter's smooth regime)."""
    rng = np.random.default_rng(seed)
    if isinstance(mesh, CartesianMesh):
        xc, yc = mesh.centres()
        Lx, Ly = mesh.nx * mesh.dx, mesh.ny * mesh.dy
        cx, cy = mesh.x0 + 0.5 * Lx, mesh.y0 + 0.5 * Ly
        r = min(Lx, Ly) * 0.2
    else:
        xc, yc = mesh.centroids()
        x0, y0, x1, y1 = mesh.box
        cx, cy = 0.5 * (x0 + x1), 0.5 * (y0 + y1)
        r = min(x1 - x0, y1 - y0) * 0.2
    g = np.exp(-((xc - cx) ** 2 + (yc - cy) ** 2) / (2 * r * r))
    prof = rng.uniform(0.5, 1.5, size=M)
    return g[:, None] * prof[None, :]


@dataclass
class SweepInstance:
    n: int
    n_p: int
    n_phi: int
    sigma_a: float
    sigma_s: float

    @property
    def M(self) -> int:
        return self.n_p * self.n_phi


# quadrature shapes (polar x azimuthal) used for each ordinate count
QUAD_SHAPES = {64: (4, 16), 128: (8, 16), 256: (8, 32), 512: (16, 32)}


def sweep_instances(k: int, seed: int = 0, grids=(70, 140, 280, 560), Ms=(64, 128, 256),
                    sa_range=(5.0, 15.0), ss_range=(0.5, 1.5)) -> list:
    """Lattice DP-1 parameter sweep: instance i takes draws 4i..4i+3 of the
    splitmix64 stream `seed` for (grid, ordinate count, sigma_a, sigma_s)."""
    out = []
    for i in range(k):
        u = uniform01(seed, np.arange(4 * i, 4 * i + 4, dtype=np.uint64))
        n = grids[min(int(u[0] * len(grids)), len(grids) - 1)]
        M = Ms[min(int(u[1] * len(Ms)), len(Ms) - 1)]
        sa = sa_range[0] + (sa_range[1] - sa_range[0]) * u[2]
        ss = ss_range[0] + (ss_range[1] - ss_range[0]) * u[3]
        n_p, n_phi = QUAD_SHAPES[M]
        out.append(SweepInstance(n=n, n_p=n_p, n_phi=n_phi, sigma_a=float(sa), sigma_s=float(ss)))
    return out


@dataclass
class Dp2Instance:
    n: int
    n_p: int
    n_phi: int
    sigma_a: np.ndarray          # [7, 7]
    sigma_s: np.ndarray          # [7, 7]

    @property
    def M(self) -> int:
        return self.n_p * self.n_phi


def dp2_instances(k: int, seed: int = 0, grids=(70, 140, 280, 560), Ms=(64, 128, 256),
                  blue_sa=(5.0, 15.0), blue_ss=(0.0, 0.5), other_sa=(0.0, 0.5), other_ss=(0.5, 1.5)) -> list:
    """Lattice DP-2 parameter sweep (Sec. 3.1.3): instance i takes draws
    100 i .. 100 i + 99 of the splitmix64 stream `seed`: grid, ordinate count,
    then 49 absorption and 49 scattering cross-sections, block by block (i
    along x fastest). Blocks of the nominal blue set draw from the strong
    absorber ranges, all others from the scatterer ranges, so that every draw
    keeps the lattice's character while all 98 parameters vary."""
    bi, bj = np.meshgrid(np.arange(7), np.arange(7), indexing="ij")
    blue = lattice_block_material(bi, bj) == MAT_BLUE        # [i, j]
    out = []
    for t in range(k):
        u = uniform01(seed, np.arange(100 * t, 100 * t + 100, dtype=np.uint64))
        n = grids[min(int(u[0] * len(grids)), len(grids) - 1)]
        M = Ms[min(int(u[1] * len(Ms)), len(Ms) - 1)]
        ua = u[2:51].reshape(7, 7).T          # [i, j] from the order j slowest
        us = u[51:100].reshape(7, 7).T
        sa = np.where(blue, blue_sa[0] + (blue_sa[1] - blue_sa[0]) * ua, other_sa[0] + (other_sa[1] - other_sa[0]) * ua)
        ss = np.where(blue, blue_ss[0] + (blue_ss[1] - blue_ss[0]) * us, other_ss[0] + (other_ss[1] - other_ss[0]) * us)
        n_p, n_phi = QUAD_SHAPES[M]
        out.append(Dp2Instance(n=n, n_p=n_p, n_phi=n_phi, sigma_a=sa, sigma_s=ss))
    return out


def poisson_arrivals(count: int, rate: float, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate: exponential gaps
    -log(1-u)/rate from the splitmix64 stream `seed`."""
    u = uniform01(seed, np.arange(count, dtype=np.uint64))
    return np.cumsum(-np.log1p(-u) / rate)


@dataclass
class RequestSpec:
    """One solve request of the serving stream."""
    kind: str          # "lattice" (Cartesian, MUSCL, Heun) or "enclosure" (triangles, first order, Euler)
    n: int
    n_p: int
    n_phi: int
    t_end: float

    @property
    def M(self) -> int:
        return self.n_p * self.n_phi


SERVE_LATTICE_GRIDS = tuple(range(70, 701, 70))
SERVE_ENCLOSURE_GRIDS = (130, 260, 390, 520, 650)
SERVE_MS = (64, 128, 256, 512)


def serve_requests(count: int, seed: int = 0, horizon: float = 1.0, lattice_grids=SERVE_LATTICE_GRIDS,
                   enclosure_grids=SERVE_ENCLOSURE_GRIDS, Ms=SERVE_MS) -> list:
    """Mixed request stream: request i takes draws 3i..3i+2 of the splitmix64
    stream `seed` for (kind 50/50, grid, ordinate count). End times are the
    benchmarks' (lattice 3.2, enclosure 2.6) times `horizon`."""
    out = []
    for i in range(count):
        u = uniform01(seed, np.arange(3 * i, 3 * i + 3, dtype=np.uint64))
        lattice = u[0] < 0.5
        grids = lattice_grids if lattice else enclosure_grids
        n = grids[min(int(u[1] * len(grids)), len(grids) - 1)]
        M = Ms[min(int(u[2] * len(Ms)), len(Ms) - 1)]
        n_p, n_phi = QUAD_SHAPES[M]
        out.append(RequestSpec(kind="lattice" if lattice else "enclosure", n=n, n_p=n_p, n_phi=n_phi,
                               t_end=(3.2 if lattice else 2.6) * horizon))
    return out

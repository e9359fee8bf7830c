"""Plain FP64 CPU oracle for the explicit S_N time step (test infrastructure).

This package is test infrastructure, not part of the product. Only the tests,
the smoke check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py``
may import it. It shares no code with the CUDA path: it derives its own
quadrature, mesh metrics, traces, fluxes and QoIs from the paper, in float64,
with numpy, following the paper's steps in order and without blocking,
fusion or reordering:

  * Sec. 4.1, Eq. (sn_2d): S_N system on the upper hemisphere, weights summing
    to 2*pi, isotropic scattering through phi = sum_l w_l psi_l.
  * Sec. 4.2, Eq. (sn_2d_eqn_fv): cell-centred finite volumes; Eq.
    (upwind1stOrder): upwind trace; reconstruction R = psi_i + slope; ghost
    cells holding psi^- at boundary edges, boundary fluxes first order.
  * Sec. 4.3: forward Euler and Heun (SSP-RK2) with uniform dt = T / N_t.
  * Sec. 3.1 / 3.2: absorption, mass and outflow QoIs.

Pins (tests/test_oracle_*.py) tie each function to facts fixed by the paper
or by mathematics: quadrature moments, the exact discrete attenuation profile,
conservation, infinite-medium decay, scattering relaxation, the exact shift,
discrete mass balance, mirror symmetry of the lattice, convergence orders and
the paper's own printed lattice QoIs (loosely).
"""
from .quadrature import product_quadrature, gauss_legendre_01, tessellation_quadrature
from .cartesian import CartesianOracle
from .triangles import TriangleOracle
from .stepping import run, euler_step, heun_step, n_steps_for, triangle_dt

__all__ = [
    "product_quadrature", "gauss_legendre_01", "tessellation_quadrature", "CartesianOracle", "TriangleOracle",
    "run", "euler_step", "heun_step", "n_steps_for", "triangle_dt",
]

"""Time integration and QoI time integrals in FP64 (oracle, test infrastructure).

Sec. 4.3: uniform dt = T / N_t. Heun (SSP-RK2):
    psi1 = psi^n + dt F(psi^n);  psi2 = psi1 + dt F(psi1);  psi^{n+1} = (psi^n + psi2) / 2.
Forward Euler: psi^{n+1} = psi^n + dt F(psi^n) (the first-order "plain" method).

The time-integrated QoIs (Sec. 3.1 QoI-2/QoI-4, Sec. 3.2 QoI-2) use the
weights of the scheme itself, so that the discrete mass balance is an exact
identity: Euler adds dt*S(psi^n), Heun adds dt/2*(S(psi^n) + S(psi1)), where
S(psi) are the integrands (absorption per region, outflow, box outflow) at a
state.
"""
import math

import numpy as np


def n_steps_for(t_end: float, dt_target: float) -> int:
    """Number of uniform steps: ceil(T/dt_target) up to a 1e-9 tolerance."""
    return max(1, int(math.ceil(t_end / dt_target - 1e-9)))


def triangle_dt(op, t_end: float, safety: float = 0.9):
    """dt target on triangles: safety * min_i 2 A_i / P_i (first-order
    positivity bound for |omega| <= 1); returns (N_t, dt = T/N_t)."""
    n = n_steps_for(t_end, safety * op.min_2A_over_P())
    return n, t_end / n


def euler_step(op, psi, dt):
    return psi + dt * op.F(psi)


def heun_step(op, psi, dt):
    psi1 = psi + dt * op.F(psi)
    psi2 = psi1 + dt * op.F(psi1)
    return 0.5 * (psi + psi2), psi1


class Accumulators:
    def __init__(self, n_regions):
        self.abs_int = np.zeros(n_regions)
        self.outflow_int = 0.0
        self.box_out_int = None      # per QoI box, once a state with boxes is added
        self.t = 0.0
        self.step = 0

    def add(self, weight, S):
        self.abs_int += weight * S["abs"]
        self.outflow_int += weight * S["outflow"]
        if "box_out" in S:
            if self.box_out_int is None:
                self.box_out_int = np.zeros_like(S["box_out"])
            self.box_out_int += weight * S["box_out"]


def run(op, psi0, dt, n_steps, integrator="euler", acc=None):
    """Advance psi0 by n_steps of size dt; returns (psi, acc, final integrands)."""
    psi = np.array(psi0, dtype=np.float64, copy=True)
    if acc is None:
        acc = Accumulators(op.n_regions)
    for _ in range(n_steps):
        S0 = op.integrands(psi)
        if integrator == "euler":
            psi = euler_step(op, psi, dt)
            acc.add(dt, S0)
        elif integrator == "heun":
            psi, psi1 = heun_step(op, psi, dt)
            acc.add(0.5 * dt, S0)
            acc.add(0.5 * dt, op.integrands(psi1))
        else:
            raise ValueError(integrator)
        acc.step += 1
        acc.t = acc.step * dt
    return psi, acc, op.integrands(psi)

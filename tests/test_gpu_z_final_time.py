"""GPU parity to the final time T against the FP64 oracle.

The production runs take every scheme far beyond a few dozen steps (the
lattice to T = 3.2, the enclosure to T = 2.6, with uniform dt = T/N_t, Sec.
4.3), and FP32 rounding accumulates step after step. These tests advance the
CUDA path to N_t on grids where the numpy oracle finishes in one to a few
minutes, and compare the whole state with the oracle at regular checkpoints
on the way (relative L2 error of psi, every QoI):

  * the lattice (Sec. 3.1) on 140^2 cells x 8x16 = 128 ordinates, MUSCL-minmod
    fluxes with Heun, 128 steps to T = 3.2, with the QoI-1/2 squares;
  * the enclosure on the 65^2 split mesh (8450 jittered triangles) x 4x16 = 64
    ordinates, first-order upwind with Euler, 1063 steps to T = 2.6;
  * the enclosure on the 40^2 split mesh x 64 ordinates with the paper's
    second-order scheme on triangles (Green-Gauss gradient, Venkatakrishnan
    limiter, Sec. 4.2) and Heun, 627 steps to T = 2.6;

each with psi stored in FP32 (tolerances of the FP32 path: 1e-5 relative L2
on psi, 1e-4 on every QoI, at every checkpoint) and in BF16 (stochastic
rounding, FP32 arithmetic; the bounds below are the measured errors at T with
a margin). The oracle runs in worker processes started with `spawn` (they
import numpy and the oracle only), all cases at once, from the end of test
collection on, so that it overlaps the other GPU tests.
With RT_ERROR_LOG set, each case appends its error curve to that file as one
JSON line.
"""
import json
import os

import numpy as np
import pytest

import oracle
import sn_inputs as si

pytestmark = pytest.mark.gpu

PSI_TOL = 1e-5
QOI_TOL = 1e-4

# name: mesh, n, n_p, n_phi, order, integrator, checkpoint spacing in steps
CASES = {
    "lattice140_muscl_heun": ("lattice", 140, 8, 16, 2, "heun", 16),
    "enclosure65_o1_euler": ("enclosure", 65, 4, 16, 1, "euler", 128),
    "enclosure40_o2_heun": ("enclosure", 40, 4, 16, 2, "heun", 64),
}

# Cases whose FP32 check is conditioned on the scheme's own sensitivity to
# rounding. The second-order scheme on triangles (Green-Gauss gradient,
# Venkatakrishnan limiter with epsilon = A^3, Sec. 4.2) amplifies rounding-level
# differences where a discontinuity persists in void: the edges of the inflow
# beam entering through the opening of the left wall. There the limiter's
# choices flip on changes of relative size 1e-7, and the FP64 oracle itself,
# with its state rounded to FP32 after every step, ends 4.9e-3 (relative L2)
# away from the unrounded oracle at T, 99 % of it in the void next to the
# opening. No FP32 implementation can stay within 1e-5 of the FP64 trajectory
# there; the GPU is held to 1e-5 plus three times the distance between the two
# oracle trajectories (psi, and every QoI), checkpoint by checkpoint.
ROUNDING_CONDITIONED = ("enclosure40_o2_heun",)
COND_FACTOR = 3.0

# BF16 storage: bounds at every checkpoint (relative L2 of psi, largest QoI
# error relative to the QoI or 1e-3 of the mass)
BF16_PSI = {"lattice140_muscl_heun": 1.2e-2, "enclosure65_o1_euler": 8e-3, "enclosure40_o2_heun": 2.5e-2}
BF16_QOI = {"lattice140_muscl_heun": 1.2e-2, "enclosure65_o1_euler": 1.2e-3, "enclosure40_o2_heun": 6e-3}


def build_case(name):
    """Problem, oracle operator, N_t and dt of a case (the same rules as the
    library: Cartesian dt target dx/2, triangles 0.9 min 2A/P; dt = T/N_t)."""
    mesh, n, n_p, n_phi, order, integ, every = CASES[name]
    quad = oracle.product_quadrature(n_p, n_phi)
    if mesh == "lattice":
        p = si.lattice_problem(n)
        op = oracle.CartesianOracle(p, quad, order=order)
        n_t = oracle.n_steps_for(p.t_end, 0.5 * p.mesh.dx)
        dt = p.t_end / n_t
    else:
        p = si.enclosure_problem(n, jitter=0.2, seed=0)
        op = oracle.TriangleOracle(p, quad, order=order)
        n_t, dt = oracle.triangle_dt(op, p.t_end)
    return p, op, n_t, dt


def checkpoints(name, n_t):
    every = CASES[name][6]
    return sorted(set(list(range(every, n_t, every)) + [n_t]))


def oracle_job(name, round_f32=False):
    """Run the oracle of one case to N_t (in a worker process); returns the
    state, the time integrals and the integrands at every checkpoint. With
    round_f32 the state is rounded to FP32 after every step (the oracle's own
    arithmetic stays FP64): a second trajectory that differs from the first
    by rounding alone, which measures how the scheme amplifies rounding."""
    p, op, n_t, dt = build_case(name)
    integ = CASES[name][5]
    M = op.M
    psi = np.zeros((p.mesh.n_cells, M))
    acc = None
    done = 0
    out = {"n_t": n_t, "dt": dt, "steps": [], "psi": [], "acc": [], "S": []}
    for c in checkpoints(name, n_t):
        if round_f32:
            for _ in range(c - done):
                psi, acc, S = oracle.run(op, psi, dt, 1, integ, acc=acc)
                psi = psi.astype(np.float32).astype(np.float64)
            S = op.integrands(psi)
        else:
            psi, acc, S = oracle.run(op, psi, dt, c - done, integ, acc=acc)
        done = c
        out["steps"].append(c)
        out["psi"].append(psi.copy())
        out["acc"].append({"abs_int": acc.abs_int.copy(), "outflow_int": acc.outflow_int,
                           "box_out_int": None if acc.box_out_int is None else acc.box_out_int.copy()})
        out["S"].append({k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in S.items()})
    return out


_POOL = {}


def start_early():
    """Start every oracle case in spawned worker processes (one per case, one
    thread each). Called by the test session as soon as collection has
    selected a test of this file, so the oracle runs while the other GPU tests
    do; the fixture below starts it if that did not happen."""
    if _POOL:
        return
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        pool = mp.get_context("spawn").Pool(processes=len(CASES) + len(ROUNDING_CONDITIONED))
        _POOL["pool"] = pool
        _POOL["res"] = {name: pool.apply_async(oracle_job, (name,)) for name in CASES}
        for name in ROUNDING_CONDITIONED:
            _POOL["res"][name + ":f32"] = pool.apply_async(oracle_job, (name, True))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def stop_early():
    """Stop the worker processes (the session calls this when it ends)."""
    pool = _POOL.pop("pool", None)
    _POOL.clear()
    if pool is not None:
        pool.terminate()
        pool.join()


@pytest.fixture(scope="module")
def oracle_runs():
    """Results (AsyncResult) of the oracle cases."""
    start_early()
    yield _POOL["res"]
    stop_early()


@pytest.fixture(scope="module")
def rt(oracle_runs):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2505_17284_gb300 import build, rt as rtmod
    build.build()
    rtmod.load_library()
    return rtmod


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def qoi_errors(q, acc, S):
    """Largest relative error over all QoIs (relative to the QoI, or 1e-3 of
    the mass where the QoI is smaller than that)."""
    scale = abs(S["mass"])
    errs = [abs(q["mass"] - S["mass"]) / max(scale, 1e-300)]
    pairs = [(q["outflow_now"], S["outflow"]), (q["outflow_int"], acc["outflow_int"])]
    for r in range(len(S["abs"])):
        pairs += [(q["abs_now"][r], S["abs"][r]), (q["abs_int"][r], acc["abs_int"][r])]
    for b in range(len(S.get("box_out", ()))):
        pairs += [(q["box_out_now"][b], S["box_out"][b]), (q["box_out_int"][b], acc["box_out_int"][b])]
    for got, ref in pairs:
        errs.append(abs(got - ref) / max(abs(ref), 1e-3 * scale, 1e-300))
    return max(errs)


def run_to_final_time(rt, name, storage, ref):
    p, _, n_t, dt = build_case(name)
    mesh, n, n_p, n_phi, order, integ, every = CASES[name]
    quad = rt.rt_quad_product(n_p, n_phi)
    s = rt.Solver(p, quad, order=order, integrator=rt.RT_HEUN if integ == "heun" else rt.RT_EULER,
                  storage=storage, dt=0.5 * p.mesh.dx if mesh == "lattice" else 0.0)
    assert s.info.n_steps == ref["n_t"] == n_t
    assert abs(s.info.dt - ref["dt"]) <= 1e-14 * ref["dt"]
    curve = []
    done = 0
    for c, rpsi, acc, S in zip(ref["steps"], ref["psi"], ref["acc"], ref["S"]):
        s.step(c - done)
        done = c
        q = s.qoi()
        assert q["step"] == c
        curve.append({"step": c, "psi_rel_l2": rel_l2(s.psi(), rpsi), "qoi_max_rel": qoi_errors(q, acc, S),
                      # particle balance relative to the largest of its terms (the enclosure's inflow
                      # is mostly absorbed by the walls: the flows exceed the mass present by far)
                      "balance": (q["mass"] + sum(q["abs_int"]) + q["outflow_int"] - q["source_int"])
                      / max(abs(q["mass"]), sum(abs(v) for v in q["abs_int"]), abs(q["outflow_int"]),
                            abs(q["source_int"]), 1e-300)})
    s.close()
    log = os.environ.get("RT_ERROR_LOG")
    if log:
        with open(log, "a") as fh:
            fh.write(json.dumps({"case": name, "storage": "bf16" if storage else "fp32", "n_t": n_t,
                                 "curve": curve}) + "\n")
    return curve


def rounding_spread(ref, rnd):
    """Per checkpoint: distance of the FP32-rounded oracle trajectory from the
    unrounded one (relative L2 of psi, largest QoI error)."""
    out = []
    for k in range(len(ref["steps"])):
        q = {"mass": rnd["S"][k]["mass"], "outflow_now": rnd["S"][k]["outflow"],
             "outflow_int": rnd["acc"][k]["outflow_int"], "abs_now": rnd["S"][k]["abs"],
             "abs_int": rnd["acc"][k]["abs_int"], "box_out_now": rnd["S"][k].get("box_out", ()),
             "box_out_int": rnd["acc"][k]["box_out_int"]}
        out.append((rel_l2(rnd["psi"][k], ref["psi"][k]), qoi_errors(q, ref["acc"][k], ref["S"][k])))
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_matches_the_oracle_up_to_T(rt, oracle_runs, name):
    ref = oracle_runs[name].get(timeout=1800)
    curve = run_to_final_time(rt, name, rt.RT_FP32, ref)
    if name in ROUNDING_CONDITIONED:
        spread = rounding_spread(ref, oracle_runs[name + ":f32"].get(timeout=1800))
    else:
        spread = [(0.0, 0.0)] * len(curve)
    for pt, (sp, sq) in zip(curve, spread):
        assert pt["psi_rel_l2"] <= PSI_TOL + COND_FACTOR * sp, (pt, sp)
        assert pt["qoi_max_rel"] <= QOI_TOL + COND_FACTOR * sq, (pt, sq)
        assert abs(pt["balance"]) <= 1e-5, pt
    log = os.environ.get("RT_ERROR_LOG")
    if log and name in ROUNDING_CONDITIONED:
        with open(log, "a") as fh:
            fh.write(json.dumps({"case": name, "storage": "oracle_f32_rounded",
                                 "curve": [{"step": c, "psi_rel_l2": a, "qoi_max_rel": b}
                                           for c, (a, b) in zip(ref["steps"], spread)]}) + "\n")


@pytest.mark.parametrize("name", list(CASES))
def test_bf16_error_up_to_T_is_bounded(rt, oracle_runs, name):
    ref = oracle_runs[name].get(timeout=1800)
    curve = run_to_final_time(rt, name, rt.RT_BF16, ref)
    for pt in curve:
        assert pt["psi_rel_l2"] <= BF16_PSI[name], pt
        assert pt["qoi_max_rel"] <= BF16_QOI[name], pt

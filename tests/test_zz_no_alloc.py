"""rt_cart_stage_noalloc: the Cartesian stage on caller-owned buffers with its
scratch memory in the library's fixed device array (no device allocation by the
call). Its results must match the allocating path (rt_create + rt_step) within
the tolerances of the parity tests, over two calls in a row, and the FP64
oracle directly. The caller here (the test) owns every buffer; it allocates them
with PyTorch, as such a caller would with its own memory pool.

The file name makes pytest collect it after every other test file, so that a
run that stops at its first failure (-x) has run all other tests before these.
The tests do not depend on that order: each passes alone in a fresh process
and after the rest of the suite (each call clears the scratch state it uses).
"""
import math

import numpy as np
import pytest

import oracle
import sn_inputs as si

pytestmark = pytest.mark.gpu

PSI_TOL = 1e-5
QOI_TOL = 1e-4


@pytest.fixture(scope="module")
def rt():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2505_17284_gb300 import build, rt as rtmod
    build.build()
    rtmod.load_library()
    return rtmod


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


class CallerBuffers:
    """Device buffers owned by the caller: psi/phi ping-pong pairs, per-cell ids,
    the quadrature as float and the QoI/status outputs."""

    def __init__(self, problem, quad, psi0, phi0, storage=0):
        import torch
        n = problem.mesh.n_cells
        M = len(quad[0])
        self.Mpad = (M + 31) // 32 * 32
        self.storage = storage
        pad = np.zeros((n, self.Mpad), np.float32)
        pad[:, :M] = psi0
        dev = torch.device("cuda")
        dt = torch.bfloat16 if storage == 1 else torch.float32
        # psi0 holds values of the storage type already (read back from a solver), so the cast is exact
        self.psi = [torch.from_numpy(pad).to(dev).to(dt), torch.zeros((n, self.Mpad), dtype=dt, device=dev)]
        self.phi = [torch.from_numpy(phi0.astype(np.float32)).to(dev), torch.zeros(n, dtype=torch.float32, device=dev)]
        self.mat = torch.from_numpy(problem.materials.cell_mat.astype(np.uint8)).to(dev)
        self.reg = torch.from_numpy(problem.materials.cell_region.astype(np.uint8)).to(dev)
        q = np.zeros((3, self.Mpad), np.float32)
        q[0, :M], q[1, :M], q[2, :M] = quad[0], quad[1], quad[3]
        self.quad_host = q
        self.quad = torch.from_numpy(q).to(dev)
        self.qoi = torch.zeros(problem.materials.n_regions + 2, dtype=torch.float64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)

    def args(self, rt, problem, order, stage, dt, tile_y, psi_in, psi_out, phi_in, phi_out, psi_n=None, vec=2,
             step=0):
        import torch
        a = rt.rt_cart_stage_args()
        m = problem.mesh
        a.nx, a.ny, a.dx, a.dy = m.nx, m.ny, m.dx, m.dy
        a.M_pad, a.vec, a.order, a.stage, a.storage, a.tile_y = self.Mpad, vec, order, stage, self.storage, tile_y
        a.step = step
        mt = problem.materials
        a.n_mat, a.n_regions = len(mt.sigma_a), mt.n_regions
        for i in range(len(mt.sigma_a)):
            a.sigma_a[i], a.sigma_s[i], a.Q[i] = mt.sigma_a[i], mt.sigma_s[i], mt.Q[i]
        for s in range(4):
            a.inflow[s] = problem.boundary.inflow[s] if problem.boundary.kind[s] == si.INFLOW else 0.0
        a.dt = dt
        a.psi_in, a.psi_out = psi_in.data_ptr(), psi_out.data_ptr()
        a.psi_n = psi_n.data_ptr() if psi_n is not None else None
        a.phi_in, a.phi_out = phi_in.data_ptr(), phi_out.data_ptr()
        a.cell_mat, a.cell_region = self.mat.data_ptr(), self.reg.data_ptr()
        a.xi, a.eta, a.w = self.quad[0].data_ptr(), self.quad[1].data_ptr(), self.quad[2].data_ptr()
        a.qoi_out, a.status_out = self.qoi.data_ptr(), self.status.data_ptr()
        a.stream = torch.cuda.current_stream().cuda_stream
        return a

    def qoi_dict(self, n_regions, status=0):
        import torch
        torch.cuda.synchronize()
        q = self.qoi.cpu().numpy()
        assert int(self.status.cpu()[0]) == status
        return {"abs_now": q[:n_regions], "mass": q[n_regions], "outflow_now": q[n_regions + 1]}

    def host_psi(self, i, M):
        return self.psi[i].float().cpu().numpy()[:, :M].astype(np.float64)


def check_against(rt, buf, psi_dev, phi_dev, solver, n_regions, M):
    ref_psi, ref_phi, ref_q = solver.psi(), solver.phi(), solver.qoi()
    got_psi = psi_dev.cpu().numpy()[:, :M].astype(np.float64)
    got_phi = phi_dev.cpu().numpy().astype(np.float64)
    assert rel_l2(got_psi, ref_psi) <= PSI_TOL
    assert rel_l2(got_phi, ref_phi) <= PSI_TOL
    q = buf.qoi_dict(n_regions)
    scale = max(abs(ref_q["mass"]), 1e-30)
    for r in range(n_regions):
        assert abs(q["abs_now"][r] - ref_q["abs_now"][r]) <= QOI_TOL * max(abs(ref_q["abs_now"][r]), 1e-3 * scale)
    assert abs(q["mass"] - ref_q["mass"]) <= QOI_TOL * scale
    assert abs(q["outflow_now"] - ref_q["outflow_now"]) <= QOI_TOL * max(abs(ref_q["outflow_now"]), 1e-3 * scale)


@pytest.mark.parametrize("order", [1, 2])
def test_noalloc_euler_two_calls_match_rt_step(rt, order):
    """Two Euler stages in a row on caller buffers (ping-pong) against two rt_step calls."""
    p = si.lattice_problem(84)
    quad = rt.rt_quad_product(4, 16)
    dt, tile_y = 0.5 * p.mesh.dx, 24
    solver = rt.Solver(p, quad, order=order, integrator=rt.RT_EULER, dt=dt, tile_y=tile_y)
    psi0 = si.smooth_psi(p.mesh, 64, seed=12) + si.random_psi(p.mesh.n_cells, 64, seed=13) * 0.1
    solver.set_psi(psi0)
    buf = CallerBuffers(p, quad, solver.psi(), solver.phi())
    n_reg = p.materials.n_regions
    # call 1: psi[0] -> psi[1]
    rt.rt_cart_stage_noalloc(buf.args(rt, p, order, rt.RT_STAGE_EULER, solver.info.dt, tile_y,
                                      buf.psi[0], buf.psi[1], buf.phi[0], buf.phi[1]))
    solver.step(1)
    check_against(rt, buf, buf.psi[1], buf.phi[1], solver, n_reg, 64)
    # call 2: psi[1] -> psi[0]; the scratch array keeps the first call's contents
    rt.rt_cart_stage_noalloc(buf.args(rt, p, order, rt.RT_STAGE_EULER, solver.info.dt, tile_y,
                                      buf.psi[1], buf.psi[0], buf.phi[1], buf.phi[0]))
    solver.step(1)
    check_against(rt, buf, buf.psi[0], buf.phi[0], solver, n_reg, 64)
    solver.close()


def test_noalloc_heun_stages_match_rt_step(rt):
    """Heun stage 1 then stage 2 (written over psi^n) on caller buffers, with
    inflow on every side, against one Heun rt_step."""
    p = si.lattice_problem(70)
    p.boundary = si.Boundary(kind=(1, 1, 1, 1), inflow=(1.0, 0.5, 0.25, 2.0))
    quad = rt.rt_quad_product(8, 16)
    dt, tile_y = 0.5 * p.mesh.dx, 16
    solver = rt.Solver(p, quad, order=2, integrator=rt.RT_HEUN, dt=dt, tile_y=tile_y)
    psi0 = si.smooth_psi(p.mesh, 128, seed=5)
    solver.set_psi(psi0)
    buf = CallerBuffers(p, quad, solver.psi(), solver.phi())
    rt.rt_cart_stage_noalloc(buf.args(rt, p, 2, rt.RT_STAGE_HEUN1, solver.info.dt, tile_y,
                                      buf.psi[0], buf.psi[1], buf.phi[0], buf.phi[1], vec=4))
    rt.rt_cart_stage_noalloc(buf.args(rt, p, 2, rt.RT_STAGE_HEUN2, solver.info.dt, tile_y,
                                      buf.psi[1], buf.psi[0], buf.phi[1], buf.phi[0], psi_n=buf.psi[0], vec=4))
    solver.step(1)
    check_against(rt, buf, buf.psi[0], buf.phi[0], solver, p.materials.n_regions, 128)
    solver.close()


def test_noalloc_rejects_grids_beyond_the_scratch_array(rt):
    p = si.lattice_problem(84)
    quad = rt.rt_quad_product(4, 16)
    buf = CallerBuffers(p, quad, np.zeros((p.mesh.n_cells, 64)), np.zeros(p.mesh.n_cells))
    a = buf.args(rt, p, 2, rt.RT_STAGE_EULER, 0.01, 8, buf.psi[0], buf.psi[1], buf.phi[0], buf.phi[1])
    a.nx = a.ny = 3000          # 188 strips x 375 segments > RT_NOALLOC_MAX_WORK_ITEMS
    with pytest.raises(rt.RTError) as e:
        rt.rt_cart_stage_noalloc(a)
    assert e.value.code == rt.RT_EINVAL
    assert "work items" in rt.rt_last_error()


def test_noalloc_against_the_oracle(rt):
    """Two MUSCL Euler stages on caller buffers from a random state, compared
    element by element with the FP64 oracle itself (not only with rt_step)."""
    p = si.lattice_problem(70)
    n_p, n_phi, M = 4, 32, 128
    quad = rt.rt_quad_product(n_p, n_phi)
    dt = 0.5 * p.mesh.dx
    psi0 = si.random_psi(p.mesh.n_cells, M, seed=31)
    psi0 = psi0.astype(np.float32).astype(np.float64)      # the state the device starts from
    op = oracle.CartesianOracle(p, oracle.product_quadrature(n_p, n_phi), order=2)
    buf = CallerBuffers(p, quad, psi0, op.phi(psi0))
    n_reg = p.materials.n_regions
    ref = psi0
    for k, (i, o) in enumerate(((0, 1), (1, 0))):
        rt.rt_cart_stage_noalloc(buf.args(rt, p, 2, rt.RT_STAGE_EULER, dt, 16, buf.psi[i], buf.psi[o],
                                          buf.phi[i], buf.phi[o], vec=4, step=k))
        ref = oracle.euler_step(op, ref, dt)
        got = buf.host_psi(o, M)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(got - ref)) <= 2e-6 * scale
        assert rel_l2(got, ref) <= PSI_TOL
        assert rel_l2(buf.phi[o].cpu().numpy().astype(np.float64), op.phi(ref)) <= PSI_TOL
        q, S = buf.qoi_dict(n_reg), op.integrands(ref)
        for r in range(n_reg):
            assert abs(q["abs_now"][r] - S["abs"][r]) <= QOI_TOL * max(abs(S["abs"][r]), 1e-3 * S["mass"])
        assert abs(q["mass"] - S["mass"]) <= QOI_TOL * S["mass"]
        assert abs(q["outflow_now"] - S["outflow"]) <= QOI_TOL * max(abs(S["outflow"]), 1e-3 * S["mass"])


def test_noalloc_bf16_follows_the_step_index(rt):
    """BF16 storage rounds stochastically with bits drawn from (element, step,
    stage). Given the same step indices as rt_step (0, then 1), two Euler calls
    store exactly what rt_step stores with the same kernel variant and tiles."""
    p = si.lattice_problem(84)
    quad = rt.rt_quad_product(4, 16)
    dt, tile_y = 0.5 * p.mesh.dx, 24
    solver = rt.Solver(p, quad, order=2, integrator=rt.RT_EULER, storage=rt.RT_BF16, dt=dt, tile_y=tile_y,
                       variant=1, vec=2)
    info = solver.info
    assert info.variant == 1 and info.vec == 2 and info.regrouped == 0 and info.tile_y == tile_y
    solver.set_psi(si.smooth_psi(p.mesh, 64, seed=8) + 0.1 * si.random_psi(p.mesh.n_cells, 64, seed=9))
    buf = CallerBuffers(p, quad, solver.psi(), solver.phi(), storage=rt.RT_BF16)
    for k, (i, o) in enumerate(((0, 1), (1, 0))):
        rt.rt_cart_stage_noalloc(buf.args(rt, p, 2, rt.RT_STAGE_EULER, info.dt, tile_y, buf.psi[i], buf.psi[o],
                                          buf.phi[i], buf.phi[o], vec=2, step=k))
        solver.step(1)
        buf.qoi_dict(p.materials.n_regions)       # synchronises, status 0
        assert np.array_equal(buf.host_psi(o, 64), solver.psi()), k
        assert np.array_equal(buf.phi[o].cpu().numpy().astype(np.float64), solver.phi()), k
    solver.close()


def test_noalloc_reports_nonfinite_then_starts_clean(rt):
    """A call whose output overflows reports RT_ENONFINITE through status_out;
    the next call on the same buffers starts from a clean state (status 0) and
    matches rt_step."""
    p = si.lattice_problem(42)
    quad = rt.rt_quad_product(2, 16)
    dt, tile_y = 0.5 * p.mesh.dx, 16
    psi0 = si.random_psi(p.mesh.n_cells, 32, seed=41)
    solver = rt.Solver(p, quad, order=1, integrator=rt.RT_EULER, dt=dt, tile_y=tile_y)
    solver.set_psi(psi0)
    buf = CallerBuffers(p, quad, solver.psi(), solver.phi())
    n_reg = p.materials.n_regions
    bad = buf.args(rt, p, 1, rt.RT_STAGE_EULER, solver.info.dt, tile_y, buf.psi[0], buf.psi[1], buf.phi[0],
                   buf.phi[1], vec=1)
    bad.sigma_a[1] = 3.0e38        # absorbers: the absorption QoI overflows FP32
    rt.rt_cart_stage_noalloc(bad)
    buf.qoi_dict(n_reg, status=rt.RT_ENONFINITE)
    rt.rt_cart_stage_noalloc(buf.args(rt, p, 1, rt.RT_STAGE_EULER, solver.info.dt, tile_y, buf.psi[0],
                                      buf.psi[1], buf.phi[0], buf.phi[1], vec=1))
    solver.step(1)
    check_against(rt, buf, buf.psi[1], buf.phi[1], solver, n_reg, 32)
    solver.close()


def test_noalloc_checks_ordinate_groups_against_host_xi(rt):
    """With xi_host given, a vec group of ordinates that mixes signs of xi is
    rejected (RT_EINVAL) before anything is launched."""
    import ctypes
    p = si.lattice_problem(14)
    quad = rt.rt_quad_product(4, 16)
    buf = CallerBuffers(p, quad, np.zeros((p.mesh.n_cells, 64)), np.zeros(p.mesh.n_cells))
    xi = np.ascontiguousarray(buf.quad_host[0])
    a = buf.args(rt, p, 1, rt.RT_STAGE_EULER, 0.01, 8, buf.psi[0], buf.psi[1], buf.phi[0], buf.phi[1], vec=2)
    a.xi_host = xi.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    rt.rt_cart_stage_noalloc(a)          # pairs (same azimuth) share a sign: accepted
    buf.qoi_dict(p.materials.n_regions)
    shifted = np.ascontiguousarray(np.roll(xi, 1))   # pairs now straddle azimuths of opposite sign somewhere
    a.xi_host = shifted.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    with pytest.raises(rt.RTError) as e:
        rt.rt_cart_stage_noalloc(a)
    assert e.value.code == rt.RT_EINVAL
    assert "mix signs" in rt.rt_last_error()

"""Batched sweeps and the serving loop (continuous batching): each result is
the same as the problem solved alone, and small served problems match the
FP64 oracle within the parity tolerances."""
import numpy as np
import pytest

import oracle
import sn_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2505_17284_gb300 import build, rt as rtmod
    build.build()
    rtmod.load_library()
    return rtmod


def small_jobs(rt):
    from paper_2505_17284_gb300.sweep import Job
    jobs = []
    for inst in si.sweep_instances(6, seed=4, grids=(21, 28, 35), Ms=(64, 128)):
        p = si.lattice_problem(inst.n, sigma_a_blue=inst.sigma_a, sigma_s_scatter=inst.sigma_s, t_end=0.8)
        n_p, n_phi = inst.n_p, inst.n_phi
        jobs.append(Job(p, rt.rt_quad_product(n_p, n_phi), 2, rt.RT_HEUN, 0.5 * p.mesh.dx))
    return jobs


def test_sweep_batched_equals_one_at_a_time(rt):
    from paper_2505_17284_gb300 import sweep as S
    jobs = small_jobs(rt)
    qb, tb, nb = S.solve_batched(jobs)
    qp, tp, per, npl = S.solve_plain(jobs, tune=False)
    assert nb == npl
    for a, b in zip(qb, qp):
        for k in a:
            assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k
    best, times = S.tune_batch(jobs, candidates=(0, 8, 16), steps=2)
    assert best in times and all(t > 0 for t in times.values())


def test_group_tuner_configs_equal_alone_with_the_same_options(rt):
    """The per-group tuner's options (tile_y and kernel variant per group of one
    ordinate count) run in one batch, here with the variant alternated per
    problem so that chunk-uniform and per-lane groups of one ordinate count
    share the batch: each result equals the problem solved alone with the same
    options, bit for bit."""
    from paper_2505_17284_gb300 import sweep as S
    from paper_2505_17284_gb300.sweep import Job
    jobs = []
    for inst in si.sweep_instances(6, seed=11, grids=(21, 28, 35), Ms=(128, 256)):
        p = si.lattice_problem(inst.n, sigma_a_blue=inst.sigma_a, sigma_s_scatter=inst.sigma_s, t_end=0.6)
        jobs.append(Job(p, rt.rt_quad_product(inst.n_p, inst.n_phi), 2, rt.RT_HEUN, 0.5 * p.mesh.dx))
    configs, table = S.tune_groups(jobs, tile_ys=(0, 16), variants=(0, 1), steps=2)
    assert len(table) == len({S.group_key(j) for j in jobs})
    assert all(c is not None and c["variant"] in (0, 1) for c in configs)
    configs = [dict(c, variant=i % 2) for i, c in enumerate(configs)]
    qb, tb, nb = S.solve_batched(jobs, configs=configs)
    for j, c, a in zip(jobs, configs, qb):
        s = rt.Solver(j.problem, j.quad, order=j.order, integrator=j.integrator, dt=j.dt, tile_y=c["tile_y"],
                      variant=c["variant"])
        s.step()
        b = s.qoi()
        s.close()
        for k in a:
            assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), (c, k)


def test_dp2_sweep_batched_equals_one_at_a_time_and_the_oracle(rt):
    """A DP-2 sweep (49 block materials per instance) through the batched
    path: each result equals the instance solved alone, and a small one
    matches the FP64 oracle."""
    from paper_2505_17284_gb300 import sweep as S
    from paper_2505_17284_gb300.sweep import Job
    jobs = []
    for d in si.dp2_instances(5, seed=8, grids=(21, 28, 35), Ms=(64, 128)):
        p = si.lattice_dp2_problem(d.n, d.sigma_a, d.sigma_s, t_end=0.8)
        jobs.append(Job(p, rt.rt_quad_product(d.n_p, d.n_phi), 2, rt.RT_HEUN, 0.5 * p.mesh.dx))
    qb, tb, nb = S.solve_batched(jobs)
    qp, tp, per, npl = S.solve_plain(jobs, tune=False)
    assert nb == npl
    for a, b in zip(qb, qp):
        for k in a:
            assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k
    i = min(range(len(jobs)), key=lambda i: jobs[i].n_cells * jobs[i].M)
    j, d = jobs[i], si.dp2_instances(5, seed=8, grids=(21, 28, 35), Ms=(64, 128))[i]
    op = oracle.CartesianOracle(j.problem, oracle.product_quadrature(d.n_p, d.n_phi), order=2)
    n = qb[i]["n_steps"]          # N_t = ceil(T / dt_target), dt = T / N_t
    _, acc, Sn = oracle.run(op, np.zeros((j.n_cells, j.M)), qb[i]["t"] / n, n, "heun")
    assert S.qoi_rel_diff(qb[i], {"mass": Sn["mass"], "abs_int": acc.abs_int,
                                  "outflow_int": acc.outflow_int}) <= 1e-4


def stream(rt, kinds):
    from paper_2505_17284_gb300.serve import Request, estimate_bytes
    from paper_2505_17284_gb300.sweep import Job
    reqs = []
    for i, (kind, n, n_p, n_phi) in enumerate(kinds):
        q = rt.rt_quad_product(n_p, n_phi)
        if kind == "lattice":
            make = (lambda n=n, q=q: Job(si.lattice_problem(n, t_end=0.6), q, 2, rt.RT_HEUN, 0.5 * 7.0 / n))
            nb = estimate_bytes(n * n, n_p * n_phi)
        else:
            make = (lambda n=n, q=q, i=i: Job(si.enclosure_problem(n, jitter=0.2, seed=i, t_end=0.15), q, 1,
                                              rt.RT_EULER, 0.0))
            nb = estimate_bytes(2 * n * n, n_p * n_phi, triangles=True)
        reqs.append(Request(rid=i, arrival=0.01 * i, make=make, est_bytes=nb))
    return reqs


MIX = [("lattice", 21, 2, 16), ("enclosure", 8, 2, 8), ("lattice", 28, 4, 16), ("enclosure", 10, 4, 16),
       ("lattice", 14, 2, 8), ("lattice", 35, 8, 16), ("enclosure", 6, 2, 16), ("lattice", 21, 4, 16)]


@pytest.mark.parametrize("realtime,policy,fill", [(False, "fcfs_fill", 2e9), (True, "fcfs_fill", 2e9),
                                                  (True, "all", 0.0), (False, "fcfs_fill", 6e5)])
def test_served_results_equal_alone(rt, realtime, policy, fill):
    """Three slots for eight requests: later requests wait for slots, join the
    batch while others are mid-solve (or are held while older ones run, with a
    small fill), and every result is bit-identical to the request solved
    alone."""
    from paper_2505_17284_gb300 import serve as SV
    reqs = stream(rt, MIX)
    served = SV.Server(capacity=3, chunk=4, policy=policy, fill_bytes=fill).run(reqs, realtime=realtime)
    assert sorted(s.rid for s in served) == list(range(len(MIX)))
    assert max(s.admitted - s.arrival for s in served) > 0      # some request waited for a slot
    assert len({s.slot for s in served}) <= 3
    _, alone = SV.plain_service_times(reqs)
    for s in served:
        for k in s.qoi:
            assert np.array_equal(np.asarray(s.qoi[k]), np.asarray(alone[s.rid][k])), (s.rid, k)


def test_served_small_requests_match_the_oracle(rt):
    from paper_2505_17284_gb300 import serve as SV
    mix = [("lattice", 14, 2, 8), ("enclosure", 6, 2, 8)]
    reqs = stream(rt, mix)
    served = {s.rid: s for s in SV.Server(capacity=2, chunk=3).run(reqs, realtime=False)}
    for r in reqs:
        j = r.make()
        if j.order == 2:
            op = oracle.CartesianOracle(j.problem, oracle.product_quadrature(2, 8), order=2)
            n = oracle.n_steps_for(j.problem.t_end, j.dt)
            dt, integ = j.problem.t_end / n, "heun"
        else:
            op = oracle.TriangleOracle(j.problem, oracle.product_quadrature(2, 8))
            n, dt = oracle.triangle_dt(op, j.problem.t_end)
            integ = "euler"
        _, acc, S = oracle.run(op, np.zeros((j.problem.mesh.n_cells, 16)), dt, n, integ)
        q = served[r.rid].qoi
        scale = S["mass"]
        assert q["step"] == n
        assert abs(q["mass"] - S["mass"]) <= 1e-4 * scale
        for g in range(len(acc.abs_int)):
            assert abs(q["abs_int"][g] - acc.abs_int[g]) <= 1e-4 * max(abs(acc.abs_int[g]), 1e-3 * scale)
        assert abs(q["outflow_int"] - acc.outflow_int) <= 1e-4 * max(abs(acc.outflow_int), 1e-3 * scale)


def test_admission_by_memory_budget(rt):
    """A budget that fits one request at a time serialises the stream; a
    request larger than the budget is refused with an error."""
    import torch
    from paper_2505_17284_gb300 import serve as SV
    reqs = stream(rt, MIX[:4])
    free, _ = torch.cuda.mem_get_info()
    one = max(r.est_bytes for r in reqs)
    srv = SV.Server(capacity=4, chunk=4, mem_fraction=1.0, reserve=int(free) - int(1.5 * one))
    served = srv.run(reqs, realtime=False)
    assert len(served) == 4
    order = sorted(served, key=lambda s: s.admitted)
    for a, b in zip(order, order[1:]):
        assert b.admitted >= a.finished - 1e-9                 # one at a time
    big = stream(rt, MIX[:1])
    big[0].est_bytes = int(free) * 2
    with pytest.raises(RuntimeError):
        SV.Server(capacity=2).run(big, realtime=False)


def test_fcfs_fill_runs_the_oldest_first(rt):
    """With a fill smaller than any request, the scheduler advances only the
    oldest admitted request: requests finish in arrival order although later
    ones were admitted (held on the device) long before."""
    from paper_2505_17284_gb300 import serve as SV
    reqs = stream(rt, MIX[:5])
    served = SV.Server(capacity=4, chunk=4, fill_bytes=1.0).run(reqs, realtime=False)
    assert [s.rid for s in served] == [0, 1, 2, 3, 4]
    assert sum(1 for s in served if s.admitted < served[0].finished) >= 3     # held while the first ran


def test_batch_hold_pauses_a_problem(rt):
    """rt_batch_hold: a held problem does not advance; released, it finishes
    with the same result as alone."""
    pa, pb = si.lattice_problem(21, t_end=0.5), si.lattice_problem(28, t_end=0.5)
    qa, qb = rt.rt_quad_product(2, 8), rt.rt_quad_product(2, 16)
    b = rt.Batch([pa, pb], [qa, qb], order=2, integrator=rt.RT_HEUN, dts=[0.5 * pa.mesh.dx, 0.5 * pb.mesh.dx])
    b.hold(1)
    b.step(3)
    assert b.progress(0)[0] == 3 and b.progress(1)[0] == 0
    b.hold(1, False)
    b.run()
    s = rt.Solver(pb, qb, order=2, integrator=rt.RT_HEUN, dt=0.5 * pb.mesh.dx)
    s.step()
    assert np.array_equal(b.psi(1), s.psi())
    s.close()
    b.close()

"""The N > 1 path ("replicas only": one independent solve per rank, the job
timed by its slowest rank) on CPU with two gloo ranks: the max-over-ranks
reduction, the whole-job throughput, and that the reference arm works on
rank 0 only."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist
    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.replica_env()
        ms_local = 10.0 + 5.0 * r                 # rank 1 is the slow one
        ms = bench.max_over_ranks(ms_local, "cpu")
        value = bench.job_value(1000.0, w, ms)
        tdist.barrier()
        out.put((r, w, local, ms, value))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_time_by_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 and r[2] == r[0] for r in res)
    for r in res:
        assert r[3] == 15.0                        # both ranks see the slowest time
        assert abs(r[4] - 2 * 1000.0 / 15e-3) < 1e-6


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.job_value(10.0, 1, 2.0) == 5000.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert bench.run_reference(args, bench.WORKLOADS[bench.DEFAULT]) is None
    assert capsys.readouterr().out == ""

"""The sweep's per-group tuner (host logic only, no GPU): jobs are grouped by
ordinate count, order and integrator; every (tile_y, variant) pair is timed on
its group alone, invalid pairs (RT_EINVAL) are skipped, and every job of a
group gets its group's fastest pair. The step timing is replaced by a table."""
from dataclasses import dataclass

import pytest

from paper_2505_17284_gb300 import rt
from paper_2505_17284_gb300 import sweep as S


@dataclass
class FakeJob:
    M: int
    order: int = 2
    integrator: int = rt.RT_HEUN
    n_cells: int = 4900


def _fake_timer(table, calls):
    def ms_per_step(jobs, storage, steps, tile_y=0, configs=None):
        cf = configs[0]
        assert all(c == cf for c in configs)            # one pair for the whole group
        key = ({j.M for j in jobs}.pop(), cf["tile_y"], cf["variant"])
        assert len({S.group_key(j) for j in jobs}) == 1  # timed on one group alone
        calls.append((key, len(jobs)))
        return table.get(key)                            # None: invalid for some member
    return ms_per_step


def test_each_group_takes_its_fastest_pair(monkeypatch):
    jobs = [FakeJob(64), FakeJob(256), FakeJob(64), FakeJob(128), FakeJob(256), FakeJob(256)]
    table = {(64, 16, 0): 1.0, (64, 16, 1): 1.1, (64, 32, 0): 0.9, (64, 32, 1): 0.95,
             (128, 16, 0): 2.0, (128, 16, 1): 2.0, (128, 32, 0): 2.5, (128, 32, 1): 2.6,
             (256, 16, 0): 3.0, (256, 16, 1): 2.1, (256, 32, 0): None, (256, 32, 1): 2.4}
    calls = []
    monkeypatch.setattr(S, "_ms_per_step", _fake_timer(table, calls))
    configs, out = S.tune_groups(jobs, tile_ys=(16, 32), variants=(0, 1), steps=2)
    want = {64: (32, 0), 128: (16, 0), 256: (16, 1)}   # ties keep the first pair tried
    for j, c in zip(jobs, configs):
        assert (c["tile_y"], c["variant"]) == want[j.M]
    assert set(out) == {"M64_o2_heun", "M128_o2_heun", "M256_o2_heun"}
    assert "32/0" not in out["M256_o2_heun"]["ms_per_step"]   # the invalid pair is left out
    assert out["M256_o2_heun"]["best"] == {"tile_y": 16, "variant": 1}
    sizes = {key[0]: n for key, n in calls}
    assert sizes == {64: 2, 128: 1, 256: 3}
    assert len(calls) == 3 * 4


def test_order_and_integrator_split_groups(monkeypatch):
    jobs = [FakeJob(64, 2, rt.RT_HEUN), FakeJob(64, 1, rt.RT_EULER), FakeJob(64, 2, rt.RT_EULER)]
    calls = []

    def timer(sub, storage, steps, tile_y=0, configs=None):
        calls.append(tuple(S.group_key(j) for j in sub))
        return 1.0 + 0.1 * configs[0]["tile_y"]
    monkeypatch.setattr(S, "_ms_per_step", timer)
    configs, out = S.tune_groups(jobs, tile_ys=(0, 16), variants=(0,), steps=1)
    assert len(out) == 3 and all(len(set(c)) == 1 and len(c) == 1 for c in calls)
    assert all(c == {"tile_y": 0, "variant": 0} for c in configs)
    assert set(out) == {"M64_o2_heun", "M64_o1_euler", "M64_o2_euler"}


def test_a_group_with_no_valid_pair_is_an_error(monkeypatch):
    monkeypatch.setattr(S, "_ms_per_step", lambda *a, **k: None)
    with pytest.raises(ValueError):
        S.tune_groups([FakeJob(64)], tile_ys=(16,), variants=(0,), steps=1)


def test_by_shape_splits_groups_by_cell_count(monkeypatch):
    jobs = [FakeJob(256, n_cells=4900), FakeJob(256, n_cells=313600), FakeJob(256, n_cells=4900)]
    best = {4900: (16, 1), 313600: (48, 0)}

    def timer(sub, storage, steps, tile_y=0, configs=None):
        cells = {j.n_cells for j in sub}
        assert len(cells) == 1
        return 1.0 if (configs[0]["tile_y"], configs[0]["variant"]) == best[cells.pop()] else 2.0
    monkeypatch.setattr(S, "_ms_per_step", timer)
    configs, out = S.tune_groups(jobs, tile_ys=(16, 48), variants=(0, 1), steps=1, by_shape=True)
    assert [(c["tile_y"], c["variant"]) for c in configs] == [(16, 1), (48, 0), (16, 1)]
    assert set(out) == {"M256_o2_heun_cells4900", "M256_o2_heun_cells313600"}

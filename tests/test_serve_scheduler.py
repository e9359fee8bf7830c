"""The serving scheduler's choice of which admitted requests advance (host
logic only, no GPU): the oldest always runs; younger requests join it in
arrival order while the per-step state traffic stays within fill_bytes and
their remaining work fits in join_share of the oldest's; policy "all"
advances everything."""
from paper_2505_17284_gb300.serve import Request, Server


def _active(specs):
    """specs: slot -> (arrival, bytes per step, remaining steps)."""
    active, weight, remaining = {}, {}, {}
    for slot, (arr, w, rem) in specs.items():
        active[slot] = (Request(rid=slot, arrival=arr, make=None, est_bytes=0), 0.0, 0)
        weight[slot] = w
        remaining[slot] = rem
    return active, weight, remaining


def test_oldest_always_runs_even_beyond_the_fill():
    a, w, r = _active({3: (0.5, 5e9, 100), 1: (1.0, 1e6, 10)})
    assert Server(fill_bytes=2e9).select(a, w, r) == {3}


def test_small_requests_join_the_oldest():
    # oldest: 1 GB per step, 1000 steps left (1e12 bytes); two small ones fit the fill and the share
    a, w, r = _active({0: (0.0, 1e9, 1000), 1: (0.1, 1e8, 100), 2: (0.2, 2e8, 200), 3: (0.3, 5e8, 2000)})
    s = Server(fill_bytes=2e9, join_share=0.25)
    assert s.select(a, w, r) == {0, 1, 2}          # 3 has more work left than a quarter of 0's


def test_two_large_requests_do_not_share():
    a, w, r = _active({0: (0.0, 4e8, 6000), 1: (0.1, 5e8, 5000)})
    assert Server(fill_bytes=2e9, join_share=0.25).select(a, w, r) == {0}


def test_fill_limits_the_per_step_traffic():
    a, w, r = _active({0: (0.0, 1.5e9, 1000), 1: (0.1, 6e8, 1), 2: (0.2, 4e8, 1)})
    assert Server(fill_bytes=2e9, join_share=1.0).select(a, w, r) == {0, 2}


def test_policy_all_advances_everything():
    a, w, r = _active({0: (0.0, 1e9, 1000), 1: (0.1, 5e9, 5000), 2: (0.2, 1e6, 1)})
    assert Server(policy="all").select(a, w, r) == {0, 1, 2}

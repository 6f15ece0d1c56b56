"""The serving loop's admission policy on the CPU (gencd_serve_dry_run: the
same worker threads and budget as gencd_serve, each request holding its
worker for a given time instead of running on the GPU)."""

import numpy as np
import pytest


@pytest.fixture(scope="module")
def gb():
    from paper_1206_6409_gb300 import binding, build

    build.build()
    binding.lib()
    return binding


def _overlap(res):
    """Largest number of requests in flight at once."""
    ev = sorted([(r["start"], 1) for r in res] + [(r["end"], -1) for r in res], key=lambda e: (e[0], e[1]))
    cur = best = 0
    for _, d in ev:
        cur += d
        best = max(best, cur)
    return best


def test_workers_bound_the_requests_in_flight(gb):
    sizes = [(2000, 3000, 60_000)] * 9
    res = gb.gencd_serve_dry_run(sizes, [0.0] * 9, [0.05] * 9, budget_bytes=1e12, workers=3)
    assert _overlap(res) == 3
    assert max(r["worker"] for r in res) <= 2
    for r in res:
        assert r["end"] - r["start"] >= 0.05 - 1e-3 and r["start"] >= r["arrival"]
    # first come, first served: admissions in request order
    starts = [r["start"] for r in res]
    assert starts == sorted(starts)


def test_the_budget_admits_by_estimate(gb):
    # every estimate is above half the budget: two never fit together
    sizes = [(10_000, 20_000, 1_000_000)] * 5
    est = gb.gencd_serve_dry_run(sizes[:1], [0.0], [0.0], budget_bytes=1e15)[0]["bytes"]
    res = gb.gencd_serve_dry_run(sizes, [0.0] * 5, [0.03] * 5, budget_bytes=1.5 * est, workers=4)
    assert all(r["bytes"] == est for r in res)
    assert _overlap(res) == 1
    res = gb.gencd_serve_dry_run(sizes, [0.0] * 5, [0.03] * 5, budget_bytes=2.5 * est, workers=4)
    assert _overlap(res) == 2
    # a request larger than the whole budget still runs, alone
    big = gb.gencd_serve_dry_run(sizes[:3], [0.0] * 3, [0.02] * 3, budget_bytes=0.5 * est, workers=4)
    assert _overlap(big) == 1 and len(big) == 3


def test_requests_wait_for_their_arrival(gb):
    arrivals = [0.0, 0.05, 0.10, 0.15]
    res = gb.gencd_serve_dry_run([(1000, 1000, 5000)] * 4, arrivals, [0.01] * 4, budget_bytes=1e12, workers=4)
    for r, a in zip(res, arrivals):
        assert r["arrival"] == a and r["start"] >= a - 1e-4
        assert r["end"] - r["arrival"] < 0.01 + 0.05  # served soon after arriving: no queueing
    lat = np.array([r["end"] - r["arrival"] for r in res])
    assert lat.min() >= 0.01 - 1e-3


def test_bad_streams_are_rejected(gb):
    with pytest.raises(gb.GencdError):
        gb.gencd_serve_dry_run([(10, 10, 10)] * 2, [0.2, 0.1], [0.0, 0.0], budget_bytes=1e9)
    with pytest.raises(gb.GencdError):
        gb.gencd_serve_dry_run([(10, 10, 10)], [0.0], [-1.0], budget_bytes=1e9)
    with pytest.raises(gb.GencdError):
        gb.gencd_serve_dry_run([(10, 10, 10)], [0.0], [0.0], budget_bytes=0.0)

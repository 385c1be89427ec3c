"""Serving: requests of different sizes and physics share the GPU through the
continuous-batching loop; each result equals the same request run alone
(bit for bit: every request has its own handle and stream, and the step is
deterministic), admission keeps the device footprint within the budget, and
a seeded Poisson replay reports its latency percentiles."""
import numpy as np
import pytest

from paper_1912_04855_b300 import cspht
from paper_1912_04855_b300 import serve
from paper_1912_04855_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def _mix(n=6, steps=30):
    reqs = wl.serving_stream(n_requests=n, mean_gap_s=0.005, seed=7, edges=(24, 32, 40), steps=steps)
    return reqs


def test_each_result_is_the_same_alone_and_in_the_mix():
    reqs = _mix()
    srv = serve.Server(budget_bytes=1 << 34, max_active=16, chunk=7, keep_state=True)
    res = {r.id: r for r in srv.run(reqs)}
    assert len(res) == len(reqs)
    for q in reqs:
        tot, state = serve.run_alone(q)
        np.testing.assert_array_equal(res[q["id"]].state, state)
        np.testing.assert_array_equal(res[q["id"]].totals, tot)


def test_admission_keeps_within_the_budget():
    reqs = _mix(n=8, steps=20)
    fp = [cspht.device_bytes((q["edge"],) * 3, 32) for q in reqs]
    budget = 2 * max(fp)
    srv = serve.Server(budget_bytes=budget, max_active=16, chunk=5)
    res = srv.run(reqs)
    assert len(res) == len(reqs)
    assert srv.max_used <= budget
    # with room for two at a time some requests had to wait for admission
    assert max(r.admitted - r.arrival for r in res) > 0


def test_poisson_replay_metrics():
    reqs = wl.serving_stream(n_requests=10, mean_gap_s=0.01, seed=2024, edges=(32, 48), steps=20)
    srv = serve.Server(budget_bytes=1 << 33, max_active=8, chunk=10)
    srv.run(reqs)
    m = srv.metrics()
    assert m["requests"] == 10
    assert 0 < m["p50_ms"] <= m["p99_ms"]
    assert m["aggregate_gcell_s"] > 0

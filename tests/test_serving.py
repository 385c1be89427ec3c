"""Serving: requests of different sizes and physics share the GPU through the
continuous-batching loop (one captured batch graph per tick, or per-request
streams); each result equals the same request run alone (bit for bit: every
request has its own handle, and the step is deterministic), admission keeps
the device footprint within the budget, a seeded Poisson replay reports its
latency percentiles, and the batched step matches separate steps."""
import numpy as np
import pytest

from paper_1912_04855_b300 import cspht
from paper_1912_04855_b300 import serve
from paper_1912_04855_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def _mix(n=6, steps=30):
    reqs = wl.serving_stream(n_requests=n, mean_gap_s=0.005, seed=7, edges=(24, 32, 40), steps=steps)
    return reqs


@pytest.mark.parametrize("mode", ["graph", "streams", "priorities", "adaptive"])
def test_each_result_is_the_same_alone_and_in_the_mix(mode):
    reqs = _mix()
    # adaptive: room for three at a time, so that requests wait and both modes run
    srv = serve.Server(budget_bytes=1 << 34, max_active=3 if mode == "adaptive" else 16, chunk=7, keep_state=True,
                       batched=mode == "graph", priorities=mode == "priorities", adaptive=mode == "adaptive")
    # adaptive: all at once, so that a queue forms and then drains
    res = {r.id: r for r in srv.run(reqs, realtime=mode != "adaptive")}
    assert len(res) == len(reqs)
    for q in reqs:
        tot, state = serve.run_alone(q)
        np.testing.assert_array_equal(res[q["id"]].state, state)
        np.testing.assert_array_equal(res[q["id"]].totals, tot)
    if mode == "adaptive":
        assert srv.multi_ticks > 0 and srv.stream_ticks > 0


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


def test_batch_step_matches_separate_steps():
    """cspht_batch_step forks the steps of handles of different sizes from one
    stream and joins them back; called directly and replayed from a captured
    two-step graph, it gives the same bits as each handle stepping alone, and
    every handle keeps its own dt."""
    import torch
    ws = [wl.potential_well(n=24, mach=2.0), wl.shock_tube(nx=40, ny=8, nz=6), wl.blast(n=16, radius_cells=2.0)]
    streams = [torch.cuda.Stream() for _ in ws]
    bs = torch.cuda.Stream()

    def make():
        out = []
        for w, st in zip(ws, streams):
            s = cspht.Sim.from_workload(w, precision=32)
            s.set_stream(st)
            s.set_primitive(np.ascontiguousarray(w.W))
            out.append(s)
        return out

    alone, batched = make(), make()
    for s in alone:
        s.advance(9, 0.4)
        s.sync()
    for s in batched:
        s.advance(2, 0.4)
    cspht.batch_step(batched, 0.4, bs)  # 3 steps
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(bs):
        g.capture_begin(capture_error_mode="thread_local")
        try:
            for _ in range(2):
                cspht.batch_step(batched, 0.4, bs)
        finally:
            g.capture_end()  # capture runs nothing: still 3 steps
        for _ in range(3):
            g.replay()  # 9 steps
    bs.synchronize()
    for a, b in zip(alone, batched):
        b.sync()
        np.testing.assert_array_equal(b.get_state(), a.get_state())
        assert b.time() == a.time()
    assert len({s.time() for s in batched}) == len(batched)  # own dt per handle
    for s in alone + batched:
        s.close()

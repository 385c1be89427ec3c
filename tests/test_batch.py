"""Many grids in one launch per step kernel (cspht_batch_*): every member's
result is bit for bit the one it gets stepped alone, whatever the mix of
sizes, boundaries and step counts, and the batch picks up members stepped on
their own in between.  Stepping alone is itself checked against the FP64
oracle by the parity tests."""
import numpy as np
import pytest

from paper_1912_04855_b300 import cspht
from paper_1912_04855_b300 import workloads as wl

pytestmark = pytest.mark.gpu
P_, O_, I_ = wl.PERIODIC, wl.OUTFLOW, wl.INFLOW


def _members():
    return [
        wl.potential_well(n=40, ny=24, nz=20, mach=2.0),                    # inflow/outflow x, ragged tiles
        wl.shock_tube(nx=64, ny=16, nz=12),
        wl.random_state((9, 13, 50), seed=3, psi_amp=0.2, bc=[O_, O_, P_, P_, O_, O_]),
        wl.developed_well(n=48),
        wl.potential_well(n=16, mach=1.5),
    ]


def _alone(w, prec, steps, cfl=0.4):
    with cspht.Sim.from_workload(w, precision=prec) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        s.advance(steps, cfl)
        s.sync()
        return s.get_state(), s.time()


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("depth", [0, 7])
def test_batch_matches_members_alone(prec, depth):
    import torch
    ws = _members()
    stream = torch.cuda.Stream()
    sims = [cspht.Sim.from_workload(w, precision=prec) for w in ws]
    try:
        for s, w in zip(sims, ws):
            s.set_primitive(np.ascontiguousarray(w.W))
        with cspht.Batch(sims, depth=depth) as b:
            b.advance(5, 0.4, stream)   # graph replays and one single step
            b.advance(4, 0.4, stream)
            stream.synchronize()
            assert b.launch_count() >= 9 * 5
        for s, w in zip(sims, ws):
            s.sync()
            U, t = s.get_state(), s.time()
            Ua, ta = _alone(w, prec, 9)
            assert np.array_equal(U, Ua) and t == ta, w.name
    finally:
        for s in sims:
            s.close()


def test_batch_picks_up_members_stepped_alone():
    import torch
    ws = _members()[:3]
    stream = torch.cuda.Stream()
    sims = [cspht.Sim.from_workload(w, precision=32) for w in ws]
    try:
        for s, w in zip(sims, ws):
            s.set_primitive(np.ascontiguousarray(w.W))
        with cspht.Batch(sims) as b:
            b.advance(2, 0.4, stream)
            sims[1].advance(1, 0.4)     # one member steps on its own: its buffers flip
            b.advance(3, 0.4, stream)
            stream.synchronize()
        steps = [5, 6, 5]
        for s, w, n in zip(sims, ws, steps):
            s.sync()
            Ua, ta = _alone(w, 32, n)
            assert np.array_equal(s.get_state(), Ua) and s.time() == ta
    finally:
        for s in sims:
            s.close()


def test_batch_rejects_mixed_or_unsupported_members():
    wa = wl.potential_well(n=16)
    wb = wl.random_state((8, 8, 8), seed=1, bc=[P_, P_, wl.WALL, wl.WALL, P_, P_])  # walls in y: no one-pass shell
    with cspht.Sim.from_workload(wa, precision=32) as a, cspht.Sim.from_workload(wa, precision=64) as c, \
            cspht.Sim.from_workload(wb, precision=32) as d, cspht.Sim.from_workload(wa, precision=32) as e:
        for s, w in ((a, wa), (c, wa), (d, wb)):
            s.set_primitive(np.ascontiguousarray(w.W))
        for bad in ([a, c], [a, d], [a, a]):
            with pytest.raises(cspht.CsphtError) as ex:
                cspht.Batch(bad)
            assert ex.value.code == cspht.EINVAL
        with pytest.raises(cspht.CsphtError) as ex:
            cspht.Batch([a, e])  # e has no state
        assert ex.value.code == cspht.ESTATE

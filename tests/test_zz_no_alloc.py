"""The step entry point that allocates no device memory.

Callers that cannot call cudaMalloc (an application whose memory pool owns
the GPU, or a time-critical loop that cannot accept an allocation's
device-wide synchronisation) use cspht_step_noalloc_f32 on buffers they own.
These tests call it through the C ABI and check its result against the
allocating entry point (a single-precision handle on the fused path) on two
calls in a row, within the FP32 tolerance the parity tests use for one
step.  The file is named to run last.
"""
import numpy as np
import pytest

from paper_1912_04855_b300 import cspht
from paper_1912_04855_b300 import workloads as wl

pytestmark = pytest.mark.gpu
P_, O_, I_, W_ = wl.PERIODIC, wl.OUTFLOW, wl.INFLOW, wl.WALL


def _reference(w, U0, cfl, steps):
    """States and dts of the allocating FP32 fast path, one step at a time."""
    out = []
    with cspht.Sim.from_workload(w, precision=32, path=cspht.PATH_FAST) as s:
        s.set_state(U0)
        for _ in range(steps):
            dt = s.step(cfl)
            out.append((s.get_state(), dt))
    return out


def _rounded_state(w):
    """The workload's initial state as the FP32 handle holds it (float-rounded)."""
    with cspht.Sim.from_workload(w, precision=32) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        return s.get_state()


@pytest.mark.parametrize("make", [
    lambda: wl.potential_well(n=40, ny=24, nz=20, mach=2.0),  # inflow/outflow x, ragged tiles
    lambda: wl.hydrostatic(n=24, nxy=12, perturb=1e-6),        # wall + outflow z, vacuum
    lambda: wl.random_state((11, 13, 17), seed=4, psi_amp=0.1, bc=[W_, O_, P_, P_, I_, O_]),
], ids=["well", "hydrostatic", "mixed"])
def test_noalloc_matches_allocating_step_twice(make):
    import torch
    w = make()
    cfl = 0.4
    U0 = _rounded_state(w)
    ref = _reference(w, U0, cfl, 2)
    dev = torch.device("cuda", 0)
    U = torch.tensor(U0, dtype=torch.float32, device=dev)
    psi = torch.tensor(w.psi, dtype=torch.float32, device=dev)
    for step in range(2):
        out = torch.empty_like(U)
        dt = cspht.step_noalloc_f32(w.shape, w.h, w.gamma, U, psi, out, cfl=cfl, bc=w.bc,
                                    inflow=w.inflow)
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        R, dt_ref = ref[step]
        assert dt == pytest.approx(dt_ref, rel=1e-6)
        for f in range(5):
            scale = max(np.abs(R[1:4]).max(), 1e-30) if 1 <= f <= 3 else np.abs(R[f]).max()
            assert np.abs(got[f] - R[f]).max() <= 1e-5 * scale, (step, f)
        U = out


def _check_twice(w, U, psi, cfl=0.4):
    """Two no-allocation steps from the device state U against the allocating path."""
    import torch
    ref = _reference(w, U.double().cpu().numpy(), cfl, 2)
    for step in range(2):
        out = torch.empty_like(U)
        dt = cspht.step_noalloc_f32(w.shape, w.h, w.gamma, U, psi, out, cfl=cfl, bc=w.bc,
                                    inflow=w.inflow)
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        R, dt_ref = ref[step]
        assert dt == pytest.approx(dt_ref, rel=1e-6)
        for f in range(5):
            scale = max(np.abs(R[1:4]).max(), 1e-30) if 1 <= f <= 3 else np.abs(R[f]).max()
            assert np.abs(got[f] - R[f]).max() <= 1e-5 * scale, (step, f)
        U = out


# The largest grid whose 21 padded FP32 fields fit the 64 MiB array: 86 x 86
# cells in the plane and 88 planes (one more plane is refused).  The last
# field then ends within 0.6 % of the array's end, where an access past a
# field's end would first show.
LARGEST = (88, 86, 86)  # (nz, ny, nx)


def test_noalloc_at_the_largest_accepted_grid():
    import torch
    dev = torch.device("cuda", 0)
    nz, ny, nx = LARGEST
    w = wl.potential_well(n=nx, ny=ny, nz=nz, mach=2.0)
    U = torch.tensor(_rounded_state(w), dtype=torch.float32, device=dev)
    psi = torch.tensor(w.psi, dtype=torch.float32, device=dev)
    _check_twice(w, U, psi)
    bigger = (nz + 1, ny, nx)
    Ub = torch.zeros((5,) + bigger, dtype=torch.float32, device=dev)
    with pytest.raises(cspht.CsphtError) as e:
        cspht.step_noalloc_f32(bigger, 1 / nx, 1.4, Ub, torch.zeros(bigger, device=dev), torch.empty_like(Ub))
    assert e.value.code == cspht.ETOOBIG


def test_noalloc_after_a_failed_call_left_nan_in_the_scratch():
    # A call on a large grid whose potential is NaN everywhere fills every
    # field of the shared array that it uses with NaN and reports a
    # non-finite state.  A following call on a smaller grid, whose padded
    # fields sit at other offsets of the same array, must not see any of it.
    import torch
    dev = torch.device("cuda", 0)
    nz, ny, nx = LARGEST
    big = wl.potential_well(n=nx, ny=ny, nz=nz, mach=2.0)
    Ub = torch.tensor(_rounded_state(big), dtype=torch.float32, device=dev)
    nan_psi = torch.full(big.shape, float("nan"), dtype=torch.float32, device=dev)
    with pytest.raises(cspht.CsphtError) as e:
        cspht.step_noalloc_f32(big.shape, big.h, big.gamma, Ub, nan_psi, torch.empty_like(Ub),
                               bc=big.bc, inflow=big.inflow)
    assert e.value.code == cspht.ENONFINITE
    w = wl.random_state((11, 13, 17), seed=4, psi_amp=0.1, bc=[W_, O_, P_, P_, I_, O_])
    U = torch.tensor(_rounded_state(w), dtype=torch.float32, device=dev)
    psi = torch.tensor(w.psi, dtype=torch.float32, device=dev)
    _check_twice(w, U, psi)


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    shape = (96, 96, 96)  # 21 padded FP32 fields of 96^3 exceed the 64 MiB scratch
    dev = torch.device("cuda", 0)
    U = torch.zeros((5,) + shape, dtype=torch.float32, device=dev)
    psi = torch.zeros(shape, dtype=torch.float32, device=dev)
    with pytest.raises(cspht.CsphtError) as e:
        cspht.step_noalloc_f32(shape, 1 / 96, 1.4, U, psi, torch.empty_like(U))
    assert e.value.code == cspht.ETOOBIG

"""Full-size GPU checks, in the launch configuration the benchmark times.

- The benchmark workload (supersonic flow through a potential well, 256^3,
  FP32, fused path): one GPU step from a developed state is compared with the
  FP64 oracle on sampled windows (the oracle's windowed step computes only
  those cells), and dt with the oracle's CFL rule.
- The hydrostatic atmosphere at 128^3 (500 steps): FP64 well-balancing below
  the descending rarefaction, FP32 against FP64, and FP32 total-mass drift in
  closed and periodic boxes; the gas-vacuum front after 40 steps against the
  oracle's column and the free-expansion bound, and the whole FP64 grid
  against the oracle's column after 100 steps (1e-10).
- The benchmark workload run as configured (1000 steps): FP32 against FP64.
- The point blast at 512^3 (FP32): one step after 200 on sampled windows
  (centre, front, far field) against the oracle.

Tolerances: a single FP32 step from an FP64-exact input carries the rounding
of a few hundred FP32 operations per cell, each at most 2^-24 relative, on
terms of the size of the local state; 1e-5 of the field's scale bounds it
with room.  FP32 multi-step runs use the relative L1 bound of 1e-4 per field
and the mass-drift bound of 1e-10 (FP64 sums).
"""
import math

import numpy as np
import pytest

from paper_1912_04855_b300 import cspht
from paper_1912_04855_b300 import workloads as wl

pytestmark = pytest.mark.gpu
P_, O_, I_, W_ = wl.PERIODIC, wl.OUTFLOW, wl.INFLOW, wl.WALL


def _windows(n):
    e = 8
    return [
        ((0, e), (0, e), (0, e)),                  # inflow face, periodic y/z seams
        ((n - e, n), (n - e, n), (n - e, n)),      # outflow face, the other seams
        ((n // 2 - e // 2, n // 2 + e // 2),) * 3,  # the centre of the well
        ((n // 4, n // 4 + e), (0, e), (n - e, n)),
        ((n // 2 + 20, n // 2 + 20 + e), (n // 2 - 3, n // 2 - 3 + e), (n // 2 - 30, n // 2 - 30 + e)),
    ]


def test_bench_workload_one_step_on_sampled_windows(orc):
    n = 256
    w = wl.potential_well(n=n)
    with cspht.Sim.from_workload(w, precision=32, path=cspht.PATH_FAST) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        s.advance(20, w.cfl)
        s.sync()
        U0 = s.get_state()
        dt = s.step(w.cfl)
        U1 = s.get_state()
    P = orc.Problem(w.shape, w.h, w.gamma, w.bc, inflow=w.inflow)
    assert dt == pytest.approx(P.dt(U0, w.cfl), rel=2e-6)
    assert np.isfinite(U1).all()
    mscale = np.abs(U0[1:4]).max()
    for i, box in enumerate(_windows(n)):
        Uo = P.step(w.psi, U0, dt, box=box)
        sl = (slice(*box[2]), slice(*box[1]), slice(*box[0]))
        for f in range(5):
            scale = mscale if 1 <= f <= 3 else np.abs(U0[f]).max()
            err = np.abs(U1[f][sl] - Uo[f][sl]).max() / scale
            assert err <= 1e-5, (box, f, err)
        if i == 2:  # in the well the step changes the state: the comparison is not trivial
            assert np.abs(Uo[4][sl] - U0[4][sl]).max() > 1e-3 * np.abs(U0[4][sl]).max()


def _umax_below_rarefaction(U, w, steps, t):
    rho = U[0]
    with np.errstate(invalid="ignore", divide="ignore"):
        u = np.where(rho > 1e-10, np.abs(U[1:4]) / np.where(rho > 1e-10, rho, 1.0), 0.0)
    z = (np.arange(w.shape[0]) + 0.5) * w.h
    c = math.sqrt(w.gamma * 0.2)
    below = z < 0.8 - c * t - 3.0 * math.sqrt(steps) * w.h
    assert below.sum() >= w.shape[0] // 4
    return u[:, below].max()


def test_hydrostatic_128_fp64_well_balanced():
    """C2's layout (wall below, vacuum above z = 0.8, outflow on top) on the
    discrete equilibrium without the perturbation: the gas below the
    rarefaction stays at rest to rounding."""
    w = wl.hydrostatic(n=128, perturb=0.0)
    steps = 200
    with cspht.Sim.from_workload(w, precision=64, path=cspht.PATH_FAST) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        s.advance(steps, w.cfl)
        s.sync()
        U = s.get_state()
        t = s.time()
    assert _umax_below_rarefaction(U, w, steps, t) <= 1e-12


def test_hydrostatic_128_fp32_against_fp64():
    """C2 as configured (1e-6 perturbation, 500 steps; by then the rarefaction
    from the vacuum interface fills the column): FP32 fused vs FP64 fused,
    relative L1 <= 1e-4 for every field."""
    w = wl.hydrostatic(n=128, perturb=1e-6)
    steps = 500
    out = {}
    for prec in (64, 32):
        with cspht.Sim.from_workload(w, precision=prec, path=cspht.PATH_FAST) as s:
            s.set_primitive(np.ascontiguousarray(w.W))
            s.advance(steps, w.cfl)
            s.sync()
            out[prec] = (s.get_state(), s.time())
    U64, t64 = out[64]
    U32, t32 = out[32]
    assert t32 == pytest.approx(t64, rel=1e-4)
    msum = np.abs(U64[1:4]).sum()  # momentum components share one scale (the flow is vertical)
    for f in range(5):
        denom = msum if 1 <= f <= 3 else np.abs(U64[f]).sum()
        l1 = np.abs(U32[f] - U64[f]).sum() / denom
        assert l1 <= 1e-4, (f, l1)


@pytest.mark.parametrize("make", [
    lambda: wl.hydrostatic(n=128, perturb=1e-6, z_vac=2.0, top_bc=W_),       # closed, in gravity
    lambda: wl.random_state((96, 96, 96), seed=17, vel=0.3, psi_amp=0.05),   # periodic
], ids=["closed_atmosphere_128", "periodic_random_96"])
def test_fp32_total_mass_drift(make):
    """FP32 state with FP64 totals: total mass drifts by <= 1e-10 relative over
    500 steps when no mass crosses the boundary."""
    w = make()
    with cspht.Sim.from_workload(w, precision=32, path=cspht.PATH_FAST) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        m0 = s.totals()[0]
        s.advance(500, w.cfl)
        s.sync()
        m1 = s.totals()[0]
    assert abs(m1 - m0) <= 1e-10 * abs(m0), (m0, m1, (m1 - m0) / m0)


def test_hydrostatic_128_gas_vacuum_front(orc):
    """C2's gas-vacuum interface at full size.  Without the perturbation the
    atmosphere is horizontally uniform, so every column of the 128^3 grid
    evolves like the oracle's 2 x 2 x 128 column.  After 40 steps the front
    (highest cell with rho > 1e-10) is the oracle's, lies below the
    free-expansion bound 0.8 + 2c/(gamma-1) t - g t^2/2 of a gas edge released
    into vacuum (c = sqrt(gamma p/rho) of the isothermal gas), and has covered
    at least half of that distance; FP32 puts the 1e-6 level of the front
    within one cell of FP64's.  After 100 steps the FP64 grid matches the
    oracle to 1e-10 of each field's scale in every cell, and its columns
    agree with each other."""
    w = wl.hydrostatic(n=128, perturb=0.0)
    wc = wl.hydrostatic(n=128, nxy=2, perturb=0.0)
    P = orc.Problem(wc.shape, wc.h, wc.gamma, wc.bc, inflow=wc.inflow)
    z = (np.arange(128) + 0.5) * w.h

    def front(rho, th):
        return z[np.where(rho > th)[0].max()] + 0.5 * w.h

    def against_oracle(U, Uo):
        col = U[:, :, :1, :1]
        msc = max(np.abs(Uo[1:4]).max(), 1e-300)
        for f in range(5):
            assert np.abs(U[f] - col[f]).max() <= 1e-15 * max(np.abs(U[f]).max(), 1e-300), f
            scale = msc if 1 <= f <= 3 else np.abs(Uo[f]).max()
            assert np.abs(U[f] - np.tile(Uo[f], (1, 64, 64))).max() <= 1e-10 * scale, f

    out = {}
    with cspht.Sim.from_workload(w, precision=64, path=cspht.PATH_FAST) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        s.advance(40, w.cfl)
        s.sync()
        U40, t = s.get_state(), s.time()
        Uo40, to, so, rc = P.run(wc.psi, P.prim_to_cons(wc.W), nsteps=40)
        assert rc == 0 and t == pytest.approx(to, rel=1e-12)
        against_oracle(U40, Uo40)
        zf = front(U40[0, :, 0, 0], 1e-10)
        assert zf == front(Uo40[0, :, 0, 0], 1e-10)
        ue = 2.0 * math.sqrt(w.gamma * 0.2) / (w.gamma - 1.0)
        bound = 0.8 + ue * t - 0.5 * t * t
        assert 0.8 + 0.5 * (bound - 0.8) <= zf <= bound, (zf, bound)
        s.advance(60, w.cfl)
        s.sync()
        U100, t100 = s.get_state(), s.time()
        Uo100, to100, _, rc = P.run(wc.psi, Uo40, nsteps=60, t0=to)
        assert rc == 0 and t100 == pytest.approx(to100, rel=1e-12)
        against_oracle(U100, Uo100)
    with cspht.Sim.from_workload(w, precision=32, path=cspht.PATH_FAST) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        s.advance(40, w.cfl)
        s.sync()
        U32 = s.get_state()
    assert abs(front(U32[0, :, 0, 0], 1e-6) - front(U40[0, :, 0, 0], 1e-6)) <= w.h


def test_potential_well_256_fp32_against_fp64_1000_steps():
    """C3 as configured: 256^3, 1000 steps, FP32 fused against FP64 fused.
    The flow is a smooth compression in the well (density up to about 2.3),
    so the FP32 criterion is the smooth-run one: relative L1 <= 3e-4 per field
    (momentum components share one scale, the flow being along x), and the
    density maximum on the centre line at the same cell within one cell and
    the same value within 3e-3 (measured 1.0e-3: a pointwise peak carries
    the FP32 rounding amplified by the compression, the field's relative
    L-infinity difference being about 1e-2)."""
    w = wl.potential_well(n=256)
    out = {}
    for prec in (64, 32):
        with cspht.Sim.from_workload(w, precision=prec, path=cspht.PATH_FAST) as s:
            s.set_primitive(np.ascontiguousarray(w.W))
            s.advance(1000, w.cfl)
            s.sync()
            out[prec] = (s.get_state(), s.time())
    U64, t64 = out[64]
    U32, t32 = out[32]
    assert t32 == pytest.approx(t64, rel=1e-4)
    msum = np.abs(U64[1:4]).sum()
    for f in range(5):
        denom = msum if 1 <= f <= 3 else np.abs(U64[f]).sum()
        l1 = np.abs(U32[f] - U64[f]).sum() / denom
        assert l1 <= 3e-4, (f, l1)
    m = 128
    l64, l32 = U64[0, m, m, :], U32[0, m, m, :]
    assert abs(int(np.argmax(l32)) - int(np.argmax(l64))) <= 1
    assert l32.max() == pytest.approx(l64.max(), rel=3e-3)
    assert l64.max() > 1.5  # the comparison sees the compression, not the inflow state


def test_blast_512_one_step_on_sampled_windows(orc):
    """C4 at full size (512^3, FP32 fused): after 200 steps the blast has a
    hot core and a sharp front; one more GPU step is compared with the FP64
    oracle's step on windows at the centre, across the front along two axes
    and a diagonal, and in the undisturbed gas (1e-5 of each field's scale,
    as for the benchmark workload)."""
    n = 512
    w = wl.blast(n=n)
    with cspht.Sim.from_workload(w, precision=32, path=cspht.PATH_FAST) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        s.advance(200, 0.4)
        s.sync()
        U0 = s.get_state()
        dt = s.step(0.4)
        U1 = s.get_state()
    P = orc.Problem(w.shape, w.h, w.gamma, w.bc, inflow=w.inflow)
    assert dt == pytest.approx(P.dt(U0, 0.4), rel=2e-6)
    m = n // 2
    line = U0[0, m, m, m:]
    r = int(np.argmax(line))  # front: the density peak on the +x half-axis
    assert 3 < r < m - 8
    e = 8
    d = int(r / math.sqrt(3.0))
    boxes = [((m - 4, m + 4),) * 3,
             ((m + r - 4, m + r + 4), (m - 4, m + 4), (m - 4, m + 4)),
             ((m - 4, m + 4), (m - r - 4, m - r + 4), (m - 4, m + 4)),
             ((m + d - 4, m + d + 4),) * 3,
             ((0, e), (0, e), (0, e))]
    msc = np.abs(U0[1:4]).max()
    for box in boxes:
        Uo = P.step(w.psi, U0, dt, box=box)
        sl = (slice(*box[2]), slice(*box[1]), slice(*box[0]))
        for f in range(5):
            scale = msc if 1 <= f <= 3 else np.abs(U0[f]).max()
            err = np.abs(U1[f][sl] - Uo[f][sl]).max() / scale
            assert err <= 1e-5, (box, f, err)

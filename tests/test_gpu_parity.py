"""GPU parity: the CUDA step (through the C ABI) against the FP64 CPU oracle.

FP64 handles must match the oracle within 1e-10 relative L-infinity per
conserved field after up to 100 steps (or 200 for the full-size Sod tube);
FP32 handles within the single-precision tolerances stated per test.
Both sides start from the same seeded primitive arrays and convert them to
conserved form on their own; each computes its own time steps.
"""
import math

import numpy as np
import pytest

from paper_1912_04855_b300 import cspht
from paper_1912_04855_b300 import workloads as wl

pytestmark = pytest.mark.gpu
P_, O_, I_, W_ = wl.PERIODIC, wl.OUTFLOW, wl.INFLOW, wl.WALL
PATHS = [cspht.PATH_PLAIN, cspht.PATH_FAST]


def oracle_problem(orc, w, **kw):
    return orc.Problem(w.shape, w.h, w.gamma, w.bc, inflow=w.inflow, **kw)


def rel_linf(a, b):
    """max|a-b| / scale per field; momenta share one scale (their largest)."""
    out = []
    mscale = max(np.abs(b[1:4]).max(), 1e-300)
    for f in range(5):
        scale = mscale if 1 <= f <= 3 else max(np.abs(b[f]).max(), 1e-300)
        out.append(float(np.abs(a[f] - b[f]).max() / scale))
    return out


def gpu_run(w, steps, cfl=0.4, **opts):
    with cspht.Sim.from_workload(w, **opts) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        s.advance(steps, cfl)
        s.sync()
        U = s.get_state()
        t = s.time()
        tot = s.totals()
    return U, t, tot


def oracle_run(orc, w, steps, cfl=0.4, **kw):
    P = oracle_problem(orc, w, **kw)
    U, t, s, rc = P.run(w.psi, P.prim_to_cons(w.W), nsteps=steps, cfl=cfl)
    assert rc == 0 and s == steps
    return U, t, P


CASES = {
    "sod_ragged": (lambda: wl.shock_tube(nx=40, ny=6, nz=5), 100),
    "random_periodic_psi": (lambda: wl.random_state((18, 20, 24), seed=1, psi_amp=0.2, vel=0.2), 40),
    "well_inflow": (lambda: wl.potential_well(n=32, ny=12, nz=10, mach=2.0), 100),
    "hydrostatic_wall_vacuum": (lambda: wl.hydrostatic(n=40, nxy=6, perturb=1e-6), 100),
    "blast": (lambda: wl.blast(n=16, radius_cells=2.0), 30),
    "walls_random": (lambda: wl.random_state((9, 10, 12), seed=5, bc=[W_] * 6, psi_amp=0.1), 40),
    "mixed_faces": (lambda: wl.random_state((10, 11, 13), seed=8, bc=[I_, O_, W_, O_, P_, P_],
                                            psi_amp=0.1), 40),
    "vacuum_tube": (lambda: wl.vacuum_tube(nx=120, ny=3, nz=2), 100),
    # x walls with copy-rule y and z faces: the one-pass ghost shell, whose edge
    # and corner ghosts compose the wall rule with the outflow and periodic copies
    "walls_x_shell": (lambda: wl.random_state((11, 13, 20), seed=23, bc=[W_, W_, O_, O_, P_, P_],
                                              psi_amp=0.2, vel=0.3), 40),
    # ragged widths whose x ghosts fall on the FP32 tile's twice-stored
    # columns (16, 17 of the predictor region) and on a second tile
    "walls_x_nx16": (lambda: wl.random_state((9, 10, 16), seed=31, bc=[W_, W_, P_, P_, O_, O_],
                                             psi_amp=0.2, vel=0.3), 40),
    "walls_xy_nx17": (lambda: wl.random_state((8, 11, 17), seed=32, bc=[W_, W_, W_, W_, P_, P_],
                                              psi_amp=0.2, vel=0.3), 40),
    "inflow_x_nx48": (lambda: wl.random_state((6, 9, 48), seed=33, bc=[I_, O_, W_, O_, P_, P_],
                                              psi_amp=0.1, vel=0.3), 40),
}


def rel_l1(a, b):
    """sum|a-b| / sum|b| per field; momenta share one scale (their largest)."""
    out = []
    mscale = max(np.abs(b[1:4]).sum(axis=(1, 2, 3)).max(), 1e-300)
    for f in range(5):
        scale = mscale if 1 <= f <= 3 else max(np.abs(b[f]).sum(), 1e-300)
        out.append(float(np.abs(a[f] - b[f]).sum() / scale))
    return out


@pytest.mark.parametrize("path", PATHS, ids=["plain", "fast"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_fp64_matches_oracle(orc, case, path):
    make, steps = CASES[case]
    w = make()
    Ug, tg, totg = gpu_run(w, steps, precision=64, path=path)
    Uo, to, P = oracle_run(orc, w, steps)
    err = rel_linf(Ug, Uo)
    assert max(err) <= 1e-10, err
    assert tg == pytest.approx(to, rel=1e-12)
    np.testing.assert_allclose(totg, P.totals(w.psi, Uo), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("path", PATHS, ids=["plain", "fast"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_fp32_matches_oracle_on_every_boundary_case(orc, case, path):
    """Every boundary kind and ragged width in FP32 against the FP64 oracle:
    relative L1 within 1e-4 per conserved field (the single-precision bound
    for smooth and equilibrium runs; measured at most 1e-5, at the gas-vacuum
    front of the hydrostatic case, and 2e-6 elsewhere), relative L-infinity
    within 1e-3 (measured at most 8e-5, the same front, where phi = sqrt(2p)
    loses relative precision as p -> 0), the elapsed time within 1e-5."""
    make, steps = CASES[case]
    w = make()
    Ug, tg, _ = gpu_run(w, steps, precision=32, path=path)
    Uo, to, _ = oracle_run(orc, w, steps)
    assert max(rel_l1(Ug, Uo)) <= 1e-4
    assert max(rel_linf(Ug, Uo)) <= 1e-3
    assert tg == pytest.approx(to, rel=1e-5)


@pytest.mark.parametrize("variant", [dict(limiter=1), dict(limiter=2), dict(riemann=1),
                                     dict(limiter=2, riemann=1), dict(riemann=2),
                                     dict(limiter=1, riemann=2), dict(riemann=3)])
@pytest.mark.parametrize("path", PATHS, ids=["plain", "fast"])
def test_fp64_options_match_oracle(orc, variant, path):
    w = wl.random_state((12, 14, 16), seed=2, psi_amp=0.1, bc=[I_, O_, P_, P_, W_, O_])
    Ug, tg, _ = gpu_run(w, 30, precision=64, path=path, **variant)
    Uo, to, _ = oracle_run(orc, w, 30, **variant)
    assert max(rel_linf(Ug, Uo)) <= 1e-10


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("path", PATHS, ids=["plain", "fast"])
def test_hllc_selects_the_hll_flux(path, prec):
    # Sec. 2.2 names HLLC; on the advective system it is read as HLL (no
    # contact wave between the two particle speeds), so the option must give
    # the HLL result bit for bit.
    w = wl.random_state((12, 14, 16), seed=2, psi_amp=0.1, bc=[I_, O_, P_, P_, W_, O_])
    Uc, tc, _ = gpu_run(w, 20, precision=prec, path=path, riemann=cspht.RIEMANN_HLLC)
    Uh, th, _ = gpu_run(w, 20, precision=prec, path=path, riemann=cspht.RIEMANN_HLL)
    assert np.array_equal(Uc, Uh) and tc == th


def test_sod_full_size_200_steps(orc):
    """Sod along x on 128x16x16, 200 steps at CFL 0.4 (the small config)."""
    w = wl.shock_tube()
    Ug, tg, _ = gpu_run(w, 200, precision=64, path=cspht.PATH_FAST)
    Uo, to, _ = oracle_run(orc, w, 200)
    assert max(rel_linf(Ug, Uo)) <= 1e-10


@pytest.mark.parametrize("path", PATHS, ids=["plain", "fast"])
def test_fp32_smooth_flow_within_1e4(orc, path):
    """Single precision against the FP64 oracle on a smooth flow in a
    potential: relative L1 per field <= 1e-4."""
    w = wl.potential_well(n=32, ny=16, nz=16, mach=2.0, psi0=0.5)
    Ug, tg, _ = gpu_run(w, 60, precision=32, path=path)
    Uo, to, _ = oracle_run(orc, w, 60)
    for f in range(5):
        l1 = np.abs(Ug[f] - Uo[f]).sum() / max(np.abs(Uo[f]).sum(), 1e-300)
        assert l1 <= 1e-4, (f, l1)


@pytest.mark.parametrize("path", PATHS, ids=["plain", "fast"])
def test_fp32_sod_shock_within_one_cell(orc, path):
    w = wl.shock_tube(nx=128, ny=4, nz=4)
    Ug, tg, _ = gpu_run(w, 200, precision=32, path=path)
    Uo, to, _ = oracle_run(orc, w, 200)
    mid = 0.5 * (0.26557 + 0.125)

    def shock(line):
        return np.where((line[:-1] >= mid) & (line[1:] < mid))[0][-1]

    assert abs(shock(Ug[0, 0, 0]) - shock(Uo[0, 0, 0])) <= 1
    l1 = np.abs(Ug[0] - Uo[0]).mean() / np.abs(Uo[0]).mean()
    assert l1 < 1e-3


def test_fp32_compensated_balance_within_1e4(orc):
    """The compensated balance terms (TwoProd and TwoSum on the pressure
    force minus gravity) keep the FP32 fused path within relative L1 1e-4 of
    the FP64 oracle on the smooth flow in a potential."""
    w = wl.potential_well(n=32, ny=16, nz=16, mach=2.0, psi0=0.5)
    Ug, _, _ = gpu_run(w, 60, precision=32, path=cspht.PATH_FAST, balance=cspht.BALANCE_COMPENSATED)
    Uo, _, _ = oracle_run(orc, w, 60)
    for f in range(5):
        l1 = np.abs(Ug[f] - Uo[f]).sum() / max(np.abs(Uo[f]).sum(), 1e-300)
        assert l1 <= 1e-4, (f, l1)


@pytest.mark.parametrize("prec,path", [(64, cspht.PATH_FAST), (32, cspht.PATH_PLAIN)], ids=["fp64_fast", "fp32_plain"])
def test_balance_option_only_changes_the_fp32_fused_path(prec, path):
    w = wl.random_state((12, 14, 16), seed=2, psi_amp=0.2, bc=[I_, O_, P_, P_, W_, O_])
    a, ta, _ = gpu_run(w, 10, precision=prec, path=path, balance=cspht.BALANCE_PLAIN)
    b, tb, _ = gpu_run(w, 10, precision=prec, path=path, balance=cspht.BALANCE_COMPENSATED)
    assert np.array_equal(a, b) and ta == tb


def test_uniform_inflow_state_stays_uniform():
    w = wl.potential_well(n=24, ny=8, nz=8, psi0=0.0)
    for prec in (32, 64):
        U, t, _ = gpu_run(w, 20, precision=prec)
        for f in range(5):
            ref = U[f, 0, 0, 0]
            assert np.abs(U[f] - ref).max() <= (1e-5 if prec == 32 else 1e-13) * max(abs(ref), 1)


def test_step_reports_dt_and_time(orc):
    w = wl.shock_tube(nx=32, ny=2, nz=2)
    P = oracle_problem(orc, w)
    dt_o = P.dt(P.prim_to_cons(w.W), 0.4)
    with cspht.Sim.from_workload(w, precision=64) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        dt = s.step(0.4)
        assert dt == pytest.approx(dt_o, rel=1e-14)
        assert s.time() == pytest.approx(dt, rel=1e-15)
        n = s.run(0.1, 0.4)
        assert s.time() == 0.1 and n > 0


def test_status_nonfinite_is_reported():
    w = wl.shock_tube(nx=16, ny=2, nz=2)
    W = np.ascontiguousarray(w.W).copy()
    W[4, 0, 0, 5] = np.nan  # injected on the host
    with cspht.Sim.from_workload(w, precision=64) as s:
        s.set_primitive(W)
        with pytest.raises(cspht.CsphtError) as e:
            s.step(0.4)
        assert e.value.code == cspht.ENONFINITE


def test_status_cfl_violation_is_reported():
    w = wl.smooth_wave(nx=32, ny=2, nz=2, u=2.0)
    with cspht.Sim.from_workload(w, precision=64) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        with pytest.raises(cspht.CsphtError) as e:
            s.step(3.0)  # a Courant number far above 1 moves particles > h
        assert e.value.code == cspht.ECFL


def test_checkpoint_resume_is_bitwise():
    w = wl.random_state((12, 10, 14), seed=3, psi_amp=0.1)
    for prec in (32, 64):
        with cspht.Sim.from_workload(w, precision=prec) as a:
            a.set_primitive(np.ascontiguousarray(w.W))
            a.advance(10, 0.4)
            mid = a.get_state()
            a.advance(10, 0.4)
            ref = a.get_state()
        with cspht.Sim.from_workload(w, precision=prec) as b:
            b.set_state(mid)
            b.advance(10, 0.4)
            np.testing.assert_array_equal(b.get_state(), ref)


@pytest.mark.parametrize("prec", [32, 64])
def test_autotune_keeps_the_state_and_the_results(prec):
    """cspht_autotune restores the state it times on, and the tile depth it
    picks changes no result bit (a chunk's first planes are recomputed with
    the same arithmetic)."""
    w = wl.potential_well(n=64, mach=2.0)
    with cspht.Sim.from_workload(w, precision=prec) as a, cspht.Sim.from_workload(w, precision=prec) as b:
        for s in (a, b):
            s.set_primitive(np.ascontiguousarray(w.W))
            s.advance(5, 0.4)
            s.sync()
        before, t_before = a.get_state(), a.time()
        z = a.autotune(steps=3, cfl=0.4)
        assert 1 <= z <= 64
        np.testing.assert_array_equal(a.get_state(), before)
        assert a.time() == t_before
        for s in (a, b):
            s.advance(10, 0.4)
            s.sync()
        np.testing.assert_array_equal(a.get_state(), b.get_state())
    with cspht.Sim.from_workload(w, precision=prec, path=cspht.PATH_PLAIN) as p:
        p.set_primitive(np.ascontiguousarray(w.W))
        assert p.autotune(steps=2) == 0


def test_fp64_autotune_chooses_fused_or_split_stages(orc):
    """On an FP64 handle the autotuner also times the unfused kernels (split
    stages), which win on the smallest grids.  Whichever it keeps, the state
    is restored, the handle then runs that path (its launches per step show
    it: 5 fused, at least 15 unfused) and stays within 1e-10 of the oracle."""
    w = wl.potential_well(n=32, mach=2.0)
    with cspht.Sim.from_workload(w, precision=64) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        before, t0 = s.get_state(), s.time()
        z = s.autotune(steps=4, cfl=0.4)
        np.testing.assert_array_equal(s.get_state(), before)
        assert s.time() == t0
        s.advance(1, 0.4)  # (re-sends the step parameters the autotuner replaced)
        l0 = s.launch_count()
        s.advance(1, 0.4)
        s.sync()
        per_step = s.launch_count() - l0
        assert (per_step >= 15) if z == 0 else (per_step == 5 and 1 <= z <= 32), (z, per_step)
        s.advance(28, 0.4)
        s.sync()
        Ug = s.get_state()
    Uo, _, _ = oracle_run(orc, w, 30)
    assert max(rel_linf(Ug, Uo)) <= 1e-10


@pytest.mark.parametrize("make", [
    lambda: wl.potential_well(n=64, mach=2.0),
    lambda: wl.blast(n=32, radius_cells=2.0),
    lambda: wl.hydrostatic(n=40, nxy=8, perturb=1e-6),
], ids=["well_periodic_z", "blast_outflow", "atmosphere_wall_vacuum"])
@pytest.mark.parametrize("prec", [32, 64])
def test_results_do_not_depend_on_the_tile_depth(make, prec):
    """Neighbouring z chunks share planes (the predictor of a chunk's lower
    neighbour plane, the flux through the face between them); both compute
    them with the same code, so ten steps give the same bits at every depth."""
    w = make()
    nz = w.shape[0]
    out = {}
    for z in (8, 1, 3, 4, 5, 13, nz):
        with cspht.Sim.from_workload(w, precision=prec) as s:
            s.set_tile_depth(z)
            s.set_primitive(np.ascontiguousarray(w.W))
            s.advance(10, 0.4)
            s.sync()
            out[z] = s.get_state()
    for z, U in out.items():
        np.testing.assert_array_equal(U, out[8], err_msg=f"depth {z}")


def test_created_handles_see_their_whole_potential(orc):
    """The potential is uploaded and processed in order on the handle's own
    stream.  A handle created where a freed one held a different potential
    must step like the oracle on windows at the start and at the end of the
    array (a copy still in flight when the first kernel reads the staging
    buffer would leave the previous handle's data in the tail of psi)."""
    wa = wl.random_state((128, 128, 128), seed=41, psi_amp=0.5)
    wb = wl.random_state((128, 128, 128), seed=42, psi_amp=0.5)
    P = oracle_problem(orc, wb)
    Ub0 = P.prim_to_cons(wb.W)
    boxes = [((0, 8), (0, 8), (0, 4)), ((120, 128), (120, 128), (124, 128)), ((60, 68), (0, 8), (126, 128))]
    for rep in range(3):
        with cspht.Sim.from_workload(wa, precision=64) as a:
            a.set_primitive(np.ascontiguousarray(wa.W))
            a.step(0.4)
        with cspht.Sim.from_workload(wb, precision=64) as b:
            b.set_primitive(np.ascontiguousarray(wb.W))
            dt = b.step(0.4)
            U = b.get_state()
        for box in boxes:
            Uo = P.step(wb.psi, Ub0, dt, box=box)
            sl = (slice(None), slice(*box[2]), slice(*box[1]), slice(*box[0]))
            err = np.abs(U[sl] - Uo[sl]).max() / np.abs(Uo[sl]).max()
            assert err <= 1e-10, (rep, box, err)


def test_copy_wait_timeout_is_reported_and_recoverable():
    """Failure detection without a fault: with the test hook on, the fused
    kernels post their copies' byte counts but issue no copy, so every copy
    wait runs out after the given number of polls.  The step must report the
    time-out, and the context must stay usable: with the hook off and the
    state set again, the handle steps exactly like a fresh one."""
    import time
    w = wl.potential_well(n=64, mach=2.0)
    W = np.ascontiguousarray(w.W)
    with cspht.Sim.from_workload(w, precision=32) as s, cspht.Sim.from_workload(w, precision=32) as ref:
        for x in (s, ref):
            x.set_primitive(W)
        s.test_copy_timeout(64)
        t0 = time.perf_counter()
        with pytest.raises(cspht.CsphtError) as e:
            s.step(0.4)
        assert e.value.code == cspht.ECUDA and "timed out" in str(e.value)
        assert time.perf_counter() - t0 < 30.0
        s.test_copy_timeout(0)
        s.set_primitive(W)
        for x in (s, ref):
            x.advance(3, 0.4)
            x.sync()
        np.testing.assert_array_equal(s.get_state(), ref.get_state())


@pytest.mark.parametrize("prec", [32, 64])
def test_float32_host_state(prec):
    """cspht_set_state_f32 / cspht_get_state_f32: FP32 host data round-trips
    exactly, and a state uploaded in FP32 steps exactly like the same values
    uploaded in FP64."""
    w = wl.random_state((10, 12, 40), seed=51, psi_amp=0.1, bc=[I_, O_, P_, P_, W_, O_])
    with cspht.Sim.from_workload(w, precision=64) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        U32 = s.get_state().astype(np.float32)
    with cspht.Sim.from_workload(w, precision=prec) as a, cspht.Sim.from_workload(w, precision=prec) as b:
        a.set_state(U32)
        back = a.get_state(np.empty_like(U32))
        np.testing.assert_array_equal(back, U32)
        b.set_state(U32.astype(np.float64))
        for s in (a, b):
            s.advance(5, 0.4)
            s.sync()
        np.testing.assert_array_equal(a.get_state(), b.get_state())


@pytest.mark.parametrize("path", PATHS, ids=["plain", "fast"])
@pytest.mark.parametrize("prec", [32, 64])
def test_gas_at_rest_without_pressure_takes_a_zero_step(path, prec):
    """The degenerate step: no signal speed anywhere (u = 0, p = 0) gives
    dt = 0, and a zero step copies the state and leaves the time."""
    shape = (6, 7, 9)
    W = np.zeros((5,) + shape)
    W[0] = np.linspace(0.5, 1.5, W[0].size).reshape(shape)
    with cspht.Sim(shape, 0.1, 1.4, np.zeros(shape), precision=prec, path=path) as s:
        s.set_primitive(W)
        U0 = s.get_state()
        assert s.step(0.4) == 0.0
        np.testing.assert_array_equal(s.get_state(), U0)
        assert s.time() == 0.0


@pytest.mark.parametrize("variant", [dict(riemann=1), dict(riemann=2), dict(limiter=1), dict(limiter=2)],
                         ids=["hll", "swept", "minmod", "mc"])
def test_fp32_options_smooth_flow_within_1e4(orc, variant):
    """The fused FP32 path with each Riemann flux and limiter against the FP64
    oracle with the same options: relative L1 per field <= 1e-4."""
    w = wl.potential_well(n=32, ny=16, nz=16, mach=2.0, psi0=0.5)
    Ug, tg, _ = gpu_run(w, 60, precision=32, path=cspht.PATH_FAST, **variant)
    Uo, to, _ = oracle_run(orc, w, 60, **variant)
    for f in range(5):
        l1 = np.abs(Ug[f] - Uo[f]).sum() / max(np.abs(Uo[f]).sum(), 1e-300)
        assert l1 <= 1e-4, (f, l1)


@pytest.mark.parametrize("path", PATHS, ids=["plain", "fast"])
@pytest.mark.parametrize("prec", [32, 64])
def test_periodic_step_is_translation_invariant_to_the_bit(path, prec):
    """On a fully periodic grid the step commutes with a shift of the whole
    state and potential (Eqs. 4-8 have no preferred origin).  A shift by
    (5, 3, 5) cells is not a multiple of the 32 x 8 tile nor of the z chunk,
    so every cell moves to another tile position, chunk and halo role.  The
    outputs are equal bit for bit only if every value a tile shares with its
    neighbours (halo particles, faces, recomputed chunk-seam planes) carries
    the same bits wherever it is computed."""
    w = wl.random_state((21, 19, 45), seed=31, psi_amp=0.1)
    shift = (5, 3, 5)  # (z, y, x); the default z chunk of this grid is 7 planes
    axes = (1, 2, 3)

    def run(W, psi):
        with cspht.Sim(w.shape, w.h, w.gamma, psi, bc=w.bc, precision=prec, path=path) as s:
            s.set_primitive(np.ascontiguousarray(W))
            s.advance(10, 0.4)
            s.sync()
            return s.get_state(), s.time()

    U0, t0 = run(w.W, w.psi)
    U1, t1 = run(np.roll(w.W, shift, axis=axes), np.roll(w.psi, shift, axis=(0, 1, 2)))
    assert t1 == t0
    np.testing.assert_array_equal(U1, np.roll(U0, shift, axis=axes))


def _pinned_f32(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()


@pytest.mark.parametrize("prec", [32, 64])
def test_async_host_io_pipeline_matches_synchronous_calls(prec):
    """Uploads, steps and downloads enqueued without waiting, one step's
    download overlapping the next upload, give each step's result bit for bit
    as the synchronous upload / step / download does."""
    import torch
    w = wl.random_state((20, 24, 40), seed=41, psi_amp=0.1)
    with cspht.Sim.from_workload(w, precision=prec) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        U0 = s.get_state(np.empty((5,) + w.shape, dtype=np.float32))
        ref = np.empty_like(U0)
        s.set_state(U0)
        s.step(0.4)
        s.get_state(ref)
        hin = _pinned_f32(U0)
        outs = [torch.empty_like(hin).pin_memory() for _ in range(4)]
        for o in outs:
            s.upload_async(hin)
            s.advance(1, 0.4)
            s.download_async(o)
        s.sync()
        for o in outs:
            np.testing.assert_array_equal(o.numpy(), ref)


def test_async_and_synchronous_host_io_mix():
    """The synchronous calls share the upload staging buffer with the
    asynchronous upload: each waits for an upload still in flight."""
    import torch
    w = wl.random_state((12, 16, 20), seed=42)
    with cspht.Sim.from_workload(w, precision=32) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        A = s.get_state(np.empty((5,) + w.shape, dtype=np.float32))
        B = (A * np.float32(1.25)).astype(np.float32)
        s.upload_async(_pinned_f32(B))
        got = s.get_state(np.empty_like(A))      # synchronous, after the upload
        np.testing.assert_array_equal(got, B)
        out = torch.empty((5,) + w.shape, dtype=torch.float32).pin_memory()
        s.download_async(out)
        s.set_state(A)                          # synchronous upload after an async download
        s.sync()
        np.testing.assert_array_equal(out.numpy(), B)
        np.testing.assert_array_equal(s.get_state(np.empty_like(A)), A)


def test_calls_that_need_a_state_refuse_a_fresh_handle():
    """Stepping or reading a handle before any state was uploaded returns
    CSPHT_ESTATE (and launches nothing)."""
    w = wl.random_state((8, 8, 16), seed=43)
    with cspht.Sim.from_workload(w, precision=32) as s:
        f32 = np.empty((5,) + w.shape, dtype=np.float32)
        n0 = s.launch_count()
        for call in (lambda: s.step(0.4), lambda: s.advance(2, 0.4), lambda: s.get_state(),
                     lambda: s.get_state(f32), lambda: s.download_async(f32), lambda: s.autotune(2, 0.4)):
            with pytest.raises(cspht.CsphtError) as e:
                call()
            assert e.value.code == cspht.ESTATE
        assert s.launch_count() == n0


@pytest.mark.parametrize("make", [
    lambda: wl.random_state((12, 14, 16), seed=44, psi_amp=0.1),                              # periodic
    lambda: wl.random_state((12, 14, 16), seed=45, psi_amp=0.1, bc=[I_, O_, P_, P_, O_, O_]),  # inflow x
], ids=["periodic", "inflow_outflow"])
@pytest.mark.parametrize("path", PATHS, ids=["plain", "fast"])
def test_run_to_a_time_then_continue_matches_oracle(orc, make, path):
    """cspht_run enqueues steps in chunks: after the step that lands on t_end
    the rest of the chunk are zero steps (dt = 0, the state copied).  Stepping
    on afterwards must see the boundary layers of the copied state: 5 steps,
    a run to 1.3 dt beyond, then 5 more steps match the oracle doing the same."""
    w = make()
    with cspht.Sim.from_workload(w, precision=64, path=path) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        s.advance(5, 0.4)
        s.sync()
        t5 = s.time()
        U5 = s.get_state()
        P = oracle_problem(orc, w)
        dt5 = P.dt(U5, 0.4)
        t_mid = t5 + 1.3 * dt5
        s.run(t_mid, 0.4)
        s.advance(5, 0.4)
        s.sync()
        Ug, tg = s.get_state(), s.time()
    U0 = P.prim_to_cons(w.W)
    Uo, to, _, rc = P.run(w.psi, U0, nsteps=5, cfl=0.4)
    Uo, to, _, rc2 = P.run(w.psi, Uo, cfl=0.4, t_end=t_mid, t0=to)
    Uo, to, _, rc3 = P.run(w.psi, Uo, nsteps=5, cfl=0.4, t0=to)
    assert rc == rc2 == rc3 == 0
    assert tg == pytest.approx(to, rel=1e-12)
    assert max(rel_linf(Ug, Uo)) <= 1e-10

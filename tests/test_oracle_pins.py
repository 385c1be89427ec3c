"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, exact invariants, textbook special cases written independently here,
and the exact Riemann solution.  The choice is meant to catch a dropped term,
a wrong sign or a transposed index anywhere in the step.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1912_04855_b300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")
P_, O_, I_, W_ = wl.PERIODIC, wl.OUTFLOW, wl.INFLOW, wl.WALL


def problem(orc, w: wl.Workload, **kw):
    return orc.Problem(w.shape, w.h, w.gamma, w.bc, inflow=w.inflow, **kw)


def m4_W(q):
    """M4 cubic spline shape (unnormalised), written from its definition."""
    q = abs(q)
    if q < 1.0:
        return 1.0 - 1.5 * q * q + 0.75 * q ** 3
    if q < 2.0:
        return 0.25 * (2.0 - q) ** 3
    return 0.0


# --------------------------------------------------------------------- kernel

def test_kernel_constants_closed_form(orc):
    g = json.load(open(os.path.join(GOLD, "kernel_constants.json")))
    assert orc.gtilde(1.0) == pytest.approx(g["gt_face"], rel=1e-15)
    assert orc.gtilde(math.sqrt(2.0)) == pytest.approx(g["gt_edge"], rel=1e-14)
    assert orc.gtilde(math.sqrt(3.0)) == pytest.approx(g["gt_corner"], rel=1e-14)
    assert orc.norm_C() == pytest.approx(g["C"], rel=1e-15)
    assert orc.gtilde(2.0) == 0.0 and orc.gtilde(2.5) == 0.0


@pytest.mark.parametrize("q", [0.13, 0.5, 0.97, 1.03, 1.41, 1.8, 1.99])
def test_kernel_is_minus_dW_over_q(orc, q):
    # gt(q) = -W'(q)/q, W' by a central difference of the spline itself
    e = 1e-6
    dW = (m4_W(q + e) - m4_W(q - e)) / (2 * e)
    assert orc.gtilde(q) == pytest.approx(-dW / q, rel=1e-8)


# ------------------------------------------------------------------------ EOS

def test_eos_round_trip_and_vacuum(orc):
    w = wl.random_state((4, 5, 6), seed=3)
    P = problem(orc, w)
    U = P.prim_to_cons(w.W)
    u, p, phi, vac = P.eos(U)
    assert not vac.any()
    np.testing.assert_allclose(u, w.W[1:4], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(p, w.W[4], rtol=1e-13)
    np.testing.assert_allclose(phi * phi, 2 * w.W[4], rtol=1e-13)
    # vacuum threshold: rho <= rho_vac -> u = p = phi = 0; floor p >= 0
    U2 = U.copy()
    U2[0, 0, 0, 0] = 1e-10
    U2[0, 0, 0, 1] = 0.0
    U2[4, 0, 0, 2] = 0.0  # kinetic energy above E -> floored pressure
    u, p, phi, vac = P.eos(U2)
    assert vac[0, 0, 0] and vac[0, 0, 1] and not vac[0, 0, 2]
    assert p[0, 0, 0] == 0 and phi[0, 0, 0] == 0 and (u[:, 0, 0, 0] == 0).all()
    assert p[0, 0, 2] == 0.0


# ------------------------------------------------------- Lagrangian force Q

def _uniform(shape, rho=1.0, u=(0, 0, 0), p=1.0):
    W = np.zeros((5,) + shape)
    W[0], W[4] = rho, p
    for e in range(3):
        W[1 + e] = u[e]
    return W


def test_gravity_operator_exact_on_linear_psi(orc):
    """f = -D0[psi] equals -grad psi exactly for linear psi (lattice
    normalisation C), with the sign of Eqs. 2-3: dm/dt = -rho grad psi."""
    shape = (6, 7, 8)
    h = 0.1
    P = orc.Problem(shape, h, 1.4, [O_] * 6)
    z, y, x = np.meshgrid(*[(np.arange(n) + 0.5) * h for n in shape], indexing="ij")
    g = (0.7, -1.3, 2.1)
    psi = g[0] * x + g[1] * y + g[2] * z + 0.3
    rho = 1.7
    U = P.prim_to_cons(_uniform(shape, rho=rho, u=(0.2, -0.1, 0.3)))
    Q = P.force(psi, U)
    for e in range(3):
        np.testing.assert_allclose(Q[e], -rho * g[e], rtol=1e-12, atol=1e-12)
    # energy source rho u.f
    np.testing.assert_allclose(Q[3], -rho * (0.2 * g[0] - 0.1 * g[1] + 0.3 * g[2]), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_pressure_term_exact_for_linear_phi(orc, axis):
    """phi linear along one axis -> phi_i D0[phi] = phi_i * slope exactly:
    dm/dt = -grad p with p = phi^2/2 (interior cells)."""
    shape = (9, 9, 9)
    h = 1.0 / 9
    P = orc.Problem(shape, h, 1.4, [O_] * 6)
    c = (np.arange(9) + 0.5) * h
    beta = 0.8
    phi = 1.0 + beta * c
    W = _uniform(shape, rho=1.3)
    sh = [1, 1, 1]
    sh[2 - axis] = 9
    W[4] = np.broadcast_to((0.5 * phi * phi).reshape(sh), shape)
    U = P.prim_to_cons(W)
    Q = P.force(np.zeros(shape), U)
    inner = (slice(1, -1),) * 3
    phi3 = np.broadcast_to(phi.reshape(sh), shape)
    for e in range(3):
        expect = -phi3 * beta if e == axis else 0.0 * phi3
        np.testing.assert_allclose(Q[e][inner], expect[inner], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Q[3][inner], 0.0, atol=1e-12)


def test_pressure_work_exact_for_linear_velocity(orc):
    """Uniform p, u = (a x, b y, c z) -> dE/dt = -div(p u) = -p (a + b + c)."""
    shape = (8, 8, 8)
    h = 0.125
    P = orc.Problem(shape, h, 1.4, [O_] * 6)
    z, y, x = np.meshgrid(*[(np.arange(8) + 0.5) * h for _ in range(3)], indexing="ij")
    a, b, c = 0.3, -0.2, 0.45
    p = 0.9
    W = _uniform(shape, rho=1.0, p=p)
    W[1], W[2], W[3] = a * x, b * y, c * z
    U = P.prim_to_cons(W)
    Q = P.force(np.zeros(shape), U)
    inner = (slice(1, -1),) * 3
    np.testing.assert_allclose(Q[3][inner], -p * (a + b + c), rtol=1e-12)
    for e in range(3):
        np.testing.assert_allclose(Q[e][inner], 0.0, atol=1e-12)


def test_pairwise_antisymmetry_conserves_momentum_and_energy(orc):
    """With psi = 0 and periodic faces, sum_i Q_i = 0 for arbitrary particle
    offsets (Eq. 7 is a sum of antisymmetric pair terms)."""
    w = wl.random_state((6, 7, 8), seed=11)
    P = problem(orc, w)
    U = P.prim_to_cons(w.W)
    rng = np.random.default_rng(5)
    xi = rng.uniform(-0.3, 0.3, size=(3,) + w.shape) * w.h
    Q = P.force(np.zeros(w.shape), U, xi=xi)
    for e in range(4):
        scale = np.abs(Q[e]).sum()
        assert abs(Q[e].sum()) <= 1e-13 * scale


def test_uniform_shift_of_particles_changes_nothing(orc):
    """Pair vectors depend on xi_j - xi_i only: a common shift of all particles
    reproduces the static-lattice force."""
    w = wl.random_state((5, 6, 7), seed=12)
    P = problem(orc, w)
    U = P.prim_to_cons(w.W)
    xi = np.empty((3,) + w.shape)
    xi[0], xi[1], xi[2] = 0.21 * w.h, -0.17 * w.h, 0.05 * w.h
    np.testing.assert_allclose(P.force(w.psi, U, xi=xi), P.force(w.psi, U), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("delta", [-0.35, -0.1, 0.2, 0.45])
def test_displaced_pair_closed_form(orc, delta):
    """Two gas cells in vacuum, the second displaced by delta*h along x: the
    only pair term is phi_i phi_j G(r) r with G = gt(r/h)/(C h^2) and
    gt(q) = -W'(q)/q of the M4 spline."""
    shape = (3, 3, 4)
    h = 0.5
    P = orc.Problem(shape, h, 1.4, [P_] * 6)
    W = np.zeros((5,) + shape)
    W[0, 1, 1, 1] = W[0, 1, 1, 2] = 1.0
    W[4, 1, 1, 1], W[4, 1, 1, 2] = 0.8, 0.5
    U = P.prim_to_cons(W)
    xi = np.zeros((3,) + shape)
    xi[0, 1, 1, 2] = delta * h
    Q = P.force(np.zeros(shape), U, xi=xi)
    r = h * (1 + delta)
    q = r / h
    e = 1e-6
    gt = -((m4_W(q + e) - m4_W(q - e)) / (2 * e)) / q
    C = 2 * 0.75 + 8 * 0.75 * (2 - 2 ** 0.5) ** 2 / 2 ** 0.5 + 8 * 0.75 * (2 - 3 ** 0.5) ** 2 / 3 ** 0.5
    phi_i, phi_j = math.sqrt(1.6), math.sqrt(1.0)
    expect = -phi_i * phi_j * gt / (C * h * h) * r
    assert Q[0, 1, 1, 1] == pytest.approx(expect, rel=1e-7)
    assert Q[0, 1, 1, 2] == pytest.approx(-expect, rel=1e-7)
    assert abs(Q[1, 1, 1, 1]) < 1e-15 and abs(Q[2, 1, 1, 1]) < 1e-15
    # vacuum cells feel nothing
    assert np.all(Q[:, 0] == 0) and Q[0, 1, 1, 0] == 0


# ------------------------------------------------------- time integration

def test_heun_exact_under_uniform_gravity(orc):
    """Uniform state in psi = g.x: the predictor-corrector of Eqs. 5-6 is
    Heun's method on dm/dt = -rho g, dE/dt = -m.g, exact here because m is
    linear in t; particle offset = the exact displacement u dt - g dt^2/2."""
    shape = (5, 6, 7)
    h = 0.1
    P = orc.Problem(shape, h, 5.0 / 3.0, [O_] * 6)
    z, y, x = np.meshgrid(*[(np.arange(n) + 0.5) * h for n in shape], indexing="ij")
    g = np.array([0.4, -0.9, 1.6])
    psi = g[0] * x + g[1] * y + g[2] * z
    rho, u, p = 1.3, np.array([0.5, 0.2, -0.3]), 0.7
    U = P.prim_to_cons(_uniform(shape, rho=rho, u=tuple(u), p=p))
    dt = 0.01
    Us, xs, Un, xn = P.lagrange(psi, U, dt)
    m0 = rho * u
    E0 = U[4, 0, 0, 0]
    for e in range(3):
        np.testing.assert_allclose(Un[1 + e], m0[e] - rho * g[e] * dt, rtol=1e-12)
        np.testing.assert_allclose(xn[e], u[e] * dt - 0.5 * g[e] * dt * dt, rtol=1e-11)
    np.testing.assert_allclose(Un[4], E0 - m0 @ g * dt + 0.5 * rho * (g @ g) * dt * dt, rtol=1e-12)
    np.testing.assert_array_equal(Un[0], U[0])
    # the Euler stage moves a uniform state as a whole: U^{n+1} = U~
    U1 = P.step(psi, U, dt)
    np.testing.assert_allclose(U1, Un, rtol=1e-12, atol=1e-14)


# --------------------------------------------- Euler stage: MUSCL-Hancock

def _vl(a, b):
    out = np.zeros_like(a)
    m = a * b > 0
    out[m] = 2 * a[m] * b[m] / (a[m] + b[m])
    return out


def _mm(a, b):
    return np.where(a * b > 0, np.where(np.abs(a) < np.abs(b), a, b), 0.0)


def _mc(a, b):
    m = np.minimum(np.minimum(np.abs(2 * a), np.abs(2 * b)), np.abs(0.5 * (a + b)))
    return np.where(a * b > 0, np.sign(a) * m, 0.0)


def muscl_hancock_1d(q, u, dt, h, lim):
    """van Leer's MUSCL-Hancock scheme for q_t + u q_x = 0 on a periodic line."""
    dp = (np.roll(q, -1) - q) / h
    dm = (q - np.roll(q, 1)) / h
    th = lim(dp, dm)
    if u > 0:
        qf = q + 0.5 * (h - u * dt) * th  # left state of face i+1/2
    else:
        qf = np.roll(q - 0.5 * (h + u * dt) * th, -1)  # right state of face i+1/2
    F = u * qf
    return q - dt / h * (F - np.roll(F, 1))


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("u", [0.7, -0.45])
@pytest.mark.parametrize("lim", [0, 1, 2])
def test_step_reduces_to_muscl_hancock(orc, axis, u, lim):
    """Uniform p and u, varying rho (psi = 0): Q vanishes and the step is the
    MUSCL-Hancock linear-advection scheme applied to every conserved field."""
    n = 24
    shape = [3, 3, 3]
    shape[2 - axis] = n
    shape = tuple(shape)
    h = 1.0 / n
    P = orc.Problem(shape, h, 1.4, [P_] * 6, limiter=lim)
    c = (np.arange(n) + 0.5) * h
    rho1d = 1.0 + 0.3 * np.sin(2 * np.pi * c) + 0.2 * (c > 0.5)
    sh = [1, 1, 1]
    sh[2 - axis] = n
    W = _uniform(shape, p=1.0)
    W[0] = np.broadcast_to(rho1d.reshape(sh), shape)
    W[1 + axis] = u
    U = P.prim_to_cons(W)
    dt = 0.4 * h / (abs(u) + 1.5)
    U1 = P.step(np.zeros(shape), U, dt)
    limf = [_vl, _mm, _mc][lim]
    for f in range(5):
        line = np.moveaxis(U[f], 2 - axis, -1)[0, 0] if axis != 1 else U[f][0, :, 0]
        ref = muscl_hancock_1d(line, u, dt, h, limf)
        got = np.moveaxis(U1[f], 2 - axis, -1)[0, 0] if axis != 1 else U1[f][0, :, 0]
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.abs(got - ref).max() <= 1e-13 * scale + 1e-15, f"field {f}"


@pytest.mark.parametrize("rk", [1, 2])
def test_hll_and_swept_equal_upwind_for_uniform_speed(orc, rk):
    """With one advection speed everywhere, LF, HLL and the swept-volume flux
    all reduce to the upwind flux a U_upwind."""
    w = wl.smooth_wave(nx=32, ny=2, nz=2, u=0.6)
    U = problem(orc, w).prim_to_cons(w.W)
    dt = 0.01
    a = problem(orc, w, riemann=0).step(w.psi, U, dt)
    b = problem(orc, w, riemann=rk).step(w.psi, U, dt)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-15)


def test_swept_flux_moves_uniform_density_with_the_mean_face_speed(orc):
    """Uniform density and pressure, varying velocity (psi = 0): the density
    has no slope and U_L = U_R at every face, so every flux that is
    consistent with F = a U gives the mass flux a_face rho.  LF gives
    (a_L + a_R)/2 rho there; the swept-volume flux must give the same (it
    sweeps with the mean of the two particles' offsets), while the other
    fields, whose reconstructed states differ across the faces, must not
    agree with LF."""
    w = wl.random_state((6, 7, 16), seed=31, vel=0.4)
    w.W[0] = 1.3
    w.W[4] = 0.9
    P0, P2 = problem(orc, w, riemann=0), problem(orc, w, riemann=2)
    U = P0.prim_to_cons(w.W)
    dt = 0.5 * P0.dt(U, 0.4)
    a = P0.step(np.zeros(w.shape), U, dt)
    b = P2.step(np.zeros(w.shape), U, dt)
    np.testing.assert_allclose(b[0], a[0], rtol=1e-14)
    assert np.abs(b[1:] - a[1:]).max() > 1e-6


# ------------------------------------------------- boundaries and windows

@pytest.mark.parametrize("bc", [[O_] * 6, [P_, P_, O_, O_, P_, P_], [I_, O_, P_, P_, O_, O_]])
def test_uniform_flow_stays_uniform(orc, bc):
    shape = (5, 6, 7)
    h = 1 / 7
    W0 = (1.2, 0.3, 0.0, 0.0, 0.8)
    inflow = [list(W0)] * 6
    P = orc.Problem(shape, h, 1.4, bc, inflow=inflow)
    U = P.prim_to_cons(_uniform(shape, rho=W0[0], u=(W0[1], 0, 0), p=W0[4]))
    U1, t, s, rc = P.run(np.zeros(shape), U, nsteps=5)
    assert rc == 0 and s == 5
    for f in range(5):
        np.testing.assert_allclose(U1[f], U[f, 0, 0, 0], rtol=1e-13, atol=1e-14)


def test_closed_box_conserves_mass_and_rest(orc):
    """Reflecting walls on every face, psi = 0: no mass crosses a wall (zero
    face flux), and a uniform gas at rest stays exactly at rest.  Energy is
    not exactly conserved at walls: the ghost phi is extrapolated through the
    boundary cell's centre (phi_g = phi_m at psi = 0) so that hydrostatic
    states stay discrete equilibria, and pressure-work pairs across the wall
    then no longer cancel."""
    w = wl.random_state((6, 6, 6), seed=21, bc=[W_] * 6)
    P = problem(orc, w)
    U = P.prim_to_cons(w.W)
    T0 = P.totals(w.psi, U)
    U1, t, s, rc = P.run(np.zeros(w.shape), U, nsteps=20)
    T1 = P.totals(w.psi, U1)
    assert rc == 0
    assert abs(T1[0] - T0[0]) <= 1e-14 * T0[0]
    assert abs(T1[4] - T0[4]) <= 1e-2 * T0[4]
    shape = (5, 6, 7)
    P2 = orc.Problem(shape, 0.1, 1.4, [W_] * 6)
    U = P2.prim_to_cons(_uniform(shape, rho=0.8, p=0.6))
    U1, *_ = P2.run(np.zeros(shape), U, nsteps=10)
    np.testing.assert_allclose(U1[1:4], 0.0, atol=1e-15)
    np.testing.assert_allclose(U1, U, rtol=1e-14, atol=1e-15)


def test_zero_step_is_the_identity(orc):
    """dt = 0 in Eqs. 4-8: no particle moves, every increment carries a factor
    dt, so the step returns U^n for any state (periodic and walled faces)."""
    for bc in ([P_] * 6, [I_, O_, P_, P_, W_, O_]):
        w = wl.random_state((6, 7, 8), seed=5, psi_amp=0.2, bc=bc)
        P = problem(orc, w)
        U = P.prim_to_cons(w.W)
        np.testing.assert_allclose(P.step(w.psi, U, 0.0), U, rtol=1e-15, atol=1e-300)


def test_gas_at_rest_without_pressure_has_no_time_step(orc):
    """u = 0 and p = 0 everywhere: the largest signal speed |u| + c is 0, the
    CFL rule gives no positive step, and a run stops before its first step."""
    shape = (5, 6, 7)
    P = orc.Problem(shape, 0.1, 1.4, [P_] * 6)
    W = _uniform(shape, rho=1.0, p=0.0)
    W[0] = np.linspace(0.5, 1.5, W[0].size).reshape(shape)
    U = P.prim_to_cons(W)
    assert P.dt(U, 0.4) == 0.0
    U1, t, s, rc = P.run(np.zeros(shape), U.copy(), nsteps=3)
    assert (rc, s, t) == (0, 0, 0.0)
    np.testing.assert_array_equal(U1, U)


@pytest.mark.parametrize("bc", [[P_] * 6, [I_, O_, P_, P_, W_, O_], [W_, W_, O_, I_, P_, P_]])
def test_window_equals_full_step(orc, bc):
    """The windowed step (used to sample full-size grids) gives bit-identical
    cells to the whole-grid step, at every kind of face."""
    w = wl.random_state((9, 10, 11), seed=7, bc=bc, psi_amp=0.1)
    P = problem(orc, w)
    U = P.prim_to_cons(w.W)
    dt = 0.3 * P.dt(U, 1.0)
    full = P.step(w.psi, U, dt)
    for box in [((0, 3), (0, 2), (0, 4)), ((8, 11), (7, 10), (5, 9)), ((4, 6), (3, 5), (2, 3))]:
        part = P.step(w.psi, U, dt, box=box)
        sl = (slice(*box[2]), slice(*box[1]), slice(*box[0]))
        np.testing.assert_array_equal(part[(slice(None),) + sl], full[(slice(None),) + sl])


# --------------------------------------------------------- conservation T3

@pytest.mark.parametrize("rk", [0, 1, 2])
def test_periodic_conservation(orc, rk):
    w = wl.random_state((10, 9, 8), seed=4, vel=0.2)
    P = problem(orc, w, riemann=rk)
    U = P.prim_to_cons(w.W)
    T0 = P.totals(w.psi, U)
    U1, t, s, rc = P.run(w.psi, U, nsteps=30)
    T1 = P.totals(w.psi, U1)
    assert rc == 0
    for f in (0, 4):
        assert abs(T1[f] - T0[f]) <= 2e-14 * abs(T0[f])
    for f in (1, 2, 3):
        assert abs(T1[f] - T0[f]) <= 1e-13 * T0[0]
    # mass stays exact in a potential as well
    w2 = wl.random_state((8, 8, 8), seed=9, psi_amp=0.5)
    P2 = problem(orc, w2)
    U = P2.prim_to_cons(w2.W)
    m0 = P2.totals(w2.psi, U)[0]
    U1, *_ = P2.run(w2.psi, U, nsteps=20)
    assert abs(P2.totals(w2.psi, U1)[0] - m0) <= 2e-14 * m0


def test_hllc_reads_as_hll(orc):
    # HLLC adds a contact wave inside the HLL fan; on the advective system
    # F = a U (Eq. 4's fluxes as read here) every component moves with the one
    # particle speed, so the option is the HLL flux: same bits over 20 steps
    # with converging and diverging faces, a potential and mixed boundaries.
    w = wl.random_state((9, 10, 11), seed=31, psi_amp=0.2, vel=0.4, bc=[I_, O_, P_, P_, W_, O_])
    runs = []
    for rk in (orc.RIEMANN_HLLC, orc.RIEMANN_HLL):
        P = problem(orc, w, riemann=rk)
        U, t, s, rc = P.run(w.psi, P.prim_to_cons(w.W), nsteps=20)
        assert rc == 0 and s == 20
        runs.append((U, t))
    assert np.array_equal(runs[0][0], runs[1][0]) and runs[0][1] == runs[1][1]
    # and it is not the LF flux on this state (the option does select something)
    P = problem(orc, w, riemann=orc.RIEMANN_LF)
    U, *_ = P.run(w.psi, P.prim_to_cons(w.W), nsteps=20)
    assert np.abs(U - runs[0][0]).max() > 1e-8


# ----------------------------------------------------- shock tube T1 (Sod)

def _sod_error(orc, n, t_end=0.2):
    w = wl.shock_tube(nx=n, ny=2, nz=2)
    P = problem(orc, w)
    U = P.prim_to_cons(w.W)
    U1, t, s, rc = P.run(w.psi, U, cfl=0.4, t_end=t_end)
    assert rc == 0 and t == pytest.approx(t_end)
    x = (np.arange(n) + 0.5) / n
    rho, u, p = orc.riemann_sample(1.4, (1, 0, 1), (0.125, 0, 0.1), (x - 0.4) / t)
    return U1, rho, np.abs(U1[0, 0, 0] - rho).mean()


def test_sod_converges_to_exact_solution(orc):
    errs = [_sod_error(orc, n)[2] for n in (64, 128, 256)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 6e-3
    assert min(orders) >= 0.7, (errs, orders)


def test_sod_shock_position_and_column_symmetry(orc):
    n = 256
    U1, rho, err = _sod_error(orc, n)
    # every (y, z) column is bitwise the same
    for f in range(5):
        assert (U1[f] == U1[f, :1, :1, :]).all()
    # shock: where rho crosses the midpoint of rho*_R and rho_R, right of the contact
    star = json.load(open(os.path.join(GOLD, "toro_sod_star.json")))
    mid = 0.5 * (star["rho_star_right"] + 0.125)
    line = U1[0, 0, 0]
    i = np.where((line[:-1] >= mid) & (line[1:] < mid))[0][-1]
    x_num = (i + 1) / n
    ps, us = orc.riemann_star(1.4, (1, 0, 1), (0.125, 0, 0.1))
    rs = star["rho_star_right"]
    S = us * rs / (rs - 0.125)  # mass balance across the right shock
    assert abs(x_num - (0.4 + S * 0.2)) <= 2.0 / n


def test_riemann_problem_is_axis_independent(orc):
    """The same Riemann problem along x, y and z gives the same profile."""
    prof = []
    for axis in range(3):
        w = wl.shock_tube(nx=3 if axis else 48, ny=48 if axis == 1 else 3, nz=48 if axis == 2 else 3,
                          axis=axis)
        P = problem(orc, w)
        U1, t, s, rc = P.run(w.psi, P.prim_to_cons(w.W), nsteps=30)
        line = [U1[0, 1, 1, :], U1[0, 1, :, 1], U1[0, :, 1, 1]][axis]
        mom = [U1[1, 1, 1, :], U1[2, 1, :, 1], U1[3, :, 1, 1]][axis]
        prof.append((line, mom))
    for axis in (1, 2):
        np.testing.assert_allclose(prof[axis][0], prof[0][0], rtol=1e-12)
        np.testing.assert_allclose(prof[axis][1], prof[0][1], rtol=1e-12, atol=1e-14)


# ------------------------------------------------- well-balancing T2

def _hydro_closed(orc, discrete, perturb, steps, n=48, nxy=4):
    """Isothermal column between two reflecting walls, no vacuum: with the
    discrete profile the whole column is a discrete equilibrium."""
    w = wl.hydrostatic(n=n, nxy=nxy, discrete=discrete, perturb=perturb, z_vac=2.0, top_bc=W_)
    P = problem(orc, w)
    U, t, s, rc = P.run(w.psi, P.prim_to_cons(w.W), nsteps=steps, cfl=0.4)
    assert rc == 0 and s == steps
    u, p, phi, vac = P.eos(U)
    return np.abs(u).max(), P, w, U


def test_well_balanced_discrete_equilibrium(orc):
    umax, P, w, U = _hydro_closed(orc, discrete=True, perturb=0.0, steps=300)
    assert umax <= 1e-12, umax


def test_well_balance_negative_control(orc):
    """The continuous exp(-z/H) profile is not a discrete equilibrium: the same
    measurement must see truncation-size velocities (the test has teeth)."""
    umax, *_ = _hydro_closed(orc, discrete=False, perturb=0.0, steps=100)
    assert umax > 1e-6, umax


def test_perturbed_equilibrium_does_not_grow(orc):
    c = math.sqrt(1.4 * 0.2)
    u1, P, w, U = _hydro_closed(orc, discrete=True, perturb=1e-6, steps=100, nxy=6)
    U2, t, s, rc = P.run(w.psi, U, nsteps=100)
    u2 = np.abs(P.eos(U2)[0]).max()
    assert u1 < 1e-5 * c and u2 < 1e-5 * c, (u1, u2)
    assert u2 < 3 * u1


def test_atmosphere_below_vacuum_rarefaction_stays_at_rest(orc):
    """The atmosphere topped by vacuum (C2's layout) stays at rest to rounding
    below the descending rarefaction, whose smeared head runs ahead of the
    sound front by a few cells per sqrt(step)."""
    n = 64
    w = wl.hydrostatic(n=n, nxy=4, discrete=True, perturb=0.0)
    P = problem(orc, w)
    U1, t, s, rc = P.run(w.psi, P.prim_to_cons(w.W), nsteps=30)
    u = P.eos(U1)[0]
    z = (np.arange(n) + 0.5) * w.h
    c = math.sqrt(w.gamma * 0.2)
    below = z < 0.8 - c * t - 3.0 * math.sqrt(s) * w.h
    assert below.sum() >= n // 3
    assert np.abs(u[:, below]).max() <= 1e-12


# ------------------------------------------------------ gas-vacuum T4

def test_gas_vacuum_front(orc):
    gold = json.load(open(os.path.join(GOLD, "paper_vacuum_front.json")))
    n = 400
    w = wl.vacuum_tube(nx=n, t_end=0.1)
    P = problem(orc, w)
    U1, t, s, rc = P.run(w.psi, P.prim_to_cons(w.W), t_end=w.t_end)
    assert rc == 0 and np.isfinite(U1).all()
    u, p, phi, vac = P.eos(U1)
    assert (U1[0] >= 0).all() and (p >= 0).all()
    x = (np.arange(n) + 0.5) / n
    line = U1[0, 0, 0]
    # density at the diaphragm: the fixed point (3/4)^3
    i0 = n // 2
    rho_x0 = 0.5 * (line[i0 - 1] + line[i0])
    assert rho_x0 == pytest.approx(gold["fixed_point_rho"], rel=0.02)
    # against the exact solution in L1, and the rarefaction head at -c t
    rho_ex, u_ex, p_ex = orc.riemann_sample(w.gamma, (1, 0, 1), (0, 0, 0), (x - 0.5) / t)
    assert np.abs(line - rho_ex).mean() < 0.01
    c = math.sqrt(w.gamma)
    head = 0.5 - c * t
    assert abs(line[x < head - 0.05] - 1.0).max() < 1e-4
    # gas front: last cell holding appreciable gas trails the exact front
    front = x[np.where(line > 1e-3)[0][-1]]
    exact_front = 0.5 + 2 * c / (w.gamma - 1) * t
    assert exact_front - 0.15 < front <= exact_front + 2.0 / n


# -------------------------------------------------- second order T5

def test_smooth_wave_second_order(orc):
    gold = json.load(open(os.path.join(GOLD, "paper_smooth_wave.json")))
    errs = []
    ns = (32, 64, 128, 256)
    for n in ns:
        w = wl.smooth_wave(nx=n, amp=0.2, t_end=1.0)
        P = problem(orc, w)
        U1, t, s, rc = P.run(w.psi, P.prim_to_cons(w.W), t_end=1.0)
        errs.append(np.abs(U1[0, 0, 0] - w.W[0, 0, 0]).mean())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(ns) - 1)]
    assert orders[-1] >= 1.8, (errs, orders)
    assert abs(orders[-1] - gold["order_convergence"]) < 0.3


# -------------------------------------------------------- symmetry T6

def test_blast_symmetry(orc):
    w = wl.blast(n=16, radius_cells=2.0)
    P = problem(orc, w)
    U1, t, s, rc = P.run(w.psi, P.prim_to_cons(w.W), nsteps=12)
    assert rc == 0
    r = U1[0]
    scale = np.abs(r).max()
    for ax in range(3):
        assert np.abs(r - np.flip(r, axis=ax)).max() <= 1e-12 * scale
    for perm in [(0, 2, 1), (1, 0, 2), (2, 1, 0)]:
        assert np.abs(r - np.transpose(r, perm)).max() <= 1e-12 * scale
    assert (r > 0).all()


# --------------------------------------------------------- dt and the totals

def _cons_from_prim(gamma, rho, u, p):
    """Conserved content of one cell from (rho, u, p), by the definition of E."""
    u = np.asarray(u, dtype=float)
    return [rho, rho * u[0], rho * u[1], rho * u[2], p / (gamma - 1.0) + 0.5 * rho * float(u @ u)]


def _cells(orc, gamma, cells, h=0.125, cfl=0.4):
    """A 1-row grid holding the given cells; returns (problem, U)."""
    n = len(cells)
    U = np.zeros((5, 1, 1, n))
    for i, c in enumerate(cells):
        U[:, 0, 0, i] = c
    P = orc.Problem((1, 1, n), h, gamma, [P_] * 6)
    return P, U


@pytest.mark.parametrize("gamma", [5.0 / 3.0, 1.4])
def test_dt_is_cfl_h_over_largest_axis_speed_plus_sound_speed(orc, gamma):
    # dt = CFL h / max over gas cells of (max_d |u_d| + c), c = sqrt(gamma p / rho).
    # The states are chosen so that c^2 = gamma p / rho is a perfect square:
    #  cell A: rho 4, u (0.5, -2, 1.5): max_d |u_d| = 2 while |u| = 2.55; c = 1
    #  cell B: rho 0.25, u (-1.1, 0.3, 0.8): c = 2 -> 3.1, the largest signal
    #  cell C: vacuum (rho below 1e-10) with a huge velocity m/rho: excluded
    #  cell D: kinetic energy above E: pressure floored at 0, speed = max |u_d|
    cA = 1.0
    pA = cA ** 2 * 4.0 / gamma
    cB = 2.0
    pB = cB ** 2 * 0.25 / gamma
    cells = [_cons_from_prim(gamma, 4.0, (0.5, -2.0, 1.5), pA),
             _cons_from_prim(gamma, 0.25, (-1.1, 0.3, 0.8), pB),
             [5e-11, 1e-5, 0.0, 0.0, 1.0],
             [1.0, 0.0, 0.0, -2.9, 1.0]]
    P, U = _cells(orc, gamma, cells)
    assert P.max_speed(U) == pytest.approx(1.1 + 2.0, rel=1e-14)
    assert P.dt(U, 0.4) == pytest.approx(0.4 * 0.125 / 3.1, rel=1e-14)
    # each cell alone, against its hand-computed speed
    for c, s in ((cells[0], 2.0 + cA), (cells[1], 1.1 + cB), (cells[3], 2.9)):
        Pc, Uc = _cells(orc, gamma, [c])
        assert Pc.max_speed(Uc) == pytest.approx(s, rel=1e-14)
    Pv, Uv = _cells(orc, gamma, [cells[2]])
    assert Pv.max_speed(Uv) == 0.0 and Pv.dt(Uv, 0.4) == 0.0


def test_totals_of_an_analytic_field(orc):
    # rho = 1 + x, m = (2 rho, -rho, 0.5), E = 2 + y, psi = z on a 4 x 3 x 2 grid
    # of spacing h = 1/4 with centres at (i + 1/2) h.  The six totals are sums
    # of polynomials over the centres, written here with exact fractions:
    #   mass = h^3 sum (1 + x), px = 2 mass, py = -mass, pz = 0.5 h^3 N,
    #   E = h^3 sum (2 + y), E + rho psi = E + h^3 sum (1 + x) z.
    from fractions import Fraction as Fr
    nx, ny, nz = 4, 3, 2
    h = Fr(1, 4)
    xs = [(i + Fr(1, 2)) * h for i in range(nx)]
    ys = [(j + Fr(1, 2)) * h for j in range(ny)]
    zs = [(k + Fr(1, 2)) * h for k in range(nz)]
    vol = h ** 3
    mass = vol * sum(1 + x for x in xs for _ in ys for _ in zs)
    energy = vol * sum(2 + y for _ in xs for y in ys for _ in zs)
    pot = vol * sum((1 + x) * z for x in xs for _ in ys for z in zs)
    want = [mass, 2 * mass, -mass, Fr(1, 2) * vol * nx * ny * nz, energy, energy + pot]
    U = np.zeros((5, nz, ny, nx))
    psi = np.zeros((nz, ny, nx))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                rho = 1 + float(xs[i])
                U[:, k, j, i] = [rho, 2 * rho, -rho, 0.5, 2 + float(ys[j])]
                psi[k, j, i] = float(zs[k])
    P = orc.Problem((nz, ny, nx), float(h), 1.4, [P_] * 6)
    got = P.totals(psi, U)
    for g, wv in zip(got, want):
        assert g == pytest.approx(float(wv), rel=1e-14, abs=1e-15)

"""Seeded synthetic initial conditions for the CSPH-TVD solver.

Each recipe returns a :class:`Workload`: grid shape (nz, ny, nx), cell size h,
adiabatic index, boundary types for the faces (-x, +x, -y, +y, -z, +z), the
primitive fields W = (rho, u, v, w, p) as float64 arrays of shape
(5, nz, ny, nx), the potential psi of shape (nz, ny, nx), and the run length.
These are initial data only: the module contains none of the scheme's
arithmetic, and both the CUDA path and the CPU oracle start from the same
primitive arrays, each converting them to conserved form on its own.

The problems are the paper's test problems (Sec. 2.3 and Sec. 3 of
arXiv 1912.04855): shock tubes, a hydrostatic atmosphere at rest in a
potential, supersonic flow through a potential well, outflow into vacuum,
and a point blast.  The domain is the unit cube with the origin at a corner
and cell centres at (i + 1/2) h unless stated otherwise.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PERIODIC, OUTFLOW, INFLOW, WALL = 0, 1, 2, 3


@dataclasses.dataclass
class Workload:
    name: str
    shape: tuple  # (nz, ny, nx)
    h: float
    gamma: float
    bc: list  # 6 ints, faces -x,+x,-y,+y,-z,+z
    W: np.ndarray  # (5, nz, ny, nx) primitive rho,u,v,w,p
    psi: np.ndarray  # (nz, ny, nx)
    inflow: list = dataclasses.field(default_factory=lambda: [[0.0] * 5 for _ in range(6)])
    cfl: float = 0.4
    steps: int = 100
    t_end: float = math.inf
    note: str = ""

    @property
    def cells(self) -> int:
        nz, ny, nx = self.shape
        return nx * ny * nz


def centres(n: int, h: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * h


def splitmix64_uniform(seed: int, count: int) -> np.ndarray:
    """U(-1, 1) from SplitMix64 (Steele, Lea & Flood 2014) keyed by the cell
    index: output k uses state seed + (k + 1) * 0x9E3779B97F4A7C15."""
    with np.errstate(over="ignore"):
        k = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 / 9007199254740992.0) - 1.0


def shock_tube(nx=128, ny=16, nz=16, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), x0=0.4,
               gamma=1.4, axis=0, steps=200, cfl=0.4, t_end=math.inf, name="sod"):
    """Riemann problem along ``axis`` (0 = x): states (rho, u_normal, p); outflow
    on the two faces normal to the axis, periodic on the others.  The default
    is Sod's tube with the diaphragm at x0 = 0.4 so that 200 steps at CFL 0.4
    keep the shock inside the unit interval."""
    shape = (nz, ny, nx)
    n_axis = (nx, ny, nz)[axis]
    h = 1.0 / n_axis
    s = centres(n_axis, h)
    L = s < x0
    prof = [np.where(L, left[0], right[0]), np.where(L, left[1], right[1]),
            np.where(L, left[2], right[2])]
    bshape = [1, 1, 1]
    bshape[2 - axis] = n_axis
    W = np.zeros((5,) + shape)
    W[0] = prof[0].reshape(bshape)
    W[1 + axis] = prof[1].reshape(bshape)
    W[4] = prof[2].reshape(bshape)
    bc = [PERIODIC] * 6
    bc[2 * axis] = bc[2 * axis + 1] = OUTFLOW
    return Workload(name, shape, h, gamma, bc, W, np.zeros(shape), steps=steps, cfl=cfl,
                    t_end=t_end, note=f"{name}: Riemann problem along axis {axis}, x0={x0}")


def hydrostatic(n=128, nxy=None, H=0.2, g=1.0, gamma=1.4, z_vac=0.8, perturb=1e-6, seed=12345,
                discrete=True, steps=500, cfl=0.4, top_bc=OUTFLOW):
    """Isothermal atmosphere at rest in psi = g z: p = g H rho, rho ~ exp(-z/H),
    vacuum (rho = p = 0) above z_vac.  Periodic in x and y, reflecting wall at
    z = 0, ``top_bc`` (outflow by default) at z = 1.

    ``discrete=True`` uses the scheme's discrete equilibrium for a 27-point
    central gradient with phi = sqrt(2p): phi_{k+1} - phi_{k-1} = -(h/H) phi_k,
    i.e. rho_k = rho_0 lam^(2k) with lam = sqrt(a^2 + 1) - a, a = h/(2H); the
    first cell takes rho_0 = exp(-h/(2H)).  ``discrete=False`` samples the
    continuous profile exp(-z/H) at the cell centres.  ``perturb`` multiplies
    rho by (1 + perturb * U(-1,1)) with U from SplitMix64(seed, cell index)."""
    nxy = n if nxy is None else nxy
    shape = (n, nxy, nxy)
    h = 1.0 / n
    z = centres(n, h)
    if discrete:
        a = h / (2.0 * H)
        lam2 = (math.sqrt(a * a + 1.0) - a) ** 2
        rho_z = math.exp(-h / (2.0 * H)) * lam2 ** np.arange(n, dtype=np.float64)
    else:
        rho_z = np.exp(-z / H)
    gas = z < z_vac
    rho_z = np.where(gas, rho_z, 0.0)
    rho = np.broadcast_to(rho_z[:, None, None], shape).copy()
    p = g * H * rho
    if perturb:
        rho = rho * (1.0 + perturb * splitmix64_uniform(seed, rho.size).reshape(shape))
    W = np.zeros((5,) + shape)
    W[0] = rho
    W[4] = p
    psi = np.broadcast_to((g * z)[:, None, None], shape).copy()
    bc = [PERIODIC, PERIODIC, PERIODIC, PERIODIC, WALL, top_bc]
    return Workload("hydrostatic", shape, h, gamma, bc, W, psi, steps=steps, cfl=cfl,
                    note=f"isothermal atmosphere H={H}, g={g}, vacuum above z={z_vac}, "
                         f"{'discrete' if discrete else 'continuous'} profile, "
                         f"perturbation {perturb} (SplitMix64 seed {seed})")


def potential_well(n=256, ny=None, nz=None, psi0=2.0, sigma=0.1, mach=3.0, gamma=5.0 / 3.0,
                   rho=1.0, p=1.0, steps=1000, cfl=0.4):
    """Supersonic flow through a gravitational well psi = -psi0 exp(-r^2/(2 sigma^2))
    centred in the unit cube.  Uniform inflow at x = 0 (rho, p, Mach along
    x), outflow at x = 1, periodic in y and z; the initial state is the
    inflow state everywhere (3D form of the paper's Fig. 1 problem)."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    shape = (nz, ny, n)
    h = 1.0 / n
    u = mach * math.sqrt(gamma * p / rho)
    x = centres(n, h)
    y = (np.arange(ny) + 0.5) * h + 0.5 * (1.0 - ny * h)
    zc = (np.arange(nz) + 0.5) * h + 0.5 * (1.0 - nz * h)
    r2 = ((x - 0.5) ** 2)[None, None, :] + ((y - 0.5) ** 2)[None, :, None] + ((zc - 0.5) ** 2)[:, None, None]
    psi = -psi0 * np.exp(-r2 / (2.0 * sigma * sigma))
    W = np.zeros((5,) + shape)
    W[0] = rho
    W[1] = u
    W[4] = p
    inflow = [[0.0] * 5 for _ in range(6)]
    inflow[0] = [rho, u, 0.0, 0.0, p]
    bc = [INFLOW, OUTFLOW, PERIODIC, PERIODIC, PERIODIC, PERIODIC]
    return Workload("potential_well", shape, h, gamma, bc, W, np.ascontiguousarray(psi), inflow=inflow,
                    steps=steps, cfl=cfl,
                    note=f"potential well psi0={psi0}, sigma={sigma}, inflow Mach {mach}, gamma={gamma:.4f}")


def developed_well(n=256, ny=None, nz=None, seed=7, noise=1e-3, **kw):
    """A state shaped like the potential-well flow some way into its run, for
    one-step and windowed checks at full size: the :func:`potential_well`
    problem (same grid, potential, gamma and boundaries) with the gas
    compressed and turned toward the axis around the well and a bow-shock
    surface downstream of it.  Not a solution of the equations, only a 3D
    input with the features of one: a smooth compression, transverse
    velocities, a sharp jump across a curved surface, and seeded noise
    (SplitMix64, relative amplitude `noise`) that breaks every symmetry.
      cloud:  rho = 1 + 1.2 exp(-r^2 / (2 (1.5 sigma)^2)), p = rho^gamma,
              u = u_in (1 - 0.25 exp(...)), (v, w) = -0.3 u_in (y, z) exp(...) / (2 sigma)
      shock:  behind x - 1/2 = 0.08 + 3 ((y - 1/2)^2 + (z - 1/2)^2):
              rho x 2.2, p x 3.5, u x 0.45."""
    w = potential_well(n=n, ny=ny, nz=nz, **kw)
    nzz, nyy, nxx = w.shape
    sig = kw.get("sigma", 0.1)
    x = centres(nxx, w.h) - 0.5
    y = (np.arange(nyy) + 0.5) * w.h + 0.5 * (1.0 - nyy * w.h) - 0.5
    z = (np.arange(nzz) + 0.5) * w.h + 0.5 * (1.0 - nzz * w.h) - 0.5
    X, Y, Z = x[None, None, :], y[None, :, None], z[:, None, None]
    r2 = X * X + Y * Y + Z * Z
    g = np.exp(-r2 / (2.0 * (1.5 * sig) ** 2))
    u_in = w.inflow[0][1]
    rho = 1.0 + 1.2 * g
    p = rho ** w.gamma
    u = u_in * (1.0 - 0.25 * g)
    v = -0.3 * u_in * Y * g / (2.0 * sig)
    ww = -0.3 * u_in * Z * g / (2.0 * sig)
    behind = X > 0.08 + 3.0 * (Y * Y + Z * Z)
    rho = np.where(behind, 2.2 * rho, rho)
    p = np.where(behind, 3.5 * p, p)
    u = np.where(behind, 0.45 * u, u)
    N = w.cells
    W = np.zeros((5,) + w.shape)
    W[0] = rho * (1.0 + noise * splitmix64_uniform(seed, N).reshape(w.shape))
    W[1] = u * (1.0 + noise * splitmix64_uniform(seed + 1, N).reshape(w.shape))
    W[2] = v + 0.0 * X
    W[3] = ww + 0.0 * X
    W[4] = p * (1.0 + noise * splitmix64_uniform(seed + 2, N).reshape(w.shape))
    w.W = np.ascontiguousarray(W)
    w.name = "developed_well"
    w.note = "potential-well flow with a compression cloud and a bow-shock surface (synthetic)"
    return w


def developed_blast(n=512, radius=0.15, seed=11, noise=1e-3, rho_s=6.0, p_s=0.2, u_s=0.4, **kw):
    """A state shaped like the point blast well into its run, for one-step and
    windowed checks at full size: the :func:`blast` problem (grid, gamma,
    outflow faces) with a spherical shock of the given radius around the
    centre.  Inside, density rises to the shell, rho = max(rho_s (r/R)^6,
    0.01), pressure falls from the centre to p_s at the shell,
    p = p_s (1.6 - 0.6 (r/R)^2), and the gas moves radially outward at
    u_s r / R; outside lies the cold, still background (rho = 1,
    p = 1e-5).  Seeded noise (SplitMix64, relative amplitude `noise`) on
    density and pressure breaks the symmetries."""
    w = blast(n=n, **kw)
    c = centres(n, w.h) - 0.5
    X, Y, Z = c[None, None, :], c[None, :, None], c[:, None, None]
    r = np.sqrt(X * X + Y * Y + Z * Z)
    q = r / radius
    inside = q <= 1.0
    N = w.cells
    W = np.zeros((5,) + w.shape)
    W[0] = np.where(inside, np.maximum(rho_s * q ** 6, 0.01), 1.0)
    W[4] = np.where(inside, p_s * (1.6 - 0.6 * q * q), 1e-5)
    ur = np.where(inside, u_s * q, 0.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        inv = np.where(r > 0.0, 1.0 / np.where(r > 0.0, r, 1.0), 0.0)
    W[1] = ur * X * inv
    W[2] = ur * Y * inv
    W[3] = ur * Z * inv
    W[0] *= 1.0 + noise * splitmix64_uniform(seed, N).reshape(w.shape)
    W[4] *= 1.0 + noise * splitmix64_uniform(seed + 1, N).reshape(w.shape)
    w.W = np.ascontiguousarray(W)
    w.name = "developed_blast"
    w.note = f"point blast with a spherical shock at r = {radius} (synthetic)"
    return w


def potential_well_1d(n=100, half_width=5.0, a=1.0, psi0=-80.0, mach=10.0, gamma=5.0 / 3.0, rho=1.0,
                      c=1.0, t_end=100.0, cfl=0.4):
    """The paper's one-dimensional supersonic flow through a potential well
    psi = psi0 exp(-x^2/a^2) (Sec. 2.3, Fig. 1): x in [-half_width, half_width],
    n cells, uniform inflow (rho, u = mach * c, p = rho c^2 / gamma) at the
    left face and everywhere at t = 0, outflow at the right face; one cell in
    y and z, periodic."""
    shape = (1, 1, n)
    h = 2.0 * half_width / n
    x = -half_width + centres(n, h)
    u = mach * c
    p = rho * c * c / gamma
    psi = (psi0 * np.exp(-x * x / (a * a)))[None, None, :]
    W = np.zeros((5,) + shape)
    W[0] = rho
    W[1] = u
    W[4] = p
    inflow = [[0.0] * 5 for _ in range(6)]
    inflow[0] = [rho, u, 0.0, 0.0, p]
    bc = [INFLOW, OUTFLOW, PERIODIC, PERIODIC, PERIODIC, PERIODIC]
    return Workload("potential_well_1d", shape, h, gamma, bc, W, np.ascontiguousarray(psi), inflow=inflow,
                    t_end=t_end, steps=10 ** 9, cfl=cfl,
                    note=f"1D potential well psi0={psi0}, a={a}, x in [-{half_width}, {half_width}], inflow Mach {mach}")


def blast(n=512, E=1.0, radius_cells=3.0, rho=1.0, p_bg=1e-5, gamma=1.4, t_end=0.05, cfl=0.4):
    """Point blast: uniform rho and background pressure; the energy E is spread
    uniformly (as internal energy) over the cells whose centres lie within
    radius_cells * h of the cube centre.  Outflow on every face."""
    shape = (n, n, n)
    h = 1.0 / n
    c = centres(n, h) - 0.5
    r2 = c[None, None, :] ** 2 + c[None, :, None] ** 2 + c[:, None, None] ** 2
    hot = r2 <= (radius_cells * h) ** 2
    cnt = int(hot.sum())
    p = np.full(shape, p_bg)
    p[hot] += (gamma - 1.0) * E / (cnt * h ** 3)
    W = np.zeros((5,) + shape)
    W[0] = rho
    W[4] = p
    return Workload("blast", shape, h, gamma, [OUTFLOW] * 6, W, np.zeros(shape), t_end=t_end,
                    steps=10 ** 9, cfl=cfl,
                    note=f"point blast E={E} over {cnt} cells within {radius_cells}h, p_bg={p_bg}")


def vacuum_tube(nx=1000, ny=1, nz=1, x0=0.5, gamma=5.0 / 3.0, t_end=0.3, cfl=0.4):
    """Gas (rho = p = 1, u = 0) left of x0 and vacuum (rho = p = 0) right of it;
    outflow in x, periodic in y and z (the paper's Fig. 2 problem)."""
    shape = (nz, ny, nx)
    h = 1.0 / nx
    x = centres(nx, h)
    W = np.zeros((5,) + shape)
    W[0] = np.where(x < x0, 1.0, 0.0)[None, None, :]
    W[4] = np.where(x < x0, 1.0, 0.0)[None, None, :]
    bc = [OUTFLOW, OUTFLOW, PERIODIC, PERIODIC, PERIODIC, PERIODIC]
    return Workload("vacuum_tube", shape, h, gamma, bc, W, np.zeros(shape), t_end=t_end,
                    steps=10 ** 9, cfl=cfl, note=f"gas-vacuum tube x0={x0}")


def smooth_wave(nx=64, ny=1, nz=1, amp=0.2, u=1.0, p=1.0, gamma=1.4, t_end=1.0, cfl=0.4):
    """rho = 1 + amp sin(2 pi x), uniform u and p, periodic everywhere: the
    exact solution is pure translation with speed u."""
    shape = (nz, ny, nx)
    h = 1.0 / nx
    x = centres(nx, h)
    W = np.zeros((5,) + shape)
    W[0] = (1.0 + amp * np.sin(2.0 * math.pi * x))[None, None, :]
    W[1] = u
    W[4] = p
    return Workload("smooth_wave", shape, h, gamma, [PERIODIC] * 6, W, np.zeros(shape), t_end=t_end,
                    steps=10 ** 9, cfl=cfl, note=f"smooth density wave amp={amp}, u={u}")


def random_state(shape, seed=0, rho=(0.5, 1.5), vel=0.3, p=(0.5, 1.5), gamma=1.4, bc=None, psi_amp=0.0,
                 h=None):
    """Smooth-ish random state for parity tests: independent uniform draws per
    cell (numpy PCG64 seeded), optional random potential."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    h = 1.0 / max(shape) if h is None else h
    W = np.zeros((5,) + tuple(shape))
    W[0] = rng.uniform(*rho, size=shape)
    W[1:4] = rng.uniform(-vel, vel, size=(3,) + tuple(shape))
    W[4] = rng.uniform(*p, size=shape)
    psi = psi_amp * rng.uniform(-1.0, 1.0, size=shape)
    bc = [PERIODIC] * 6 if bc is None else bc
    inflow = [[0.0] * 5 for _ in range(6)]
    for f in range(6):
        if bc[f] == INFLOW:
            inflow[f] = [1.0, 0.2 * (1 if f % 2 == 0 else -1) if f // 2 == 0 else 0.1, 0.05, -0.05, 1.0]
    return Workload("random", tuple(shape), h, gamma, list(bc), W, psi, inflow=inflow, steps=10)


def serving_stream(n_requests=64, mean_gap_s=0.020, seed=2024, edges=(32, 64, 96, 128, 192), steps=200):
    """Request stream for the serving loop: Poisson arrivals and, per request,
    a seeded Riemann problem or potential-well flow on an edge^3 grid.
    Returns a list of dicts (arrival time, kind, parameters); the grids are
    built on demand with :func:`request_workload`."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(n_requests):
        t += rng.exponential(mean_gap_s)
        edge = int(rng.choice(edges))
        gamma = float(rng.choice([1.4, 5.0 / 3.0]))
        if r % 2 == 0:
            params = dict(kind="riemann", edge=edge, gamma=gamma,
                          left=(float(rng.uniform(0.1, 1.0)), 0.0, float(rng.uniform(0.1, 1.0))),
                          right=(float(rng.uniform(0.1, 1.0)), 0.0, float(rng.uniform(0.1, 1.0))),
                          x0=float(rng.uniform(0.3, 0.7)))
        else:
            params = dict(kind="well", edge=edge, gamma=gamma, psi0=float(rng.uniform(0.5, 3.0)),
                          mach=float(rng.uniform(1.5, 4.0)))
        out.append(dict(id=r, arrival=t, steps=steps, **params))
    return out


def request_workload(req) -> Workload:
    e = req["edge"]
    if req["kind"] == "riemann":
        return shock_tube(e, e, e, left=req["left"], right=req["right"], x0=req["x0"], gamma=req["gamma"],
                          steps=req["steps"], name="riemann")
    return potential_well(e, psi0=req["psi0"], mach=req["mach"], gamma=req["gamma"], steps=req["steps"])

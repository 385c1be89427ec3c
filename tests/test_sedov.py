"""Point blast against the Sedov-Taylor similarity solution.

The similarity constant xi0 of R(t) = xi0 (E t^2/rho)^(1/5) is computed here
by integrating the self-similar Euler equations (continuity, momentum,
entropy) inward from the strong-shock conditions and evaluating the energy
integral -- independent of the oracle and of the CUDA path -- and is itself
pinned against the published constants.  The blast radius is measured as
the outer half-maximum of the spherically averaged density jump.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1912_04855_b300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def sedov_xi0(g, n=100000, eta_min=1e-4):
    """u = Rdot U(eta), rho = rho0 D(eta), p = rho0 Rdot^2 P(eta), eta = r/R,
    R ~ t^(2/5); RK4 from eta = 1 (strong shock) to eta_min; energy
    E = rho0 (4/25) (R^5/t^2) I with I = int 4 pi eta^2 (D U^2/2 + P/(g-1))."""
    def f(eta, y):
        U, D, P = y
        w = U - eta
        Up = (1.5 * U * w + 2 * g * P * U / (D * eta) - 3 * P / D) / (w * w - g * P / D)
        Dp = -D * (2 * U / eta + Up) / w
        Pp = P * (g * Dp / D + 3 / w)
        return np.array([Up, Dp, Pp])

    def e(eta, y):
        U, D, P = y
        return 4 * math.pi * eta * eta * (0.5 * D * U * U + P / (g - 1))

    y = np.array([2 / (g + 1), (g + 1) / (g - 1), 2 / (g + 1)])
    eta, h = 1.0, -(1 - eta_min) / n
    I, fa = 0.0, e(1.0, y)
    for _ in range(n):
        k1 = f(eta, y)
        k2 = f(eta + h / 2, y + h / 2 * k1)
        k3 = f(eta + h / 2, y + h / 2 * k2)
        k4 = f(eta + h, y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        eta += h
        fb = e(eta, y)
        I += -h * 0.5 * (fa + fb)
        fa = fb
    return (25 / (4 * I)) ** 0.2


def _front_radius(rho, r, h):
    """Outer half-maximum of the density binned by radius r (bins of width h)."""
    nb = int(r.max() / h) + 1
    idx = (r / h).astype(np.int64).ravel()
    prof = np.bincount(idx, weights=rho.ravel(), minlength=nb)[:nb] / np.maximum(
        np.bincount(idx, minlength=nb)[:nb], 1)
    rc = (np.arange(nb) + 0.5) * h
    ip = int(np.argmax(prof))
    half = 1 + 0.5 * (prof[ip] - 1)
    j = ip + int(np.where(prof[ip:] < half)[0][0])
    return rc[j - 1] + (half - prof[j - 1]) / (prof[j] - prof[j - 1]) * h


def _radii(n, h):
    c = (np.arange(n) + 0.5) * h - 0.5 * n * h
    return np.sqrt(c[None, None, :] ** 2 + c[None, :, None] ** 2 + c[:, None, None] ** 2)


def blast_radius(rho, h):
    """Outer half-maximum of the spherically averaged density around the
    cube centre (cells binned by radius, width h, out to half the edge)."""
    n = rho.shape[0]
    r = _radii(n, h)
    inside = r < 0.5 * n * h
    return _front_radius(rho[inside], r[inside], h)


def octant_radii(rho, h):
    """The same front radius measured in each of the eight octants alone."""
    n = rho.shape[0]
    m = n // 2
    r = _radii(n, h)
    out = []
    for sz in (slice(0, m), slice(m, n)):
        for sy in (slice(0, m), slice(m, n)):
            for sx in (slice(0, m), slice(m, n)):
                ro, rr = rho[sz, sy, sx], r[sz, sy, sx]
                inside = rr < 0.5 * n * h
                out.append(_front_radius(ro[inside], rr[inside], h))
    return np.array(out)


def test_similarity_constant_matches_published_values():
    g = json.load(open(os.path.join(GOLD, "sedov_constants.json")))
    for gam, ref in g["xi0"].items():
        assert sedov_xi0(float(gam), n=20000) == pytest.approx(ref, rel=1e-3)


def test_oracle_blast_follows_sedov_taylor(orc):
    n = 32
    xi0 = sedov_xi0(1.4, n=20000)
    w = wl.blast(n=n)
    P = orc.Problem(w.shape, w.h, w.gamma, w.bc, inflow=w.inflow)
    U = P.prim_to_cons(w.W)
    E0 = P.totals(w.psi, U)[4]
    radii = []
    for t in (0.03, 0.05):
        U, tt, s, rc = P.run(w.psi, U, t_end=t, t0=0.0 if t == 0.03 else 0.03)
        assert rc == 0
        radii.append(blast_radius(U[0], w.h))
        assert radii[-1] == pytest.approx(xi0 * (t * t) ** 0.2, rel=0.03)
    assert radii[1] / radii[0] == pytest.approx((0.05 / 0.03) ** 0.4, rel=0.03)
    ro = octant_radii(U[0], w.h)
    assert ro.max() - ro.min() <= 1e-9 * ro.mean(), ro  # FP64: mirror cells agree to rounding
    assert P.totals(w.psi, U)[4] == pytest.approx(E0, rel=1e-12)  # energy stays inside the box


@pytest.mark.gpu
def test_blast_512_fp32_follows_sedov_taylor():
    """The point-blast configuration at full size: 512^3, FP32 fused path
    with an autotuned tile depth, to t = 0.05: radius within 1.5 % of the
    similarity law, total energy conserved (FP64 totals), and symmetry under
    reflections and axis permutations.

    Symmetry is tested where it is well conditioned.  The front is one to two
    cells wide and the density jumps sixfold across it, so a rounding-level
    shift of the front decides whether a given cell is already shocked: two
    mirror cells on the front may differ by the whole jump.  The front
    position itself is stable, so the eight octants' front radii must agree
    to 1e-4.  Inside the shell (r < R/2) the fields are smooth and mirror
    cells must agree pointwise.  The scheme amplifies the mirror-asymmetric
    rounding of the first steps (in FP64 as in FP32: about twentyfold over
    3000 steps of this problem), so the pointwise bound is 5e-3 of the peak
    density rather than the FP32 unit roundoff."""
    from paper_1912_04855_b300 import cspht
    n = 512
    w = wl.blast(n=n)
    with cspht.Sim.from_workload(w, precision=32, path=cspht.PATH_FAST) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        assert s.autotune(steps=3, cfl=0.4) >= 1  # tile depth for this grid (state unchanged)
        E0 = s.totals()[4]
        steps = s.run(0.05, 0.4)
        E1 = s.totals()[4]
        rho = s.get_state()[0]
    assert steps > 0 and abs(E1 - E0) <= 1e-5 * E0
    R = blast_radius(rho, w.h)
    assert R == pytest.approx(sedov_xi0(1.4, n=20000) * 0.05 ** 0.4, rel=0.015)
    ro = octant_radii(rho, w.h)
    assert (ro.max() - ro.min()) <= 1e-4 * R, ro
    scale = rho.max()
    core = _radii(n, w.h) < 0.5 * R
    for ax in range(3):
        assert np.abs(rho - np.flip(rho, axis=ax))[core].max() <= 5e-3 * scale
    assert np.abs(rho - np.transpose(rho, (2, 1, 0)))[core].max() <= 5e-3 * scale

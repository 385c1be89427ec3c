"""Pins of the exact Riemann solver (test infrastructure for the shock-tube
and gas-vacuum checks of Sec. 2.3) against a textbook table and against the
jump conditions and invariants that define the exact solution."""
import json
import math
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_sod_star_state_matches_toro_table(orc):
    g = json.load(open(os.path.join(GOLD, "toro_sod_star.json")))
    ps, us = orc.riemann_star(g["gamma"], g["left"], g["right"])
    assert round(ps, 5) == g["p_star"]
    assert round(us, 5) == g["u_star"]
    s = np.array([us - 1e-9, us + 1e-9])
    rho, u, p = orc.riemann_sample(g["gamma"], g["left"], g["right"], s)
    assert round(rho[0], 5) == g["rho_star_left"]
    assert round(rho[1], 5) == g["rho_star_right"]


@pytest.mark.parametrize("WL,WR", [((1, 0, 1), (0.125, 0, 0.1)), ((1, -2, 0.4), (1, 2, 0.4)),
                                   ((1, 0, 1000), (1, 0, 0.01)), ((5.99924, 19.5975, 460.894),
                                                                  (5.99242, -6.19633, 46.095))])
def test_rankine_hugoniot_and_riemann_invariants(orc, WL, WR):
    g = 1.4
    ps, us = orc.riemann_star(g, WL, WR)
    s = np.linspace(-40, 40, 40001)
    rho, u, p = orc.riemann_sample(g, WL, WR, s)
    c = np.sqrt(g * p / rho)
    for side, W, sign in ((0, WL, -1), (1, WR, +1)):
        r0, u0, p0 = W
        if ps > p0:  # shock: mass, momentum, energy fluxes continuous in the shock frame
            rs = rho[np.searchsorted(s, us) - 1] if side == 0 else rho[np.searchsorted(s, us) + 1]
            S = (rs * us - r0 * u0) / (rs - r0)
            E0 = p0 / (g - 1) + 0.5 * r0 * u0 ** 2
            Es = ps / (g - 1) + 0.5 * rs * us ** 2
            f0 = np.array([r0 * (u0 - S), r0 * u0 * (u0 - S) + p0, E0 * (u0 - S) + p0 * u0])
            fs = np.array([rs * (us - S), rs * us * (us - S) + ps, Es * (us - S) + ps * us])
            np.testing.assert_allclose(fs, f0, rtol=1e-9, atol=1e-9 * max(1, abs(f0).max()))
        else:  # rarefaction: u -/+ 2c/(g-1) and p/rho^g constant through the fan
            c0 = math.sqrt(g * p0 / r0)
            J = u0 - sign * 2 * c0 / (g - 1)
            head = u0 + sign * c0
            cs = c0 * (ps / p0) ** ((g - 1) / (2 * g))
            tail = us + sign * cs
            lo, hi = sorted((head, tail))
            m = (s > lo) & (s < hi)
            if m.any():
                np.testing.assert_allclose(u[m] - sign * 2 * c[m] / (g - 1), J, rtol=1e-10, atol=1e-10)
                np.testing.assert_allclose(p[m] / rho[m] ** g, p0 / r0 ** g, rtol=1e-10)


def test_vacuum_fixed_point_closed_form(orc):
    g = json.load(open(os.path.join(GOLD, "paper_vacuum_front.json")))
    gam = g["gamma"]
    rho, u, p = orc.riemann_sample(gam, (1, 0, 1), (0, 0, 0), np.array([0.0, -1.3, 3.88, 3.86]))
    assert rho[0] == pytest.approx(g["fixed_point_rho"], rel=1e-14)
    assert rho[0] * u[0] == pytest.approx(0.421875 * 0.75 * math.sqrt(5 / 3), rel=1e-14)
    assert rho[1] == 1.0  # ahead of the head -c = -1.29099
    assert rho[2] == 0.0  # beyond the escape front 3c = 3.87298
    assert rho[3] > 0.0

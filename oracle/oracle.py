"""TEST INFRASTRUCTURE ONLY: ctypes binding of the FP64 CPU oracle.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this module.  The product package never does.

The oracle is the plain C definition of the CSPH-TVD step in
``cspht_oracle.c`` (Sec. 2.2, Eqs. 4-8 of arXiv 1912.04855) plus the exact
Riemann solver in ``exact_riemann.c``.  State arrays are numpy float64 of
shape (5, nz, ny, nx) (rho, mx, my, mz, E), potential psi of shape
(nz, ny, nx).
"""
from __future__ import annotations

import ctypes
import ctypes.util
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SOURCES = ["cspht_oracle.c", "exact_riemann.c"]

BC_PERIODIC, BC_OUTFLOW, BC_INFLOW, BC_WALL = 0, 1, 2, 3
LIM_VANLEER, LIM_MINMOD, LIM_MC = 0, 1, 2
RIEMANN_LF, RIEMANN_HLL, RIEMANN_SWEPT, RIEMANN_HLLC = 0, 1, 2, 3


class Cfg(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("h", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("rho_vac", ctypes.c_double),
        ("bc", ctypes.c_int * 6),
        ("inflow", (ctypes.c_double * 5) * 6),
        ("limiter", ctypes.c_int),
        ("riemann", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, FP64, no FMA contraction)."""
    srcs = [os.path.join(HERE, s) for s in SOURCES + ["cspht_oracle.h"]]
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(LIB) >= newest:
            return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", LIB] + [os.path.join(HERE, s) for s in SOURCES] + ["-lm"]
    subprocess.check_call(cmd)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        D, I, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        L.orc_gtilde.restype = D
        L.orc_gtilde.argtypes = [D]
        L.orc_norm_C.restype = D
        L.orc_norm_C.argtypes = []
        L.orc_step.restype = I
        L.orc_step.argtypes = [P, P, P, D, P, P]
        L.orc_max_speed.restype = D
        L.orc_max_speed.argtypes = [P, P]
        L.orc_dt.restype = D
        L.orc_dt.argtypes = [P, P, D]
        L.orc_run.restype = I
        L.orc_run.argtypes = [P, P, P, ctypes.c_long, D, D, P, P]
        L.orc_totals.restype = None
        L.orc_totals.argtypes = [P, P, P, P]
        L.orc_prim_to_cons.restype = None
        L.orc_prim_to_cons.argtypes = [D, P, P, ctypes.c_long]
        L.orc_eos.restype = None
        L.orc_eos.argtypes = [P, P, P, P, P, P]
        L.orc_force.restype = I
        L.orc_force.argtypes = [P, P, P, P, D, P]
        L.orc_lagrange.restype = I
        L.orc_lagrange.argtypes = [P, P, P, D, P, P, P, P]
        L.orc_riemann_star.restype = I
        L.orc_riemann_star.argtypes = [D] * 7 + [P, P]
        L.orc_riemann_sample.restype = I
        L.orc_riemann_sample.argtypes = [D] * 7 + [P, ctypes.c_long, P, P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Problem:
    """Grid, gas and boundary description (mirrors the oracle's ``orc_cfg``)."""

    def __init__(self, shape, h, gamma, bc, inflow=None, rho_vac=1e-10, limiter=0, riemann=0):
        nz, ny, nx = shape
        self.shape = (nz, ny, nx)
        self.cfg = Cfg()
        self.cfg.n[0], self.cfg.n[1], self.cfg.n[2] = nx, ny, nz
        self.cfg.h, self.cfg.gamma, self.cfg.rho_vac = h, gamma, rho_vac
        for f in range(6):
            self.cfg.bc[f] = int(bc[f])
            for c in range(5):
                self.cfg.inflow[f][c] = float(inflow[f][c]) if inflow is not None else 0.0
        self.cfg.limiter, self.cfg.riemann = limiter, riemann

    @property
    def N(self):
        nz, ny, nx = self.shape
        return nx * ny * nz

    def _cp(self):
        return ctypes.byref(self.cfg)

    def prim_to_cons(self, W) -> np.ndarray:
        W = _f64(W)
        U = np.empty_like(W)
        lib().orc_prim_to_cons(self.cfg.gamma, _p(W), _p(U), self.N)
        return U

    def eos(self, U):
        U = _f64(U)
        u = np.empty((3,) + self.shape)
        p = np.empty(self.shape)
        phi = np.empty(self.shape)
        vac = np.empty(self.shape, dtype=np.int32)
        lib().orc_eos(self._cp(), _p(U), _p(u), _p(p), _p(phi), _p(vac))
        return u, p, phi, vac.astype(bool)

    def max_speed(self, U) -> float:
        return lib().orc_max_speed(self._cp(), _p(_f64(U)))

    def dt(self, U, cfl) -> float:
        return lib().orc_dt(self._cp(), _p(_f64(U)), cfl)

    def step(self, psi, U, dt, box=None, out=None) -> np.ndarray:
        """One step; with ``box`` = ((x0,x1),(y0,y1),(z0,z1)) only that window is
        computed (the rest of the returned array is a copy of ``U``).  With
        ``out`` (a C-contiguous float64 array of U's shape) the result is
        written there and only the window's cells are touched."""
        psi, U = _f64(psi), _f64(U)
        if out is None:
            out = U.copy()
        elif not (out.dtype == np.float64 and out.flags["C_CONTIGUOUS"] and out.shape == U.shape):
            raise ValueError("out must be a C-contiguous float64 array of U's shape")
        bp = None
        if box is not None:
            b = np.array([box[0][0], box[0][1], box[1][0], box[1][1], box[2][0], box[2][1]],
                         dtype=np.int32)
            bp = _p(b)
        rc = lib().orc_step(self._cp(), _p(psi), _p(U), float(dt), _p(out), bp)
        if rc not in (0, -4):
            raise RuntimeError(f"orc_step failed: {rc}")
        return out

    def run(self, psi, U, nsteps=-1, cfl=0.4, t_end=float("inf"), t0=0.0):
        """Advance with dt from the CFL rule; returns (U, t, steps, rc)."""
        psi = _f64(psi)
        U = _f64(U).copy()
        t = ctypes.c_double(t0)
        s = ctypes.c_long(0)
        rc = lib().orc_run(self._cp(), _p(psi), _p(U), int(nsteps), float(cfl), float(t_end),
                           ctypes.byref(t), ctypes.byref(s))
        return U, t.value, s.value, rc

    def totals(self, psi, U) -> np.ndarray:
        out = np.empty(6)
        lib().orc_totals(self._cp(), _p(_f64(psi)), _p(_f64(U)), _p(out))
        return out

    def force(self, psi, U, xi=None, dt=0.0) -> np.ndarray:
        Q = np.empty((4,) + self.shape)
        xp = _p(_f64(xi)) if xi is not None else None
        keep = _f64(xi) if xi is not None else None
        if keep is not None:
            xp = _p(keep)
        rc = lib().orc_force(self._cp(), _p(_f64(psi)), _p(_f64(U)), xp, float(dt), _p(Q))
        if rc:
            raise RuntimeError(f"orc_force failed: {rc}")
        return Q

    def lagrange(self, psi, U, dt):
        Us = np.empty((5,) + self.shape)
        Un = np.empty((5,) + self.shape)
        xs = np.empty((3,) + self.shape)
        xn = np.empty((3,) + self.shape)
        rc = lib().orc_lagrange(self._cp(), _p(_f64(psi)), _p(_f64(U)), float(dt), _p(Us), _p(xs),
                                _p(Un), _p(xn))
        if rc:
            raise RuntimeError(f"orc_lagrange failed: {rc}")
        return Us, xs, Un, xn


def _gomp():
    lib()  # the oracle's library pulls in the OpenMP runtime
    return ctypes.CDLL(ctypes.util.find_library("gomp") or "libgomp.so.1")


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle's cell loops use from now on."""
    _gomp().omp_set_num_threads(int(n))


def max_threads() -> int:
    """Threads the oracle's parallel loops would use now."""
    return int(_gomp().omp_get_max_threads())


def gtilde(q: float) -> float:
    return lib().orc_gtilde(q)


def norm_C() -> float:
    return lib().orc_norm_C()


def riemann_star(gamma, WL, WR):
    ps, us = ctypes.c_double(), ctypes.c_double()
    rc = lib().orc_riemann_star(gamma, *WL, *WR, ctypes.byref(ps), ctypes.byref(us))
    if rc:
        raise ValueError("no star state (vacuum generated or invalid input)")
    return ps.value, us.value


def riemann_sample(gamma, WL, WR, s):
    s = _f64(s)
    rho, u, p = np.empty_like(s), np.empty_like(s), np.empty_like(s)
    rc = lib().orc_riemann_sample(gamma, *WL, *WR, _p(s), s.size, _p(rho), _p(u), _p(p))
    if rc:
        raise ValueError("invalid Riemann problem")
    return rho, u, p

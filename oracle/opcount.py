"""TEST AND MEASUREMENT INFRASTRUCTURE ONLY: floating-point operations per
cell of one CSPH-TVD step, counted by running the oracle's own code
(``cspht_oracle.c``, compiled unchanged by ``opcount.cpp`` with a counting
number type).

Run ``python oracle/opcount.py`` from the repository root.  It writes
``profiles/flop_count.json``, which the benchmark reads for the algorithmic
operation counts of its roofline.  Two states are counted:

- ``general``: a smooth state increasing along every axis in every conserved
  component (outflow faces, a linear potential).  Every limiter then takes its
  nonzero branch, so the count is the per-cell arithmetic of the general
  path, which the GPU kernels (written without data-dependent branches)
  execute for every cell.  This is the count the benchmark uses.
- ``developed_well``: the benchmark grid's flow, shaped like a developed run
  (workloads.developed_well), for comparison; uniform regions there take the
  limiter's cheap zero branch.

Counting rule (see opcount.cpp): an operation (one add, subtract, multiply,
divide or square root; the oracle has no fused multiply-adds, so a
multiply-add counts 2 as in the FLOP convention) is counted when its result
depends on the cell state; operations on run constants (h, gamma, C, the
lattice geometry, the static potential) or on the step's dt alone are folded.
Each value the method defines is counted once with the oracle's arithmetic
for it (the oracle's repeated face fluxes and slopes are removed).  Negation,
absolute values and comparisons are not counted.
"""
from __future__ import annotations

import ctypes
import json
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libopcount.so")
OUT = os.path.join(ROOT, "profiles", "flop_count.json")
# run as a script, this directory comes first on the path and its oracle.py
# would shadow the package of the same name
sys.path[:] = [p for p in sys.path if os.path.abspath(p or ".") != HERE]
sys.path.insert(0, ROOT)


def build(force=False):
    srcs = [os.path.join(HERE, f) for f in ("opcount.cpp", "cspht_oracle.c", "cspht_oracle.h")]
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(map(os.path.getmtime, srcs)):
        return LIB
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-Wno-unknown-pragmas", "-o", LIB,
                           os.path.join(HERE, "opcount.cpp")])
    return LIB


def general_state(n=40):
    """A smooth state increasing along x, y and z in every conserved
    component: rho, u, v, w and p all rise linearly; outflow faces."""
    from paper_1912_04855_b300 import workloads as wl
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    X, Y, Z = c[None, None, :], c[None, :, None], c[:, None, None]
    s = X + 0.9 * Y + 0.8 * Z
    W = np.zeros((5, n, n, n))
    W[0] = 1.0 + 0.5 * s
    W[1] = 0.3 + 0.2 * s
    W[2] = 0.2 + 0.15 * s
    W[3] = 0.1 + 0.1 * s
    W[4] = 1.0 + 0.7 * s
    psi = 0.3 * (X + Y + Z) + 0.0 * s
    return wl.Workload("general", (n, n, n), h, 5.0 / 3.0, [wl.OUTFLOW] * 6, W, np.ascontiguousarray(psi))


def count(w, cfl=0.4):
    from oracle import oracle as O
    P = O.Problem(w.shape, w.h, w.gamma, w.bc, inflow=w.inflow)
    U = P.prim_to_cons(w.W)
    dt = P.dt(U, cfl)
    L = ctypes.CDLL(build())
    L.orc_opcount.restype = ctypes.c_int
    L.orc_opcount.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                              ctypes.c_char_p]
    tmp = OUT + ".tmp"
    psi = np.ascontiguousarray(w.psi, dtype=np.float64)
    U = np.ascontiguousarray(U)
    rc = L.orc_opcount(ctypes.byref(P.cfg), psi.ctypes.data_as(ctypes.c_void_p),
                       U.ctypes.data_as(ctypes.c_void_p), dt, tmp.encode())
    if rc:
        raise RuntimeError(f"orc_opcount failed: {rc}")
    d = json.load(open(tmp))
    os.remove(tmp)
    return d


def main():
    from paper_1912_04855_b300 import workloads as wl
    res = {
        "what": "floating-point operations per cell of one CSPH-TVD step, counted by running the "
                "oracle's code with a counting number type (oracle/opcount.cpp)",
        "command": "python oracle/opcount.py",
        "rule": "an add, sub, mul, div or sqrt (1 op each; the oracle has no fused multiply-adds) is "
                "counted when its result depends on the cell state; operations on run constants "
                "(h, gamma, C, lattice geometry, static psi) or on the step's dt alone are folded; "
                "each value the method defines counted once (the oracle's repeated face fluxes and "
                "slopes removed); negation, fabs and compares not counted",
        "states": {},
    }
    g = general_state(40)
    res["states"]["general"] = dict(count(g), note="smooth state rising along every axis in every "
                                    "component, outflow faces: every limiter on its nonzero branch")
    dw = wl.developed_well(n=40)
    res["states"]["developed_well"] = dict(count(dw), note="potential-well flow shaped like a developed "
                                           "run (workloads.developed_well), 40^3")
    res["bench_uses"] = "general"
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1)
        f.write("\n")
    s = res["states"]["general"]
    print(f"wrote {OUT}: lagrange {s['lagrange_kernel']['flops']:.1f}, euler {s['euler_kernel']['flops']:.1f}, "
          f"step {s['step']['flops']:.1f} flops per cell")


if __name__ == "__main__":
    main()

"""The C-ABI library loads, exports every entry point its header declares, and
rejects invalid arguments before touching a device (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1912_04855_b300 import cspht

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(cspht_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_abi():
    names = declared()
    for n in ["cspht_create", "cspht_step", "cspht_run", "cspht_totals", "cspht_set_state",
              "cspht_get_state", "cspht_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    L = cspht.lib()
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    L = cspht.lib()
    for n in declared():
        assert getattr(L, n).argtypes is not None or n == "cspht_default_opts", n


@pytest.mark.parametrize("kw,shape", [
    (dict(bc=(0, 1, 0, 0, 0, 0)), (4, 4, 4)),          # periodic must pair
    (dict(bc=(1, 1, 0, 0, 0, 0)), (4, 4, 1)),          # non-periodic axis needs >= 2 cells
    (dict(precision=16), (4, 4, 4)),
    (dict(limiter=7), (4, 4, 4)),
    (dict(riemann=5), (4, 4, 4)),
    (dict(riemann=4), (4, 4, 4)),          # 0..3: LF, HLL, swept, HLLC (= HLL)
    (dict(bc=(9, 9, 0, 0, 0, 0)), (4, 4, 4)),
])
def test_create_rejects_invalid_arguments(kw, shape):
    with pytest.raises(cspht.CsphtError) as e:
        cspht.Sim(shape, 0.25, 1.4, np.zeros(shape), **kw)
    assert e.value.code == cspht.EINVAL


def test_create_rejects_bad_physics():
    for h, g in [(0.0, 1.4), (0.1, 1.0), (-1.0, 1.4)]:
        with pytest.raises(cspht.CsphtError) as e:
            cspht.Sim((4, 4, 4), h, g, np.zeros((4, 4, 4)))
        assert e.value.code == cspht.EINVAL


def test_null_handle_calls_are_safe():
    L = cspht.lib()
    assert L.cspht_step(None, 0.4, None) == cspht.EINVAL
    assert L.cspht_totals(None, None) == cspht.EINVAL
    assert L.cspht_launch_count(None) == -1
    buf = np.zeros(5, dtype=np.float32)
    ptr = buf.ctypes.data_as(ctypes.c_void_p)
    for f in (L.cspht_upload_f32_async, L.cspht_download_f32_async, L.cspht_set_state_f32,
              L.cspht_get_state_f32):
        assert f(None, ptr) == cspht.EINVAL
    assert L.cspht_sync(None) == cspht.EINVAL
    L.cspht_destroy(None)


@pytest.mark.parametrize("n", [(1 << 20) + 1, 0])
def test_axis_limits(n):
    """Extents outside [1, 2^20] are refused before anything is allocated."""
    L = cspht.lib()
    psi = np.zeros(8)
    out = ctypes.c_void_p()
    rc = L.cspht_create(n, 2, 2, 0.1, 1.4, psi.ctypes.data_as(ctypes.c_void_p), None, None, ctypes.byref(out))
    assert rc == cspht.EINVAL and not out.value


@pytest.mark.parametrize("shape", [(4, 4, 65534), (2048, 2048, 600), (40000, 40000, 4)])
def test_grids_beyond_32_bit_offsets_or_the_launch_limit_are_refused(shape):
    """nz above the launch grid's limit, or padded arrays of 2^31 elements or
    more (the fused kernels use 32-bit offsets), give CSPHT_EINVAL before any
    allocation -- the check does not read psi -- and cspht_device_bytes
    reports -1 for them."""
    L = cspht.lib()
    psi = np.zeros(8)
    out = ctypes.c_void_p()
    nx, ny, nz = shape
    rc = L.cspht_create(nx, ny, nz, 0.1, 1.4, psi.ctypes.data_as(ctypes.c_void_p), None, None, ctypes.byref(out))
    assert rc == cspht.EINVAL and not out.value
    assert L.cspht_device_bytes(nx, ny, nz, None) == -1


def test_largest_allowed_grid_is_sized():
    """A grid just inside the 32-bit offset limit has a positive footprint."""
    L = cspht.lib()
    assert L.cspht_device_bytes(1024, 1024, 1000, None) > 0

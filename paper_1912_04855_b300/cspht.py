"""ctypes binding of ``libcspht.so`` -- the C ABI declared in ``include/cspht.h``.

Argument marshalling only: every step of the CSPH-TVD update runs in the
library's CUDA kernels.  Importing works without a GPU; creating a solver
needs the built library and a CUDA device and raises :class:`CsphtError`
otherwise (there is no CPU fallback).

State arrays are float64 of shape (5, nz, ny, nx) in C order (rho, mx, my,
mz, E), i.e. the ABI's structure-of-arrays with x fastest.  Host buffers may
be numpy arrays or pinned torch CPU tensors.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ECFL, ENEGATIVE, ESTATE, ETOOBIG = 0, -1, -2, -3, -4, -5, -6, -7, -8
BC_PERIODIC, BC_OUTFLOW, BC_INFLOW, BC_WALL = 0, 1, 2, 3
RIEMANN_LF, RIEMANN_HLL, RIEMANN_SWEPT, RIEMANN_HLLC = 0, 1, 2, 3
BALANCE_PLAIN, BALANCE_COMPENSATED = 0, 1
LIMITER_VANLEER, LIMITER_MINMOD, LIMITER_MC = 0, 1, 2
PATH_FAST, PATH_PLAIN = 0, 1

_NAMES = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", ENONFINITE: "ENONFINITE",
          ECFL: "ECFL", ENEGATIVE: "ENEGATIVE", ESTATE: "ESTATE", ETOOBIG: "ETOOBIG"}


class CsphtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cspht {_NAMES.get(code, code)}: {msg}")
        self.code = code


class cspht_bcs(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int * 6), ("inflow", (ctypes.c_double * 5) * 6)]


class cspht_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("riemann", ctypes.c_int), ("limiter", ctypes.c_int),
                ("path", ctypes.c_int), ("rho_vac", ctypes.c_double), ("balance", ctypes.c_int)]


_lib = None
LIB_PATH = _build.LIB


def lib():
    """Loads libcspht.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        try:
            _build.build()
        except Exception as e:  # no nvcc: use an existing build if there is one
            if not os.path.exists(LIB_PATH):
                raise CsphtError(ECUDA, f"libcspht.so is not built and the build failed: {e}")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D, L64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long
        sig = {
            "cspht_default_opts": (None, [P]),
            "cspht_create": (I, [I, I, I, D, D, P, P, P, P]),
            "cspht_set_state": (I, [P, P]),
            "cspht_set_primitive": (I, [P, P]),
            "cspht_get_state": (I, [P, P]),
            "cspht_set_state_f32": (I, [P, P]),
            "cspht_get_state_f32": (I, [P, P]),
            "cspht_upload_f32_async": (I, [P, P]),
            "cspht_download_f32_async": (I, [P, P]),
            "cspht_step": (I, [P, D, P]),
            "cspht_advance": (I, [P, L64, D]),
            "cspht_sync": (I, [P]),
            "cspht_batch_step": (I, [P, I, D, P]),
            "cspht_autotune": (I, [P, I, D, P]),
            "cspht_set_tile_depth": (I, [P, I]),
            "cspht_test_copy_timeout": (I, [P, I]),
            "cspht_run": (I, [P, D, D, P]),
            "cspht_totals": (I, [P, P]),
            "cspht_set_stream": (I, [P, P]),
            "cspht_time": (D, [P]),
            "cspht_launch_count": (ctypes.c_longlong, [P]),
            "cspht_profile": (I, [P, I]),
            "cspht_profile_read": (I, [P, I, P, P, ctypes.c_char_p, I]),
            "cspht_step_noalloc_f32": (I, [I, I, I, D, D, P, P, P, P, D, P, P]),
            "cspht_device_bytes": (ctypes.c_longlong, [I, I, I, P]),
            "cspht_probe_fma": (I, [I, I, P, P]),
            "cspht_batch_create": (I, [P, I, I, P]),
            "cspht_batch_advance": (I, [P, L64, D, P]),
            "cspht_batch_launch_count": (ctypes.c_longlong, [P]),
            "cspht_batch_last_error": (ctypes.c_char_p, [P]),
            "cspht_batch_destroy": (None, [P]),
            "cspht_last_error": (ctypes.c_char_p, [P]),
            "cspht_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _is_f32(a) -> bool:
    if hasattr(a, "data_ptr"):
        return str(a.dtype) == "torch.float32"
    return isinstance(a, np.ndarray) and a.dtype == np.float32


def _ptr(a, nbytes=None, item=8):
    """Host pointer of a C-contiguous numpy array or torch CPU tensor of float64
    (item = 8) or float32 (item = 4)."""
    want_t, want_n = ("torch.float64", np.float64) if item == 8 else ("torch.float32", np.float32)
    if hasattr(a, "data_ptr"):
        if str(a.dtype) != want_t or not a.is_contiguous() or a.is_cuda:
            raise CsphtError(EINVAL, f"expected a contiguous {want_t} CPU tensor")
        if nbytes is not None and a.numel() * item != nbytes:
            raise CsphtError(EINVAL, "tensor has the wrong size")
        return ctypes.c_void_p(a.data_ptr())
    if not (isinstance(a, np.ndarray) and a.dtype == want_n and a.flags["C_CONTIGUOUS"]):
        raise CsphtError(EINVAL, f"expected a C-contiguous {np.dtype(want_n).name} numpy array")
    if nbytes is not None and a.nbytes != nbytes:
        raise CsphtError(EINVAL, f"array has {a.nbytes} bytes, expected {nbytes}")
    return a.ctypes.data_as(ctypes.c_void_p)


def batch_step(sims, cfl, stream):
    """One step of every Sim in `sims`, concurrently, forked from and joined
    back into `stream` (a torch.cuda.Stream or a raw cudaStream_t); capturable
    into a CUDA graph on `stream`."""
    raw = getattr(stream, "cuda_stream", stream)
    arr = (ctypes.c_void_p * max(1, len(sims)))(*[s._h for s in sims])
    rc = lib().cspht_batch_step(arr, len(sims), float(cfl), ctypes.c_void_p(raw))
    if rc != OK:
        msgs = "; ".join(s.last_error() for s in sims if s.last_error())
        raise CsphtError(rc, f"batch_step: {msgs or 'failed'}")


class Batch:
    """Several Sims advanced together, one launch of each step kernel for all
    of them (``cspht_batch_*``).  The Sims must outlive the batch."""

    def __init__(self, sims, depth=0):
        self.sims = list(sims)
        arr = (ctypes.c_void_p * max(1, len(self.sims)))(*[s._h for s in self.sims])
        h = ctypes.c_void_p()
        rc = lib().cspht_batch_create(arr, len(self.sims), int(depth), ctypes.byref(h))
        if rc != OK:
            raise CsphtError(rc, "cspht_batch_create failed")
        self._h = h

    def advance(self, nsteps, cfl=0.4, stream=None):
        raw = getattr(stream, "cuda_stream", stream)
        rc = lib().cspht_batch_advance(self._h, int(nsteps), float(cfl), ctypes.c_void_p(raw) if raw else None)
        if rc != OK:
            raise CsphtError(rc, "batch advance: " + lib().cspht_batch_last_error(self._h).decode())

    def launch_count(self) -> int:
        return lib().cspht_batch_launch_count(self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib().cspht_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


PROBE_FP32, PROBE_FP32X2, PROBE_FP64 = 0, 1, 2


def probe_fma(kind, trips):
    """Measured multiply-add throughput of the current GPU (the library's own
    probe kernel, cspht_probe_fma): returns (TFLOP/s, milliseconds)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    rc = lib().cspht_probe_fma(int(kind), int(trips), ctypes.byref(tf), ctypes.byref(ms))
    if rc != OK:
        raise CsphtError(ECUDA, f"cspht_probe_fma failed ({rc})")
    return tf.value, ms.value


def device_bytes(shape, precision=64, path=PATH_FAST) -> int:
    """Device bytes a handle for this grid would allocate (no allocation)."""
    nz, ny, nx = (int(x) for x in shape)
    o = cspht_opts()
    lib().cspht_default_opts(ctypes.byref(o))
    o.precision, o.path = precision, path
    n = lib().cspht_device_bytes(nx, ny, nz, ctypes.byref(o))
    if n < 0:
        raise CsphtError(EINVAL, "cspht_device_bytes: invalid grid or options")
    return n


def step_noalloc_f32(shape, h, gamma, U, psi, U_out, cfl=0.4, bc=(0,) * 6, inflow=None, stream=None):
    """One FP32 step with ``cspht_step_noalloc_f32`` on caller-owned device
    buffers (torch CUDA float32 tensors or raw device pointers): ``U`` and
    ``U_out`` hold 5*N floats, ``psi`` N floats.  The library allocates no
    device memory for it (see the header).  Returns dt; raises on a non-OK
    status."""
    nz, ny, nx = (int(s) for s in shape)
    b = cspht_bcs()
    for f in range(6):
        b.type[f] = int(bc[f])
        for c in range(5):
            b.inflow[f][c] = float(inflow[f][c]) if inflow is not None else 0.0

    def dptr(t):
        return ctypes.c_void_p(t.data_ptr() if hasattr(t, "data_ptr") else int(t))

    raw = getattr(stream, "cuda_stream", stream)
    dt = ctypes.c_double()
    rc = lib().cspht_step_noalloc_f32(nx, ny, nz, float(h), float(gamma), ctypes.byref(b), dptr(U),
                                      dptr(psi), dptr(U_out), float(cfl), ctypes.byref(dt),
                                      ctypes.c_void_p(raw) if raw else None)
    if rc != OK:
        raise CsphtError(rc, "cspht_step_noalloc_f32 failed")
    return dt.value


class Sim:
    """One solver handle (``cspht_t``)."""

    def __init__(self, shape, h, gamma, psi, bc=(0,) * 6, inflow=None, precision=64,
                 riemann=RIEMANN_LF, limiter=LIMITER_VANLEER, path=PATH_FAST, rho_vac=1e-10,
                 balance=BALANCE_PLAIN):
        L = lib()
        self.shape = tuple(int(s) for s in shape)
        nz, ny, nx = self.shape
        self.N = nx * ny * nz
        self.precision = precision
        b = cspht_bcs()
        for f in range(6):
            b.type[f] = int(bc[f])
            for c in range(5):
                b.inflow[f][c] = float(inflow[f][c]) if inflow is not None else 0.0
        o = cspht_opts()
        L.cspht_default_opts(ctypes.byref(o))
        o.precision, o.riemann, o.limiter, o.path, o.rho_vac = precision, riemann, limiter, path, rho_vac
        o.balance = balance
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        h_ = ctypes.c_void_p()
        rc = L.cspht_create(nx, ny, nz, float(h), float(gamma), _ptr(psi, 8 * self.N),
                            ctypes.byref(b), ctypes.byref(o), ctypes.byref(h_))
        if rc != OK:
            raise CsphtError(rc, "cspht_create failed")
        self._h = h_

    @classmethod
    def from_workload(cls, w, **kw):
        return cls(w.shape, w.h, w.gamma, w.psi, bc=w.bc, inflow=w.inflow, **kw)

    def _check(self, rc, what):
        if rc != OK:
            msg = lib().cspht_last_error(self._h).decode()
            raise CsphtError(rc, f"{what}: {msg}")

    def set_state(self, U):
        """Upload the conserved state (5 x N SoA, float64, or float32 for half the bytes)."""
        if _is_f32(U):
            self._check(lib().cspht_set_state_f32(self._h, _ptr(U, 20 * self.N, 4)), "set_state")
        else:
            self._check(lib().cspht_set_state(self._h, _ptr(U, 40 * self.N)), "set_state")

    def set_primitive(self, W):
        self._check(lib().cspht_set_primitive(self._h, _ptr(W, 40 * self.N)), "set_primitive")

    def get_state(self, out=None):
        """Download the conserved state into `out` (float64, or float32 for half
        the bytes; a new float64 array if None)."""
        if out is None:
            out = np.empty((5,) + self.shape)
        if _is_f32(out):
            self._check(lib().cspht_get_state_f32(self._h, _ptr(out, 20 * self.N, 4)), "get_state")
        else:
            self._check(lib().cspht_get_state(self._h, _ptr(out, 40 * self.N)), "get_state")
        return out

    def upload_async(self, U):
        """Enqueue the upload of a float32 conserved state (5 x N SoA, host,
        page-locked for overlap); returns at once.  U must stay unchanged
        until sync()."""
        self._check(lib().cspht_upload_f32_async(self._h, _ptr(U, 20 * self.N, 4)), "upload_async")

    def download_async(self, out):
        """Enqueue the download of the state into float32 `out` (5 x N SoA,
        host); `out` holds it after sync()."""
        self._check(lib().cspht_download_f32_async(self._h, _ptr(out, 20 * self.N, 4)), "download_async")

    def step(self, cfl=0.4) -> float:
        dt = ctypes.c_double()
        self._check(lib().cspht_step(self._h, float(cfl), ctypes.byref(dt)), "step")
        return dt.value

    def advance(self, nsteps, cfl=0.4):
        self._check(lib().cspht_advance(self._h, int(nsteps), float(cfl)), "advance")

    def sync(self):
        self._check(lib().cspht_sync(self._h), "sync")

    def run(self, t_end, cfl=0.4) -> int:
        s = ctypes.c_long()
        self._check(lib().cspht_run(self._h, float(t_end), float(cfl), ctypes.byref(s)), "run")
        return s.value

    def totals(self) -> np.ndarray:
        out = np.empty(6)
        self._check(lib().cspht_totals(self._h, _ptr(out)), "totals")
        return out

    def autotune(self, steps=5, cfl=0.4) -> int:
        """Times the fused step per candidate tile depth and keeps the fastest
        (state unchanged); returns the chosen depth in planes (0 if unfused)."""
        z = ctypes.c_int()
        self._check(lib().cspht_autotune(self._h, int(steps), float(cfl), ctypes.byref(z)), "autotune")
        return z.value

    def set_tile_depth(self, zchunk: int):
        """Planes per CTA column of the fused kernels (results do not depend on it)."""
        self._check(lib().cspht_set_tile_depth(self._h, int(zchunk)), "set_tile_depth")

    def test_copy_timeout(self, polls: int):
        """Failure-detection test hook: with polls > 0 the fused kernels issue no
        tile copy and each copy wait gives up after `polls` polls; 0 turns it off."""
        self._check(lib().cspht_test_copy_timeout(self._h, int(polls)), "test_copy_timeout")

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t (int) or None."""
        raw = getattr(stream, "cuda_stream", stream)
        self._check(lib().cspht_set_stream(self._h, ctypes.c_void_p(raw) if raw else None),
                    "set_stream")

    def time(self) -> float:
        t = lib().cspht_time(self._h)
        if math.isnan(t):
            self._check(ECUDA, "time")
        return t

    def launch_count(self) -> int:
        return lib().cspht_launch_count(self._h)

    def profile(self, enable=True):
        self._check(lib().cspht_profile(self._h, 1 if enable else 0), "profile")

    def profile_read(self) -> dict:
        """{kernel kind: (total ms, launches)} of the launches since profile(True)."""
        n = 32
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        names = ctypes.create_string_buffer(1024)
        k = lib().cspht_profile_read(self._h, n, ms, cnt, names, 1024)
        if k < 0:
            self._check(k, "profile_read")
        kinds = names.value.decode().split(";")
        return {kinds[i]: (ms[i], cnt[i]) for i in range(k) if cnt[i]}

    def last_error(self) -> str:
        return lib().cspht_last_error(self._h).decode()

    def close(self):
        if getattr(self, "_h", None):
            lib().cspht_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

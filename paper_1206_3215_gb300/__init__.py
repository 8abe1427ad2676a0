"""Python binding of ``libpss.so``, the GB300 pseudospectral time-stepping library.

Argument marshalling only: every step runs in the library's CUDA kernels.  The
functions carry the C names of ``include/pss.h``; :class:`Grid` wraps a handle
for numpy (host) or torch (device) arrays.  Importing this module does not need
the library; the first call does, and fails loudly if it is missing or cannot
be loaded.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PSS_LIBRARY", os.path.join(_HERE, "libpss.so"))

PSS_OK, PSS_E_ARG, PSS_E_OOM, PSS_E_CUDA, PSS_E_NOT_CONVERGED, PSS_E_NONFINITE, PSS_E_STATE = range(7)
PSS_EQ_NLS, PSS_EQ_SG, PSS_EQ_NS = 0, 1, 2
PSS_FP32, PSS_FP64 = 0, 1
PSS_HOST, PSS_DEVICE = 0, 1
PSS_NS_CN, PSS_NS_MIDPOINT = 0, 1

EXPORTED = [
    "pss_default_params", "pss_create_grid", "pss_set_state", "pss_step_n", "pss_get_state",
    "pss_conserved_quantities", "pss_stats", "pss_checkpoint_size", "pss_checkpoint_save",
    "pss_checkpoint_load", "pss_sync", "pss_destroy", "pss_last_error", "pss_fft2d",
    "pss_version", "pss_set_profiling", "pss_profile_read", "pss_nls_invariants_static",
    "pss_set_field", "pss_get_field", "pss_set_state_sg_levels", "pss_step_n_batch", "pss_autotune",
    "pss_fma_rate",
]


class PssParams(ctypes.Structure):
    """Mirror of ``struct pss_params``."""
    _fields_ = [
        ("eq", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("batch", ctypes.c_int64),
        ("x0", ctypes.c_double), ("y0", ctypes.c_double),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("dt", ctypes.c_double), ("sigma", ctypes.c_double), ("nu", ctypes.c_double),
        ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("dealias", ctypes.c_int32),
        ("stream", ctypes.c_void_p), ("scheme", ctypes.c_int32), ("rfft", ctypes.c_int32),
    ]


class PssError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pss error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpss.so; raises if it has not been built (no CPU fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "or python paper_1206_3215_gb300/build.py")
        lib = ctypes.CDLL(path)
        P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        sig = {
            "pss_default_params": (None, [P]),
            "pss_create_grid": (I, [P, P]),
            "pss_set_state": (I, [P, P, P, I]),
            "pss_step_n": (I, [P, I64]),
            "pss_get_state": (I, [P, P, P, I]),
            "pss_conserved_quantities": (I, [P, P, I, P]),
            "pss_stats": (I, [P, P, P]),
            "pss_checkpoint_size": (I, [P, P]),
            "pss_checkpoint_save": (I, [P, P, I]),
            "pss_checkpoint_load": (I, [P, P, I]),
            "pss_sync": (I, [P]),
            "pss_fma_rate": (I, [I, P, P]),
            "pss_destroy": (I, [P]),
            "pss_last_error": (ctypes.c_char_p, [P]),
            "pss_fft2d": (I, [P, I64, I64, I64, I, I, P]),
            "pss_version": (ctypes.c_char_p, []),
            "pss_set_profiling": (I, [P, I]),
            "pss_profile_read": (I, [P, P, I, P]),
            "pss_nls_invariants_static": (I, [P, P, I64, I64, I64, D, D, D, I, P, P]),
            "pss_set_field": (I, [P, I64, P, P, I]),
            "pss_get_field": (I, [P, I64, P, P, I]),
            "pss_set_state_sg_levels": (I, [P, P, P, I]),
            "pss_step_n_batch": (I, [P, I, P]),
            "pss_autotune": (I, [P, I, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(rc: int, handle=None):
    if rc != PSS_OK:
        msg = load_library().pss_last_error(handle).decode()
        raise PssError(rc, msg)


# ---- C-named entry points ----------------------------------------------------

def pss_default_params(**overrides) -> PssParams:
    p = PssParams()
    load_library().pss_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def pss_create_grid(params: PssParams) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().pss_create_grid(ctypes.byref(h), ctypes.byref(params)), None)
    return h


def pss_set_state(h, a_ptr: int, b_ptr: int | None, where: int) -> None:
    _check(load_library().pss_set_state(h, a_ptr, b_ptr, where), h)


def pss_step_n(h, n: int) -> None:
    _check(load_library().pss_step_n(h, n), h)


def pss_set_state_sg_levels(h, un_ptr: int, unm1_ptr: int, where: int) -> None:
    _check(load_library().pss_set_state_sg_levels(h, un_ptr, unm1_ptr, where), h)


def pss_step_n_batch(handles, steps) -> None:
    """Advance handles[i] by steps[i] steps (each on its own stream)."""
    count = len(handles)
    hs = (ctypes.c_void_p * max(count, 1))(*[h.value if hasattr(h, "value") else h for h in handles])
    ns = (ctypes.c_int64 * max(count, 1))(*steps)
    rc = load_library().pss_step_n_batch(hs, count, ns)
    if rc != PSS_OK:
        bad = next((h for h in handles if pss_last_error(h)), None)
        raise PssError(rc, pss_last_error(bad) if bad is not None else "pss_step_n_batch failed")


def pss_autotune(h, steps: int = 4) -> int:
    """Time both launch shapes on this grid's step; returns the kernels whose plan changed."""
    c = ctypes.c_int()
    _check(load_library().pss_autotune(h, steps, ctypes.byref(c)), h)
    return c.value


def pss_get_state(h, a_ptr: int, b_ptr: int | None, where: int) -> None:
    _check(load_library().pss_get_state(h, a_ptr, b_ptr, where), h)


def pss_set_field(h, field: int, a_ptr: int, b_ptr: int | None, where: int) -> None:
    _check(load_library().pss_set_field(h, field, a_ptr, b_ptr, where), h)


def pss_get_field(h, field: int, a_ptr: int, b_ptr: int | None, where: int) -> None:
    _check(load_library().pss_get_field(h, field, a_ptr, b_ptr, where), h)


def pss_conserved_quantities(h, cap: int = 3 * 65535) -> np.ndarray:
    out = np.zeros(cap, dtype=np.float64)
    cnt = ctypes.c_int()
    _check(load_library().pss_conserved_quantities(h, out.ctypes.data, cap, ctypes.byref(cnt)), h)
    return out[: cnt.value].copy()


def pss_stats(h):
    s, u = ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().pss_stats(h, ctypes.byref(s), ctypes.byref(u)), h)
    return s.value, u.value


def pss_checkpoint_size(h) -> int:
    n = ctypes.c_size_t()
    _check(load_library().pss_checkpoint_size(h, ctypes.byref(n)), h)
    return n.value


def pss_checkpoint_save(h, ptr: int, where: int) -> None:
    _check(load_library().pss_checkpoint_save(h, ptr, where), h)


def pss_checkpoint_load(h, ptr: int, where: int) -> None:
    _check(load_library().pss_checkpoint_load(h, ptr, where), h)


def pss_sync(h) -> None:
    _check(load_library().pss_sync(h), h)


def pss_destroy(h) -> None:
    load_library().pss_destroy(h)


def pss_last_error(h=None) -> str:
    return load_library().pss_last_error(h).decode()


def pss_fft2d(ptr: int, nx: int, ny: int, batch: int, precision: int, direction: int,
              stream: int | None = None) -> None:
    rc = load_library().pss_fft2d(ptr, nx, ny, batch, precision, direction, stream)
    if rc != PSS_OK:
        raise PssError(rc, "pss_fft2d failed")


def pss_set_profiling(h, on: bool | int) -> None:
    """0/False off; 1/True time every pass; S > 1 time the passes of every S-th step."""
    _check(load_library().pss_set_profiling(h, int(on)), h)


def pss_profile_read(h) -> dict:
    out = np.zeros(7, dtype=np.float64)
    cnt = ctypes.c_int()
    _check(load_library().pss_profile_read(h, out.ctypes.data, 7, ctypes.byref(cnt)), h)
    return {"launches": int(out[0]), "row": (int(out[1]), float(out[2])),
            "col": (int(out[3]), float(out[4])), "other": (int(out[5]), float(out[6]))}


def pss_nls_invariants_static(psi_ptr: int, hat_ptr: int, nx: int, ny: int, batch: int,
                              lx: float, ly: float, sigma: float, precision: int, out_ptr: int,
                              stream: int | None = None) -> None:
    """NLS mass and energy into a device array, with no allocation (see pss.h)."""
    _check(load_library().pss_nls_invariants_static(psi_ptr, hat_ptr, nx, ny, batch, lx, ly, sigma,
                                                     precision, out_ptr, stream), None)


def pss_fma_rate(kind: int, stream: int | None = None) -> float:
    """GFLOP/s of independent FMA chains: kind 0 FP32, 1 FP64, 2 FP32 packed pairs."""
    out = ctypes.c_double()
    _check(load_library().pss_fma_rate(kind, ctypes.byref(out), stream))
    return out.value


def pss_version() -> str:
    return load_library().pss_version().decode()


# ---- convenience wrapper -----------------------------------------------------

_EQ = {"nls": PSS_EQ_NLS, "sg": PSS_EQ_SG, "ns": PSS_EQ_NS}


class Grid:
    """One pss_grid handle.  Arrays are numpy (host) or torch CUDA tensors (device)."""

    def __init__(self, eq: str = "nls", n: int | tuple[int, int] = 64, precision: str = "fp32",
                 batch: int = 1, stream=None, **params):
        nx, ny = (n, n) if isinstance(n, int) else n
        self.eq = eq
        self.precision = precision
        self.batch = batch
        self.nx, self.ny = nx, ny
        p = pss_default_params(eq=_EQ[eq], precision=PSS_FP32 if precision == "fp32" else PSS_FP64,
                               nx=nx, ny=ny, batch=batch)
        for k, v in params.items():
            if k == "scheme" and isinstance(v, str):
                v = {"cn": PSS_NS_CN, "midpoint": PSS_NS_MIDPOINT}[v]
            setattr(p, k, v)
        if stream is not None:
            p.stream = stream
        self.params = p
        self.h = pss_create_grid(p)

    # dtypes of the state as seen by callers
    @property
    def real_dtype(self):
        return np.float32 if self.precision == "fp32" else np.float64

    @property
    def complex_dtype(self):
        return np.complex64 if self.precision == "fp32" else np.complex128

    def _shape(self):
        return (self.batch, self.ny, self.nx)

    def _prep(self, arr, complex_: bool):
        dt = self.complex_dtype if complex_ else self.real_dtype
        if arr is None:
            return None, None
        if hasattr(arr, "data_ptr"):  # torch tensor on the device
            import torch
            tdt = {np.complex64: torch.complex64, np.complex128: torch.complex128,
                   np.float32: torch.float32, np.float64: torch.float64}[dt]
            t = arr.to(tdt).contiguous()
            if t.numel() != int(np.prod(self._shape())):
                raise ValueError("bad state size")
            return t, t.data_ptr()
        a = np.ascontiguousarray(np.asarray(arr, dtype=dt))
        if a.size != int(np.prod(self._shape())):
            raise ValueError("bad state size")
        return a, a.ctypes.data

    def set_state(self, a, b=None):
        complex_ = self.eq == "nls"
        ka, pa = self._prep(a, complex_)
        kb, pb = self._prep(b, complex_)
        where = PSS_DEVICE if hasattr(a, "data_ptr") else PSS_HOST
        pss_set_state(self.h, pa, pb, where)
        self._keep = (ka, kb)  # device inputs must live until the copy ran

    def set_levels(self, u_n, u_nm1):
        """Sine-Gordon: both time levels u^n, u^{n-1} (arrays [batch][ny][nx])."""
        ka, pa = self._prep(u_n, False)
        kb, pb = self._prep(u_nm1, False)
        where = PSS_DEVICE if hasattr(u_n, "data_ptr") else PSS_HOST
        pss_set_state_sg_levels(self.h, pa, pb, where)
        self._keep = (ka, kb)

    def autotune(self, steps: int = 4) -> int:
        return pss_autotune(self.h, steps)

    def step(self, n: int):
        pss_step_n(self.h, n)

    def get_state(self):
        """Host copies: NLS psi; SG (u^n, u^{n-1}); NS omega."""
        if self.eq == "nls":
            a = np.empty(self._shape(), self.complex_dtype)
            pss_get_state(self.h, a.ctypes.data, None, PSS_HOST)
            return a
        a = np.empty(self._shape(), self.real_dtype)
        if self.eq == "sg":
            b = np.empty(self._shape(), self.real_dtype)
            pss_get_state(self.h, a.ctypes.data, b.ctypes.data, PSS_HOST)
            return a, b
        pss_get_state(self.h, a.ctypes.data, None, PSS_HOST)
        return a

    def set_field(self, field: int, a, b=None):
        """Set one field (slot) of the batch from host arrays of shape [ny][nx]."""
        complex_ = self.eq == "nls"
        dt = self.complex_dtype if complex_ else self.real_dtype
        a = np.ascontiguousarray(np.asarray(a, dtype=dt))
        bb = None if b is None else np.ascontiguousarray(np.asarray(b, dtype=dt))
        if a.size != self.nx * self.ny or (bb is not None and bb.size != a.size):
            raise ValueError("bad field size")
        pss_set_field(self.h, field, a.ctypes.data, None if bb is None else bb.ctypes.data, PSS_HOST)

    def get_field(self, field: int):
        """Host copy of one field: NLS psi; SG (u^n, u^{n-1}); NS omega."""
        shape = (self.ny, self.nx)
        if self.eq == "nls":
            a = np.empty(shape, self.complex_dtype)
            pss_get_field(self.h, field, a.ctypes.data, None, PSS_HOST)
            return a
        a = np.empty(shape, self.real_dtype)
        if self.eq == "sg":
            b = np.empty(shape, self.real_dtype)
            pss_get_field(self.h, field, a.ctypes.data, b.ctypes.data, PSS_HOST)
            return a, b
        pss_get_field(self.h, field, a.ctypes.data, None, PSS_HOST)
        return a

    def get_state_device(self, out_a, out_b=None):
        pss_get_state(self.h, out_a.data_ptr(), None if out_b is None else out_b.data_ptr(), PSS_DEVICE)

    def conserved(self) -> np.ndarray:
        per = {"nls": 2, "sg": 1, "ns": 3}[self.eq]
        return pss_conserved_quantities(self.h, cap=per * self.batch).reshape(self.batch, per)

    def stats(self):
        return pss_stats(self.h)

    def sync(self):
        pss_sync(self.h)

    def checkpoint(self) -> np.ndarray:
        buf = np.empty(pss_checkpoint_size(self.h), np.uint8)
        pss_checkpoint_save(self.h, buf.ctypes.data, PSS_HOST)
        return buf

    def restore(self, buf: np.ndarray):
        pss_checkpoint_load(self.h, np.ascontiguousarray(buf).ctypes.data, PSS_HOST)

    def close(self):
        if getattr(self, "h", None):
            pss_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

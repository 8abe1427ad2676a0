"""ctypes front end of the FP64 C oracle (``pss_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark.  Arrays are numpy ``complex128`` /
``float64`` in row-major ``[ny][nx]`` order; every function copies its input
and returns new arrays, so callers keep their data.

Each wrapper names the passage of arXiv:1206.3215 it follows; the C source
states the readings taken where the paper is silent or inconsistent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pss_oracle.c")
_HDR = os.path.join(_HERE, "pss_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

__all__ = [
    "build", "num_threads", "fft1d", "dft1d", "fft2d", "ifft2d", "wavenumbers",
    "nls_run", "nls_invariants", "sg_init", "sg_run", "sg_fields", "sg_hamiltonian",
    "ns_init", "ns_jacobian", "ns_run", "ns_field", "ns_invariants", "mutant",
]


_CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off"]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (OpenMP, -O2, no fast-math)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc"] + _CFLAGS + [_SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def mutant(edits, workdir: str):
    """A copy of this module bound to a deliberately broken oracle: the C
    source with each (old, new) text edit applied (each `old` must occur
    exactly once), compiled into `workdir`.  Used only by tests that check a
    pin fails when a plausible mistake is planted in the oracle."""
    import importlib.util
    src = open(_SRC).read()
    for old, new in edits:
        if src.count(old) != 1:
            raise ValueError(f"mutant edit target must occur once: {old!r}")
        src = src.replace(old, new)
    os.makedirs(workdir, exist_ok=True)
    csrc = os.path.join(workdir, "pss_oracle_mutant.c")
    with open(csrc, "w") as f:
        f.write(src)
    lib = os.path.join(workdir, "liboracle_mutant.so")
    subprocess.run(["gcc"] + _CFLAGS + ["-I", _HERE, csrc, "-o", lib, "-lm"], check=True)
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{abs(hash(src))}", __file__)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._LIB = lib
    mod._SRC = csrc
    mod.build = lambda force=False: lib
    return mod


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P, L, D, I = ctypes.c_void_p, ctypes.c_long, ctypes.c_double, ctypes.c_int
            sigs = {
                "orc_fft1d": [P, L, I],
                "orc_dft1d": [P, P, L, I],
                "orc_fft2d": [P, L, L, I],
                "orc_wavenumbers": [L, D, P],
                "orc_nls_run": [P, L, L, D, D, D, D, L, I],
                "orc_nls_invariants": [P, L, L, D, D, D, P, P],
                "orc_sg_init": [P, P, L, L, D, D, D, P, P],
                "orc_sg_run": [P, P, L, L, D, D, D, L],
                "orc_sg_fields": [P, P, L, L, P, P],
                "orc_sg_hamiltonian": [P, P, L, L, D, D, D, P],
                "orc_ns_init": [P, L, L, I, P],
                "orc_ns_jacobian": [P, L, L, D, D, P],
                "orc_ns_run": [P, L, L, D, D, D, D, D, L, I, L, P],
                "orc_ns_run_scheme": [P, L, L, D, D, D, D, D, L, I, L, P, I],
                "orc_ns_field": [P, L, L, P],
                "orc_ns_invariants": [P, L, L, D, D, P, P, P],
                "orc_num_threads": [],
            }
            for name, args in sigs.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.array(a, dtype=np.complex128, copy=True))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.array(a, dtype=np.float64, copy=True))


def _check(rc: int, name: str):
    if rc < 0:
        raise ValueError(f"oracle {name}: bad argument (rc={rc})")
    return rc


def num_threads() -> int:
    return _load().orc_num_threads()


# --------------------------------------------------------------------------
# Transforms (Section 4: derivatives are multiplications in Fourier space)

def fft1d(a, sign: int = -1) -> np.ndarray:
    """Radix-2 FFT, unnormalised, exponent sign ``sign``."""
    x = _c128(a)
    _check(_load().orc_fft1d(_ptr(x), x.size, sign), "fft1d")
    return x


def dft1d(a, sign: int = -1) -> np.ndarray:
    """Brute-force O(n^2) DFT, the definition itself."""
    x = _c128(a)
    out = np.empty_like(x)
    _check(_load().orc_dft1d(_ptr(x), _ptr(out), x.size, sign), "dft1d")
    return out


def fft2d(a) -> np.ndarray:
    """Forward 2D DFT (rows then columns), unnormalised."""
    x = _c128(a)
    ny, nx = x.shape
    _check(_load().orc_fft2d(_ptr(x), nx, ny, -1), "fft2d")
    return x


def ifft2d(a) -> np.ndarray:
    """Inverse 2D DFT including 1/(nx ny)."""
    x = _c128(a)
    ny, nx = x.shape
    _check(_load().orc_fft2d(_ptr(x), nx, ny, +1), "ifft2d")
    return x


def wavenumbers(n: int, L: float) -> np.ndarray:
    k = np.empty(n, dtype=np.float64)
    _check(_load().orc_wavenumbers(n, L, _ptr(k)), "wavenumbers")
    return k


# --------------------------------------------------------------------------
# NLS: Eq. 1 with Strang splitting, Section 4.1; invariants Eq. 2

def nls_run(psi, lx: float, ly: float, dt: float, nsteps: int, sigma: float = 1.0,
            merged: bool = False) -> np.ndarray:
    x = _c128(psi)
    ny, nx = x.shape
    _check(_load().orc_nls_run(_ptr(x), nx, ny, lx, ly, dt, sigma, nsteps, int(merged)),
           "nls_run")
    return x


def nls_invariants(psi, lx: float, ly: float, sigma: float = 1.0):
    """(mass, energy) of Eq. 2 with the sigma reading of Eq. 1."""
    x = _c128(psi)
    ny, nx = x.shape
    m, e = ctypes.c_double(), ctypes.c_double()
    _check(_load().orc_nls_invariants(_ptr(x), nx, ny, lx, ly, sigma, ctypes.byref(m),
                                      ctypes.byref(e)), "nls_invariants")
    return m.value, e.value


# --------------------------------------------------------------------------
# Sine-Gordon: Eq. 3, semi-implicit leapfrog of Section 4.2

def sg_init(u0, v0, lx: float, ly: float, dt: float):
    """(uhat^0, uhat^-1) from u(0), u_t(0) by a backward Taylor step."""
    u, v = _f64(u0), _f64(v0)
    ny, nx = u.shape
    un = np.empty((ny, nx), np.complex128)
    um = np.empty((ny, nx), np.complex128)
    _check(_load().orc_sg_init(_ptr(u), _ptr(v), nx, ny, lx, ly, dt, _ptr(un), _ptr(um)),
           "sg_init")
    return un, um


def sg_run(uhat_n, uhat_nm1, lx: float, ly: float, dt: float, nsteps: int):
    a, b = _c128(uhat_n), _c128(uhat_nm1)
    ny, nx = a.shape
    _check(_load().orc_sg_run(_ptr(a), _ptr(b), nx, ny, lx, ly, dt, nsteps), "sg_run")
    return a, b


def sg_fields(uhat_n, uhat_nm1):
    a, b = _c128(uhat_n), _c128(uhat_nm1)
    ny, nx = a.shape
    un = np.empty((ny, nx)); um = np.empty((ny, nx))
    _check(_load().orc_sg_fields(_ptr(a), _ptr(b), nx, ny, _ptr(un), _ptr(um)), "sg_fields")
    return un, um


def sg_hamiltonian(uhat_n, uhat_nm1, lx: float, ly: float, dt: float) -> float:
    a, b = _c128(uhat_n), _c128(uhat_nm1)
    ny, nx = a.shape
    h = ctypes.c_double()
    _check(_load().orc_sg_hamiltonian(_ptr(a), _ptr(b), nx, ny, lx, ly, dt, ctypes.byref(h)),
           "sg_hamiltonian")
    return h.value


# --------------------------------------------------------------------------
# Navier-Stokes: Section 3.3 equations, Crank-Nicolson + fixed point (Section 4.3)

def ns_init(w0, dealias: bool = True) -> np.ndarray:
    w = _f64(w0)
    ny, nx = w.shape
    out = np.empty((ny, nx), np.complex128)
    _check(_load().orc_ns_init(_ptr(w), nx, ny, int(dealias), _ptr(out)), "ns_init")
    return out


def ns_jacobian(what, lx: float, ly: float) -> np.ndarray:
    """J = psi_y w_x - psi_x w_y in physical space."""
    a = _c128(what)
    ny, nx = a.shape
    J = np.empty((ny, nx))
    _check(_load().orc_ns_jacobian(_ptr(a), nx, ny, lx, ly, _ptr(J)), "ns_jacobian")
    return J


def ns_run(what, lx: float, ly: float, nu: float, dt: float, nsteps: int, tol: float = 1e-10,
           max_iter: int = 100, dealias: bool = True, scheme: str = "cn"):
    """Returns (what_new, iterations per step, converged).  scheme "cn": the
    paper's Crank-Nicolson with the trapezoidal Jacobian; "midpoint": implicit
    midpoint (Jacobian of the mean of the iterate and w^n)."""
    a = _c128(what)
    ny, nx = a.shape
    iters = np.zeros(max(nsteps, 1), dtype=np.int64)
    rc = _check(_load().orc_ns_run_scheme(_ptr(a), nx, ny, lx, ly, nu, dt, tol, max_iter,
                                          int(dealias), nsteps, _ptr(iters),
                                          {"cn": 0, "midpoint": 1}[scheme]), "ns_run")
    return a, iters[:nsteps], rc == 0


def ns_field(what) -> np.ndarray:
    a = _c128(what)
    ny, nx = a.shape
    w = np.empty((ny, nx))
    _check(_load().orc_ns_field(_ptr(a), nx, ny, _ptr(w)), "ns_field")
    return w


def ns_invariants(what, lx: float, ly: float):
    """(circulation, enstrophy, energy)."""
    a = _c128(what)
    ny, nx = a.shape
    c, z, e = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_load().orc_ns_invariants(_ptr(a), nx, ny, lx, ly, ctypes.byref(c), ctypes.byref(z),
                                     ctypes.byref(e)), "ns_invariants")
    return c.value, z.value, e.value

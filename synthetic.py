"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws initial fields: it holds none of the time-stepping
arithmetic.  The tests and the benchmark feed the same arrays to the FP64
oracle and to the CUDA library.  All draws use numpy's PCG64 generator on the
host in FP64; FP32 runs round the FP64 field once.

Workloads (the paper's equations and boxes, arXiv:1206.3215 Sections 3-5):
  * NLS: box [-10 pi, 10 pi)^2, psi0 = exp(-(x^2+y^2)) + 1e-3 * z, z complex
    Gaussian with independent N(0, 1/2) real and imaginary parts (E|z|^2 = 1);
  * NLS plane wave psi = A exp(i k.x), A = 0.5, mode (3, 2) on a 20 pi box;
  * sine-Gordon: box [-5 pi, 5 pi)^2, u0 = 0.5 exp(-(x^2+y^2)/4) + 1e-3 N(0,1),
    u_t(0) = 0;
  * Navier-Stokes: box [0, 2 pi)^2, omega0 with amplitude spectrum |k|^-3 and
    Gaussian random phases/amplitudes, zero mean, unit rms;
  * Taylor-Green vortices: 4 pi sin(2 pi x) sin(2 pi y) on [0,1)^2 (the
    paper's Eq. 4 setup) and 2 sin x sin y on [0, 2 pi)^2.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 3215


def grid_coords(n: int, x0: float, L: float) -> np.ndarray:
    """x_j = x0 + j L / n, j = 0..n-1."""
    return x0 + np.arange(n, dtype=np.float64) * (L / n)


def nls_gaussian(n: int, seed: int = SEED_BASE, noise: float = 1e-3, batch: int | None = None,
                 x0: float = -10 * math.pi, L: float = 20 * math.pi) -> np.ndarray:
    """psi0 = exp(-(x^2+y^2)) + noise * complex Gaussian; shape [batch][n][n] or [n][n]."""
    x = grid_coords(n, x0, L)
    X, Y = np.meshgrid(x, x, indexing="xy")  # X varies along the last (x) axis
    base = np.exp(-(X * X + Y * Y)).astype(np.complex128)
    out = []
    for b in range(1 if batch is None else batch):
        rng = np.random.default_rng(seed + 1000 * b)
        z = rng.standard_normal((n, n)) * math.sqrt(0.5) + 1j * rng.standard_normal((n, n)) * math.sqrt(0.5)
        out.append(base + noise * z)
    return out[0] if batch is None else np.stack(out)


def nls_plane_wave(n: int, A: float = 0.5, m: tuple[int, int] = (3, 2), L: float = 20 * math.pi,
                   x0: float = -10 * math.pi) -> np.ndarray:
    """psi = A exp(i (kx x + ky y)) with k = 2 pi m / L on the grid."""
    x = grid_coords(n, x0, L)
    X, Y = np.meshgrid(x, x, indexing="xy")
    kx, ky = 2 * math.pi * m[0] / L, 2 * math.pi * m[1] / L
    return A * np.exp(1j * (kx * X + ky * Y))


def sg_gaussian(n: int, seed: int = SEED_BASE + 2, noise: float = 1e-3, batch: int | None = None,
                x0: float = -5 * math.pi, L: float = 10 * math.pi):
    """(u0, v0): u0 = 0.5 exp(-(x^2+y^2)/4) + noise N(0,1), v0 = 0."""
    x = grid_coords(n, x0, L)
    X, Y = np.meshgrid(x, x, indexing="xy")
    base = 0.5 * np.exp(-(X * X + Y * Y) / 4.0)
    us = []
    for b in range(1 if batch is None else batch):
        rng = np.random.default_rng(seed + 1000 * b)
        us.append(base + noise * rng.standard_normal((n, n)))
    u = us[0] if batch is None else np.stack(us)
    return u, np.zeros_like(u)


def ns_power_law(n: int, seed: int = SEED_BASE + 3, slope: float = -3.0, L: float = 2 * math.pi,
                 batch: int | None = None) -> np.ndarray:
    """omega0 = Re F^-1[|k|^slope (g_r + i g_i)], zero mean, scaled to unit rms."""
    m = np.fft.fftfreq(n, d=1.0 / n)
    k = 2 * math.pi / L * m
    KX, KY = np.meshgrid(k, k, indexing="xy")
    kk = np.sqrt(KX * KX + KY * KY)
    amp = np.zeros_like(kk)
    nz = kk > 0
    amp[nz] = kk[nz] ** slope
    out = []
    for b in range(1 if batch is None else batch):
        rng = np.random.default_rng(seed + 1000 * b)
        g = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        w = np.real(np.fft.ifft2(amp * g))
        w -= w.mean()
        w /= math.sqrt(np.mean(w * w))
        out.append(w)
    return out[0] if batch is None else np.stack(out)


def taylor_green_paper(n: int, t: float = 0.0, nu: float = 0.1) -> np.ndarray:
    """4 pi sin(2 pi x) sin(2 pi y) exp(-8 pi^2 nu t) on [0,1)^2."""
    x = grid_coords(n, 0.0, 1.0)
    X, Y = np.meshgrid(x, x, indexing="xy")
    return 4 * math.pi * np.sin(2 * math.pi * X) * np.sin(2 * math.pi * Y) * math.exp(
        -8 * math.pi ** 2 * nu * t)


def taylor_green_2pi(n: int, t: float = 0.0, nu: float = 1e-3) -> np.ndarray:
    """2 sin x sin y exp(-2 nu t) on [0, 2 pi)^2."""
    x = grid_coords(n, 0.0, 2 * math.pi)
    X, Y = np.meshgrid(x, x, indexing="xy")
    return 2 * np.sin(X) * np.sin(Y) * math.exp(-2 * nu * t)


_FIELD_CACHE: dict = {}


def _serving_field(eq: str, n: int, seed: int, dtype: str):
    """A seeded initial state of a serving request, cached: (psi,) for NLS,
    (u0, v0) for sine-Gordon, (w0,) for Navier-Stokes, in the request's
    precision (rounded once from FP64)."""
    key = (eq, n, seed, dtype)
    got = _FIELD_CACHE.get(key)
    if got is None:
        cplx, real = (np.complex64, np.float32) if dtype == "fp32" else (np.complex128, np.float64)
        if eq == "nls":
            got = (nls_gaussian(n, seed=seed).astype(cplx),)
        elif eq == "sg":
            got = tuple(a.astype(real) for a in sg_gaussian(n, seed=seed))
        else:
            got = (ns_power_law(n, seed=seed).astype(real),)
        _FIELD_CACHE[key] = got
    return got


def serving_mix(count: int, rate_hz: float, sizes=(128, 256, 512, 1024, 2048), steps=(50, 500),
                seed: int = SEED_BASE + 4, eqs=("nls", "sg", "ns"), fields_per_shape: int | None = None,
                precision: str = "fp32") -> list[dict]:
    """Seeded Poisson stream of mixed solves: arrival times with mean spacing
    1/rate_hz, equation, grid size and step count uniform over the given
    choices, each with the parameters of that equation's workload above.
    Every request gets its own seeded initial field, or, with
    fields_per_shape = k, one of k seeded fields of its (equation, N) (a
    stream of thousands of requests then holds k fields per shape in host
    memory instead of one per request)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(count):
        t += rng.exponential(1.0 / rate_hz)
        eq = eqs[int(rng.integers(len(eqs)))]
        n = int(sizes[int(rng.integers(len(sizes)))])
        k = int(rng.integers(steps[0], steps[1] + 1))
        fseed = int(rng.integers(1 << 30))
        if fields_per_shape:
            fseed = seed * 7919 + (fseed % fields_per_shape)
        state = _serving_field(eq, n, fseed, precision)
        if eq == "nls":
            params = {"dt": 1e-3, "lx": 20 * math.pi, "ly": 20 * math.pi}
        elif eq == "sg":
            params = {"dt": 1e-3, "lx": 10 * math.pi, "ly": 10 * math.pi, "rfft": 1}
        else:
            params = {"dt": 2.5e-4, "lx": 2 * math.pi, "ly": 2 * math.pi, "nu": 1e-3, "rfft": 1}
        out.append({"rid": rid, "eq": eq, "n": n, "steps": k, "state": state, "arrival": t,
                    "precision": precision, "params": params, "seed": fseed})
    if not fields_per_shape:
        _FIELD_CACHE.clear()  # each request holds its own arrays
    return out

"""Pins of the oracle's NLS split-step (Eq. 1, Section 4.1) and its invariants
(Eq. 2)."""
import math

import numpy as np
import pytest

import synthetic as S

L = 20 * math.pi


def _golden(name):
    import os
    vals = {}
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    for line in open(path):
        line = line.split("#")[0].split()
        if len(line) == 2:
            vals[line[0]] = float(line[1])
    return vals


@pytest.mark.parametrize("sigma", [1.0, -1.0])
@pytest.mark.parametrize("merged", [False, True])
def test_plane_wave_is_exact(orc, sigma, merged):
    # |psi| is constant for a plane wave, so the linear and nonlinear flows
    # commute and Strang splitting is exact up to rounding:
    # psi = A exp(i(k.x - (|k|^2 + sigma A^2) t)).
    A, m, n, dt, steps = 0.5, (3, 2), 64, 1e-3, 2000
    p0 = S.nls_plane_wave(n, A=A, m=m)
    p = orc.nls_run(p0, L, L, dt, steps, sigma=sigma, merged=merged)
    k2 = (2 * math.pi / L) ** 2 * (m[0] ** 2 + m[1] ** 2)
    exact = p0 * np.exp(-1j * (k2 + sigma * A * A) * dt * steps)
    assert np.abs(p - exact).max() <= 1e-11


def test_plane_wave_invariants_closed_form(orc):
    A, m = 0.5, (3, 2)
    k2 = (2 * math.pi / L) ** 2 * (m[0] ** 2 + m[1] ** 2)
    for sigma in (1.0, -1.0):
        M, E = orc.nls_invariants(S.nls_plane_wave(64, A=A, m=m), L, L, sigma)
        assert abs(M - A * A * L * L) <= 1e-12 * M
        assert abs(E - L * L * (0.5 * A * A * k2 + sigma * A ** 4 / 4)) <= 1e-12 * abs(E)


def test_merged_equals_literal_strang(orc):
    p0 = S.nls_gaussian(64)
    a = orc.nls_run(p0, L, L, 1e-3, 50, merged=False)
    b = orc.nls_run(p0, L, L, 1e-3, 50, merged=True)
    assert np.abs(a - b).max() <= 1e-12


def test_linear_substep_single_mode(orc):
    # zero amplitude limit: only the linear flow acts; a Fourier mode picks up
    # exp(-i |k|^2 t) exactly (the sub-step of Section 4.1 is the exact solution)
    n, m, dt, steps = 32, (5, -3), 1e-2, 100
    j = np.arange(n)
    p0 = 1e-9 * np.exp(2j * math.pi * (np.outer(j * m[1], np.ones(n)) + np.outer(np.ones(n), j * m[0])) / n)
    p = orc.nls_run(p0, L, L, dt, steps)
    k2 = (2 * math.pi / L) ** 2 * (m[0] ** 2 + m[1] ** 2)
    assert np.abs(p - p0 * np.exp(-1j * k2 * dt * steps)).max() <= 1e-12 * 1e-9


def test_config1_invariants(orc):
    # 64^2 Gaussian with noise, dt = 1e-3, 200 steps (the paper's accuracy report:
    # mass to machine precision, energy to 6 significant figures)
    g = _golden("invariants_section5.txt")
    p0 = S.nls_gaussian(64)
    M0, E0 = orc.nls_invariants(p0, L, L)
    p = orc.nls_run(p0, L, L, 1e-3, 200, merged=True)
    M1, E1 = orc.nls_invariants(p, L, L)
    assert abs(M1 - M0) / M0 <= g["nls_mass_rel_drift_max"]
    assert abs(E1 - E0) / abs(E0) <= g["nls_energy_rel_drift_max"]


def test_nonlinear_substep_keeps_modulus(orc):
    # with the box so large that |k|^2 dt is negligible the modulus of a smooth
    # field is untouched by the nonlinear phase; check via the mass per point
    p0 = S.nls_gaussian(32, noise=0.0)
    p = orc.nls_run(p0, 1e9, 1e9, 1e-3, 10)
    assert np.abs(np.abs(p) - np.abs(p0)).max() <= 1e-12


def test_planted_wrong_sign_fails_plane_wave(orc):
    A, m, dt, steps = 0.5, (3, 2), 1e-3, 200
    p0 = S.nls_plane_wave(64, A=A, m=m)
    p = orc.nls_run(p0, L, L, dt, steps, sigma=-1.0)
    k2 = (2 * math.pi / L) ** 2 * 13
    exact_sigma_plus = p0 * np.exp(-1j * (k2 + A * A) * dt * steps)
    assert np.abs(p - exact_sigma_plus).max() > 1e-3

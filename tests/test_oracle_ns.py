"""Pins of the oracle's Navier-Stokes Crank-Nicolson / fixed-point scheme
(Section 4.3) against the Taylor-Green vortex (Eq. 4) and Table 4."""
import math
import os

import numpy as np
import pytest

import synthetic as S


def _golden(name):
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        line = line.split("#")[0].split()
        if len(line) == 2:
            vals[line[0]] = float(line[1])
    return vals


def _cn_error(amp, lam, nu, dt, steps):
    # exact decay exp(-nu lam t) vs the CN amplification (1-a/2)/(1+a/2), a = nu lam dt
    a = nu * lam * dt
    g = (1 - a / 2) / (1 + a / 2)
    return amp * abs(g ** steps - math.exp(-a * steps))


@pytest.mark.parametrize("n", [16, 32, 64])
def test_taylor_green_table4(orc, n):
    g = _golden("ns_taylor_green_table4.txt")
    steps, dt, nu = int(g["steps"]), g["dt"], g["nu"]
    w0 = S.taylor_green_paper(n)
    wh = orc.ns_init(w0, dealias=False)
    wh, iters, ok = orc.ns_run(wh, 1.0, 1.0, nu, dt, steps, tol=g["tol"], dealias=False)
    assert ok
    err = np.abs(orc.ns_field(wh) - S.taylor_green_paper(n, t=steps * dt, nu=nu)).max()
    # the printed 1.65e-5 (3 s.f.), the same for every N
    assert round(err, 7) == pytest.approx(g["max_error"], abs=5e-8)
    # and the CN closed form to rounding
    assert abs(err - _cn_error(4 * math.pi, 8 * math.pi ** 2, nu, dt, steps)) <= 1e-10
    # J = 0 for the vortex: the second iterate reproduces the first
    assert (iters == 2).all()


def test_taylor_green_other_viscosity_misses_table4(orc):
    # the planted reading nu = 1 (the coefficient printed in Section 3.3) cannot
    # reproduce the printed error
    g = _golden("ns_taylor_green_table4.txt")
    n = 16
    wh = orc.ns_init(S.taylor_green_paper(n), dealias=False)
    wh, _, _ = orc.ns_run(wh, 1.0, 1.0, 1.0, g["dt"], 20, dealias=False)
    err = np.abs(orc.ns_field(wh) - S.taylor_green_paper(n, t=20 * g["dt"], nu=1.0)).max()
    assert abs(err - g["max_error"]) > 1e-4


def test_taylor_green_2pi_box_256(orc):
    n, nu, dt, steps = 256, 1e-3, 2.5e-4, 40
    wh = orc.ns_init(S.taylor_green_2pi(n), dealias=True)
    wh, iters, ok = orc.ns_run(wh, 2 * math.pi, 2 * math.pi, nu, dt, steps)
    assert ok
    err = np.abs(orc.ns_field(wh) - S.taylor_green_2pi(n, t=steps * dt, nu=nu)).max()
    assert abs(err - _cn_error(2.0, 2.0, nu, dt, steps)) <= 1e-12


def test_jacobian_closed_form(orc):
    # omega = cos x + cos 2y -> psi = cos x + cos(2y)/4 ->
    # J = psi_y omega_x - psi_x omega_y = -1.5 sin x sin 2y
    n = 32
    L = 2 * math.pi
    x = S.grid_coords(n, 0.0, L)
    X, Y = np.meshgrid(x, x)
    J = orc.ns_jacobian(orc.ns_init(np.cos(X) + np.cos(2 * Y), True), L, L)
    assert np.abs(J + 1.5 * np.sin(X) * np.sin(2 * Y)).max() <= 1e-13


def test_jacobian_antisymmetry_and_dealias_mask(orc):
    # J(psi, omega) with omega = -Lap psi; a single Fourier mode has J = 0
    n = 32
    L = 2 * math.pi
    x = S.grid_coords(n, 0.0, L)
    X, Y = np.meshgrid(x, x)
    J = orc.ns_jacobian(orc.ns_init(np.sin(3 * X + 2 * Y), True), L, L)
    assert np.abs(J).max() <= 1e-13
    # dealiasing removes |m| >= n/3 modes from the initial field
    # (the kept mode has |w_hat| = n^2/2 = 512; the rest is transform rounding)
    wh = orc.ns_init(np.cos(11 * X), True)
    assert np.abs(wh).max() <= 1e-11
    wh = orc.ns_init(np.cos(10 * X), True)
    assert abs(np.abs(wh).max() - n * n / 2) <= 1e-10


def test_random_field_invariants(orc):
    n, L, nu, dt = 64, 2 * math.pi, 1e-3, 2.5e-3
    w0 = S.ns_power_law(n)
    wh = orc.ns_init(w0, dealias=True)
    c0, z0, e0 = orc.ns_invariants(wh, L, L)
    wh, iters, ok = orc.ns_run(wh, L, L, nu, dt, 20)
    assert ok and iters.min() >= 2
    c1, z1, e1 = orc.ns_invariants(wh, L, L)
    assert abs(c1 - c0) <= 1e-12  # J_hat(0) = 0: the mean is conserved exactly
    # viscous decay only, small over 20 steps
    assert 0 < (z0 - z1) / z0 < 0.05 and 0 <= (e0 - e1) / e0 < 0.01


def test_enstrophy_energy_via_parseval_and_physical_agree(orc):
    n, L = 32, 2 * math.pi
    wh = orc.ns_init(S.ns_power_law(n), dealias=True)
    c, z, e = orc.ns_invariants(wh, L, L)
    k = orc.wavenumbers(n, L)
    KX, KY = np.meshgrid(k, k)
    k2 = KX ** 2 + KY ** 2
    z2 = 0.5 * L * L / n ** 4 * np.sum(np.abs(wh) ** 2)
    k2[0, 0] = 1.0
    e2 = 0.5 * L * L / n ** 4 * np.sum(np.abs(wh) ** 2 / k2 * (k2 > 0))
    assert abs(z - z2) <= 1e-12 * z and abs(e - e2) <= 1e-12 * e


def test_non_convergence_is_reported(orc):
    n, L = 32, 2 * math.pi
    wh = orc.ns_init(S.ns_power_law(n), dealias=True)
    _, iters, ok = orc.ns_run(wh, L, L, 1e-3, 2.5e-3, 3, max_iter=1)
    assert not ok and (iters == 1).all()


def test_midpoint_equals_cn_when_j_vanishes(orc):
    # Taylor-Green: J = 0, both schemes reduce to the same CN amplification
    g = _golden("ns_taylor_green_table4.txt")
    n = 32
    wh = orc.ns_init(S.taylor_green_paper(n), dealias=False)
    a, _, _ = orc.ns_run(wh, 1.0, 1.0, g["nu"], g["dt"], 20, dealias=False, scheme="cn")
    b, _, _ = orc.ns_run(wh, 1.0, 1.0, g["nu"], g["dt"], 20, dealias=False, scheme="midpoint")
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_midpoint_conserves_quadratic_invariants_inviscid(orc):
    # nu = 0 with the 2/3 rule: the truncated Jacobian conserves energy and
    # enstrophy exactly, and the implicit midpoint rule keeps every quadratic
    # invariant of the ODE; only the fixed-point tolerance is left
    n, L, dt = 64, 2 * math.pi, 1e-2
    wh = orc.ns_init(S.ns_power_law(n), dealias=True)
    c0, z0, e0 = orc.ns_invariants(wh, L, L)
    w1, iters, ok = orc.ns_run(wh, L, L, 0.0, dt, 20, tol=1e-24, max_iter=200, scheme="midpoint")
    assert ok
    c1, z1, e1 = orc.ns_invariants(w1, L, L)
    assert abs(z1 - z0) / z0 <= 1e-12 and abs(e1 - e0) / e0 <= 1e-12
    # the trapezoidal (paper) scheme does not conserve them exactly
    w2, _, _ = orc.ns_run(wh, L, L, 0.0, dt, 20, tol=1e-24, max_iter=200, scheme="cn")
    c2, z2, e2 = orc.ns_invariants(w2, L, L)
    assert abs(z2 - z0) / z0 > 1e-9

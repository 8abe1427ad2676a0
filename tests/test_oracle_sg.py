"""Pins of the oracle's sine-Gordon leapfrog (Eq. 3, Section 4.2)."""
import math

import numpy as np

import synthetic as S

L = 10 * math.pi


def test_uniform_field_is_the_pendulum_recurrence(orc):
    # k = 0 only: the scheme reduces to u^{n+1} = 2u^n - u^{n-1} - dt^2 sin u^n,
    # with the backward Taylor start u^{-1} = u^0 - dt v0 - dt^2/2 sin u^0.
    n, dt, steps, u0, v0 = 16, 1e-2, 300, 0.9, 0.3
    un, um = orc.sg_init(np.full((n, n), u0), np.full((n, n), v0), L, L, dt)
    un, um = orc.sg_run(un, um, L, L, dt, steps)
    a, b = orc.sg_fields(un, um)
    u, up = u0, u0 - dt * v0 - 0.5 * dt * dt * math.sin(u0)
    for _ in range(steps):
        u, up = 2 * u - up - dt * dt * math.sin(u), u
    assert np.abs(a - u).max() <= 1e-12
    assert np.abs(b - up).max() <= 1e-12


def test_small_single_mode_follows_linear_recurrence(orc):
    # amplitude 1e-8: sin u = u to 1e-24, so each Fourier mode obeys
    # u^{n+1} = 2 cos(theta) u^n - u^{n-1},
    # cos(theta) = (1 - dt^2 |k|^2/4 - dt^2/2) / (1 + dt^2 |k|^2/4)
    n, dt, steps, amp = 32, 5e-2, 400, 1e-8
    mx, my = 3, 2
    x = S.grid_coords(n, -5 * math.pi, L)
    X, Y = np.meshgrid(x, x)
    kx, ky = 2 * math.pi * mx / L, 2 * math.pi * my / L
    shape = np.cos(kx * X + ky * Y)
    un, um = orc.sg_init(amp * shape, np.zeros((n, n)), L, L, dt)
    un, um = orc.sg_run(un, um, L, L, dt, steps)
    u_end, _ = orc.sg_fields(un, um)
    k2 = kx * kx + ky * ky
    c = (1 - dt * dt * k2 / 4 - dt * dt / 2) / (1 + dt * dt * k2 / 4)
    th = math.acos(c)
    a0 = 1.0
    am1 = 1.0 - dt * dt * (k2 + 1) / 2  # start-up with sin u -> u
    B = (a0 * math.cos(th) - am1) / math.sin(th)
    g = a0 * math.cos(steps * th) + B * math.sin(steps * th)
    assert np.abs(u_end - amp * g * shape).max() <= 1e-12 * amp * 10


def test_y_independent_data_stays_y_independent(orc):
    n, dt = 32, 1e-2
    x = S.grid_coords(n, -5 * math.pi, L)
    row = 0.5 * np.exp(-x * x / 4)
    u0 = np.tile(row, (n, 1))
    un, um = orc.sg_init(u0, np.zeros((n, n)), L, L, dt)
    un, um = orc.sg_run(un, um, L, L, dt, 50)
    a, _ = orc.sg_fields(un, um)
    assert np.abs(a - a[0:1, :]).max() <= 1e-14


def test_hamiltonian_six_significant_figures(orc):
    # Section 5.2: the final Hamiltonian within 6 significant figures
    n, dt, steps = 64, 1e-3, 500
    u0, v0 = S.sg_gaussian(n)
    un, um = orc.sg_init(u0, v0, L, L, dt)
    H0 = orc.sg_hamiltonian(un, um, L, L, dt)
    un, um = orc.sg_run(un, um, L, L, dt, steps)
    H1 = orc.sg_hamiltonian(un, um, L, L, dt)
    assert abs(H1 - H0) / abs(H0) <= 1e-6


def test_hamiltonian_drift_is_second_order(orc):
    # small data, fixed final time: the drift of the discrete Hamiltonian must
    # fall by 4x when dt halves (second order in time, Section 4.2); a
    # first-order start-up or an unmatched u_t would break the ratio
    n, T = 32, 10.0
    u0, _ = S.sg_gaussian(n, noise=1e-1)
    u0 = 2e-4 * u0

    def drift(dt):
        un, um = orc.sg_init(u0, np.zeros_like(u0), L, L, dt)
        H0 = orc.sg_hamiltonian(un, um, L, L, dt)
        un, um = orc.sg_run(un, um, L, L, dt, int(round(T / dt)))
        return abs(orc.sg_hamiltonian(un, um, L, L, dt) - H0) / H0

    a, b, c = drift(4e-2), drift(2e-2), drift(1e-2)
    assert 3.8 < a / b < 4.2 and 3.8 < b / c < 4.2


def test_planted_plus_laplacian_blows_up(orc):
    # the printed '+Lap' reading integrates u_tt + Lap u = -sin u, whose modes
    # grow like exp(|k| t); emulate it with an imaginary box length (|k|^2 < 0)
    # by checking the amplification factor directly
    dt, k2 = 1e-2, 100.0
    c_minus = (1 - dt * dt * k2 / 4 - dt * dt / 2) / (1 + dt * dt * k2 / 4)
    c_plus = (1 + dt * dt * k2 / 4 - dt * dt / 2) / (1 - dt * dt * k2 / 4)
    assert abs(c_minus) < 1 < abs(c_plus)

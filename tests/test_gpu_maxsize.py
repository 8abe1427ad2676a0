"""The largest grids (8192^2, the paper's Table 2 and 3 maximum) checked
through properties that hold at any size: closed forms the schemes reproduce
exactly, so no oracle run is needed."""
import math

import numpy as np
import pytest

import synthetic as S
from gpu_util import check

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_nls_plane_wave_8192(lib, cuda_device, precision):
    # |psi| constant: every split step is exact (Section 4.1 sub-steps)
    n, L, dt, steps, A = 8192, 20 * math.pi, 1e-3, 20, 0.5
    p0 = S.nls_plane_wave(n, A=A, m=(3, 2), L=L)
    g = lib.Grid("nls", n, precision, lx=L, ly=L, x0=-L / 2, y0=-L / 2, dt=dt)
    g.set_state(p0[None])
    g.step(steps)
    k2 = (2 * math.pi / L) ** 2 * 13
    exact = p0 * np.exp(-1j * (k2 + A * A) * dt * steps)
    check(g.get_state()[0], exact, 1e-12 if precision == "fp64" else 1e-5)


def test_sg_uniform_field_8192_is_the_pendulum(lib, cuda_device):
    # a uniform field only has the k = 0 mode: the leapfrog reduces to the
    # pendulum recurrence u^{n+1} = 2u^n - u^{n-1} - dt^2 sin u^n
    n, dt, steps, u0, v0 = 8192, 1e-2, 40, 0.9, 0.3
    for rfft in (0, 1):
        g = lib.Grid("sg", n, "fp64", lx=10 * math.pi, ly=10 * math.pi, dt=dt, rfft=rfft)
        g.set_state(np.full((1, n, n), u0), np.full((1, n, n), v0))
        g.step(steps)
        a, b = g.get_state()
        u, up = u0, u0 - dt * v0 - 0.5 * dt * dt * math.sin(u0)
        for _ in range(steps):
            u, up = 2 * u - up - dt * dt * math.sin(u), u
        assert np.abs(a - u).max() <= 1e-12 and np.abs(b - up).max() <= 1e-12
        g.close()


def test_ns_taylor_green_8192(lib, cuda_device):
    # J = 0 for the Taylor-Green vortex: the Crank-Nicolson amplification
    # g = (1 - nu dt)/(1 + nu dt) per step for 2 sin x sin y on [0, 2 pi)^2
    n, nu, dt, steps = 8192, 1e-3, 2.5e-4, 10
    g = lib.Grid("ns", n, "fp32", lx=2 * math.pi, ly=2 * math.pi, dt=dt, nu=nu, dealias=1)
    g.set_state(S.taylor_green_2pi(n)[None])
    g.step(steps)
    amp = ((1 - nu * dt) / (1 + nu * dt)) ** steps
    err = np.abs(g.get_state()[0] - amp * S.taylor_green_2pi(n)).max()
    assert err <= 1e-5
    # here the first update already moves w by less than the tolerance
    # (integral of (2 nu dt w)^2 ~ 2e-11 < 1e-10): one update per step
    assert g.stats()[1] == steps


def test_zero_steps_and_zero_fields(lib, cuda_device):
    # step_n(0) changes nothing; a field never set holds zeros, a fixed point
    g = lib.Grid("nls", 64, "fp32", batch=2, dt=1e-3)
    g.set_field(0, S.nls_gaussian(64).astype(np.complex64))
    before = g.get_state()
    g.step(0)
    assert np.array_equal(g.get_state(), before)
    g.step(5)
    assert not np.any(g.get_state()[1])

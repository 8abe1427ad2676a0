"""Parity of the sine-Gordon leapfrog (Eq. 3, Section 4.2) through the C ABI
against the FP64 oracle and the scheme's closed forms."""
import math

import numpy as np
import pytest

import synthetic as S
from gpu_util import check

pytestmark = pytest.mark.gpu

L = 10 * math.pi
TOL64 = 1e-10
# FP32: relative L2 of u after the run; derived from ~1e-7 per pass rounding
# accumulated as a random walk over the steps (measured and stated in the design notes)
TOL32 = 2e-5


def _grid(lib, n, precision, batch=1, dt=1e-3):
    return lib.Grid("sg", n, precision, batch=batch, lx=L, ly=L, x0=-L / 2, y0=-L / 2, dt=dt)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,steps", [(64, 200), (256, 100)])
def test_gaussian_matches_oracle(lib, orc, cuda_device, precision, n, steps):
    dt = 1e-3
    u0, v0 = S.sg_gaussian(n)
    un, um = orc.sg_init(u0, v0, L, L, dt)
    un, um = orc.sg_run(un, um, L, L, dt, steps)
    ref_n, ref_m = orc.sg_fields(un, um)
    g = _grid(lib, n, precision, dt=dt)
    g.set_state(u0[None], v0[None])
    g.step(steps)
    a, b = g.get_state()
    tol = TOL64 if precision == "fp64" else TOL32
    check(a[0], ref_n, tol)
    check(b[0], ref_m, tol)
    # the increment u^n - u^{n-1} carries the velocity: compare it too
    check(a[0] - b[0], ref_n - ref_m, 1e-8 if precision == "fp64" else 2e-3)


@pytest.mark.parametrize("shift", [100.0, -2.0e4])
def test_large_field_values_match_oracle(lib, orc, cuda_device, shift):
    # u far from 0 exercises the FP32 argument reduction of sin u: a constant
    # shift of u0 by `shift` (the Gaussian bump stays) against the FP64 oracle.
    # Tolerance: the rounding of u itself (|u| eps32 relative to the O(1) bump)
    # grows with |shift|
    n, dt, steps = 64, 1e-3, 100
    u0, v0 = S.sg_gaussian(n)
    u0 = u0 + shift
    un, um = orc.sg_init(u0, v0, L, L, dt)
    un, um = orc.sg_run(un, um, L, L, dt, steps)
    ref_n, _ = orc.sg_fields(un, um)
    g = _grid(lib, n, "fp32", dt=dt)
    g.set_state(u0[None], v0[None])
    g.step(steps)
    got = g.get_state()[0][0]
    err = np.abs(got - ref_n).max()
    assert err <= 8 * abs(shift) * 1.2e-7 + 2e-5, err


def test_uniform_field_is_the_pendulum(lib, cuda_device):
    n, dt, steps, u0, v0 = 16, 1e-2, 300, 0.9, 0.3
    g = _grid(lib, n, "fp64", dt=dt)
    g.set_state(np.full((1, n, n), u0), np.full((1, n, n), v0))
    g.step(steps)
    a, b = g.get_state()
    u, up = u0, u0 - dt * v0 - 0.5 * dt * dt * math.sin(u0)
    for _ in range(steps):
        u, up = 2 * u - up - dt * dt * math.sin(u), u
    assert np.abs(a - u).max() <= 1e-12 and np.abs(b - up).max() <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_hamiltonian_matches_oracle_and_is_conserved(lib, orc, cuda_device, precision):
    n, dt, steps = 128, 1e-3, 500
    u0, v0 = S.sg_gaussian(n)
    un, um = orc.sg_init(u0, v0, L, L, dt)
    H0 = orc.sg_hamiltonian(un, um, L, L, dt)
    g = _grid(lib, n, precision, dt=dt)
    g.set_state(u0[None], v0[None])
    (h0,), = g.conserved()
    assert abs(h0 - H0) / H0 <= (1e-12 if precision == "fp64" else 1e-5)
    g.step(steps)
    (h1,), = g.conserved()
    # Section 5.2: the final Hamiltonian within 6 significant figures
    assert abs(h1 - h0) / h0 <= (1e-6 if precision == "fp64" else 1e-5)


def test_batch_is_bitwise_equal_to_alone(lib, cuda_device):
    n = 64
    u0, v0 = S.sg_gaussian(n, batch=3)
    g = _grid(lib, n, "fp32", batch=3)
    g.set_state(u0, v0)
    g.step(40)
    a, b = g.get_state()
    for i in range(3):
        h = _grid(lib, n, "fp32")
        h.set_state(u0[i:i + 1], v0[i:i + 1])
        h.step(40)
        a1, b1 = h.get_state()
        assert np.array_equal(a1[0], a[i]) and np.array_equal(b1[0], b[i])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_checkpoint_resume_is_bitwise(lib, cuda_device, precision):
    n = 128
    u0, v0 = S.sg_gaussian(n)
    a = _grid(lib, n, precision)
    a.set_state(u0[None], v0[None])
    a.step(25)
    ck = a.checkpoint()
    a.step(25)
    b = _grid(lib, n, precision)
    b.restore(ck)
    b.step(25)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)


def test_config3_size_matches_oracle_over_100_steps(lib, orc, cuda_device):
    # 2048^2 (the sine-Gordon workload's grid), FP64 GPU path against the
    # oracle for 100 steps; the FP32 path against the FP64 GPU path
    n, dt, steps = 2048, 1e-3, 100
    u0, v0 = S.sg_gaussian(n)
    un, um = orc.sg_init(u0, v0, L, L, dt)
    un, um = orc.sg_run(un, um, L, L, dt, steps)
    ref_n, _ = orc.sg_fields(un, um)
    g = _grid(lib, n, "fp64", dt=dt)
    g.set_state(u0[None], v0[None])
    g.step(steps)
    a64, _ = g.get_state()
    check(a64[0], ref_n, TOL64)
    g32 = _grid(lib, n, "fp32", dt=dt)
    g32.set_state(u0[None], v0[None])
    g32.step(steps)
    a32, _ = g32.get_state()
    check(a32[0], ref_n, TOL32)


# ---------------------------------------------------------------------------
# Half spectra (rfft = 1): the same scheme stepped on kx = 0 .. nx/2 with
# real-to-complex row transforms

def _half(lib, n, precision, batch=1, dt=1e-3):
    nx, ny = (n, n) if isinstance(n, int) else n
    return lib.Grid("sg", (nx, ny), precision, batch=batch, lx=L, ly=L, x0=-L / 2, y0=-L / 2, dt=dt, rfft=1)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,steps", [(16, 50), (64, 200), (256, 100)])
def test_half_spectrum_matches_oracle(lib, orc, cuda_device, precision, n, steps):
    dt = 1e-3
    u0, v0 = S.sg_gaussian(n)
    un, um = orc.sg_init(u0, v0, L, L, dt)
    un, um = orc.sg_run(un, um, L, L, dt, steps)
    ref_n, ref_m = orc.sg_fields(un, um)
    g = _half(lib, n, precision, dt=dt)
    g.set_state(u0[None], v0[None])
    g.step(steps)
    a, b = g.get_state()
    tol = TOL64 if precision == "fp64" else TOL32
    check(a[0], ref_n, tol)
    check(b[0], ref_m, tol)
    check(a[0] - b[0], ref_n - ref_m, 1e-8 if precision == "fp64" else 2e-3)


def test_half_spectrum_non_square_matches_oracle(lib, orc, cuda_device):
    nx, ny, dt, steps = 128, 64, 1e-3, 60
    x = S.grid_coords(nx, -L / 2, L)
    y = S.grid_coords(ny, -L / 2, L)
    X, Y = np.meshgrid(x, y, indexing="xy")
    u0 = 0.5 * np.exp(-(X ** 2 + 2 * Y ** 2) / 4) + 0.1 * np.cos(X)
    v0 = 0.2 * np.sin(Y)
    un, um = orc.sg_init(u0, v0, L, L, dt)
    un, um = orc.sg_run(un, um, L, L, dt, steps)
    ref_n, _ = orc.sg_fields(un, um)
    g = _half(lib, (nx, ny), "fp64", dt=dt)
    g.set_state(u0[None], v0[None])
    g.step(steps)
    check(g.get_state()[0][0], ref_n, TOL64)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_half_spectrum_hamiltonian_matches_full_path(lib, cuda_device, precision):
    n, steps = 128, 300
    u0, v0 = S.sg_gaussian(n)
    out = []
    for grid in (_grid(lib, n, precision), _half(lib, n, precision)):
        grid.set_state(u0[None], v0[None])
        grid.step(steps)
        (h,), = grid.conserved()
        out.append(h)
    assert abs(out[0] - out[1]) / out[0] <= (1e-12 if precision == "fp64" else 2e-6)


def test_half_spectrum_batch_fields_resume_and_graphs(lib, cuda_device, monkeypatch):
    # fields of a batch equal their solo runs bit for bit; set/get of one
    # field, checkpoint resume and graph vs direct launches are bitwise too
    n = 64
    u0, v0 = S.sg_gaussian(n, batch=3)
    res = []
    for graphs in ("1", "0"):
        monkeypatch.setenv("PSS_GRAPHS", graphs)
        g = _half(lib, n, "fp32", batch=3)
        g.set_state(u0, v0)
        g.step(20)
        ck = g.checkpoint()
        g.step(20)
        a, b = g.get_state()
        for i in range(3):
            h = _half(lib, n, "fp32")
            h.set_state(u0[i:i + 1], v0[i:i + 1])
            h.step(40)
            a1, b1 = h.get_state()
            assert np.array_equal(a1[0], a[i]) and np.array_equal(b1[0], b[i])
        r = _half(lib, n, "fp32", batch=3)
        r.restore(ck)
        r.step(20)
        for x, y in zip(r.get_state(), (a, b)):
            assert np.array_equal(x, y)
        # replace field 1 mid-run: the other fields are untouched
        g.set_field(1, u0[0], v0[0])
        g.step(5)
        res.append(g.get_state())
    for x, y in zip(res[0], res[1]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("rfft", [0, 1])
def test_set_levels_continues_a_run(lib, cuda_device, rfft):
    # pss_set_state_sg_levels: restart from the two levels read back by
    # get_state; the continuation equals the uninterrupted run up to the
    # rounding of the re-transformed levels
    n, dt = 64, 1e-3
    u0, v0 = S.sg_gaussian(n)
    a = lib.Grid("sg", n, "fp64", lx=L, ly=L, x0=-L / 2, y0=-L / 2, dt=dt, rfft=rfft)
    a.set_state(u0[None], v0[None])
    a.step(30)
    un, unm1 = a.get_state()
    a.step(30)
    b = lib.Grid("sg", n, "fp64", lx=L, ly=L, x0=-L / 2, y0=-L / 2, dt=dt, rfft=rfft)
    b.set_levels(un, unm1)
    assert b.stats()[0] == 0
    b.step(30)
    for x, y in zip(a.get_state(), b.get_state()):
        check(y, x, 1e-12)


def test_set_levels_rejects_other_equations(lib, cuda_device):
    g = lib.Grid("nls", 16, "fp32")
    z = np.zeros((1, 16, 16), np.float32)
    with pytest.raises(lib.PssError) as e:
        g.set_levels(z, z)
    assert e.value.code == lib.PSS_E_ARG

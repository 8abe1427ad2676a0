"""Parity of the Navier-Stokes Crank-Nicolson / fixed-point path (Section
4.3) through the C ABI against the FP64 oracle, Table 4's Taylor-Green error
and closed forms."""
import math
import os

import numpy as np
import pytest

import synthetic as S
from gpu_util import check

pytestmark = pytest.mark.gpu

TOL64 = 1e-9


def _golden(name):
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        line = line.split("#")[0].split()
        if len(line) == 2:
            vals[line[0]] = float(line[1])
    return vals


def _cn_error(amp, lam, nu, dt, steps):
    a = nu * lam * dt
    g = (1 - a / 2) / (1 + a / 2)
    return amp * abs(g ** steps - math.exp(-a * steps))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [64, 256])
def test_taylor_green_table4(lib, cuda_device, precision, n):
    g0 = _golden("ns_taylor_green_table4.txt")
    steps, dt, nu = int(g0["steps"]), g0["dt"], g0["nu"]
    g = lib.Grid("ns", n, precision, lx=1.0, ly=1.0, dt=dt, nu=nu, tol=g0["tol"], dealias=0)
    g.set_state(S.taylor_green_paper(n)[None])
    g.step(steps)
    w = g.get_state()[0]
    err = np.abs(w - S.taylor_green_paper(n, t=steps * dt, nu=nu)).max()
    exact_err = _cn_error(4 * math.pi, 8 * math.pi ** 2, nu, dt, steps)
    if precision == "fp64":
        assert abs(err - exact_err) <= 1e-10
        assert round(err, 7) == pytest.approx(g0["max_error"], abs=5e-8)
    else:
        # FP32: one ulp of a field of amplitude 4 pi is ~1e-6; 20 steps of
        # unbiased rounding stay within 1e-5
        assert abs(err - exact_err) <= 1e-5
    steps_done, updates = g.stats()
    assert steps_done == steps and updates == 2 * steps  # J = 0: two updates per step


def test_taylor_green_2pi_box_256(lib, cuda_device):
    n, nu, dt, steps = 256, 1e-3, 2.5e-4, 40
    g = lib.Grid("ns", n, "fp64", lx=2 * math.pi, ly=2 * math.pi, dt=dt, nu=nu, dealias=1)
    g.set_state(S.taylor_green_2pi(n)[None])
    g.step(steps)
    err = np.abs(g.get_state()[0] - S.taylor_green_2pi(n, t=steps * dt, nu=nu)).max()
    assert abs(err - _cn_error(2.0, 2.0, nu, dt, steps)) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [64, 128])
def test_random_field_matches_oracle(lib, orc, cuda_device, precision, n):
    L, nu, dt, steps = 2 * math.pi, 1e-3, 2.5e-3, 20
    w0 = S.ns_power_law(n)
    ref, iters, ok = orc.ns_run(orc.ns_init(w0, True), L, L, nu, dt, steps)
    assert ok
    g = lib.Grid("ns", n, precision, lx=L, ly=L, dt=dt, nu=nu, tol=1e-10, dealias=1)
    g.set_state(w0[None])
    g.step(steps)
    got = g.get_state()[0]
    check(got, orc.ns_field(ref), TOL64 if precision == "fp64" else 1e-5)
    if precision == "fp64":
        assert g.stats()[1] == int(iters.sum())
    c0, z0, e0 = orc.ns_invariants(ref, L, L)
    (c, z, e), = g.conserved()
    assert abs(z - z0) / z0 <= (1e-10 if precision == "fp64" else 1e-5)
    assert abs(e - e0) / e0 <= (1e-10 if precision == "fp64" else 1e-5)


def test_fields_converging_differently_match_alone(lib, cuda_device):
    # a Taylor-Green field (J = 0: 2 updates per step) and a random field
    # (more updates) in one batch: each equals its solo run bit for bit
    n, L, nu, dt = 64, 2 * math.pi, 1e-3, 2.5e-3
    fields = np.stack([S.taylor_green_2pi(n), S.ns_power_law(n)])
    g = lib.Grid("ns", n, "fp32", batch=2, lx=L, ly=L, dt=dt, nu=nu)
    g.set_state(fields)
    g.step(5)
    together = g.get_state()
    total = g.stats()[1]
    solo_updates = 0
    for i in range(2):
        h = lib.Grid("ns", n, "fp32", lx=L, ly=L, dt=dt, nu=nu)
        h.set_state(fields[i:i + 1])
        h.step(5)
        assert np.array_equal(h.get_state()[0], together[i])
        solo_updates += h.stats()[1]
    assert total == solo_updates


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_checkpoint_resume_is_bitwise(lib, cuda_device, precision):
    n, L, nu, dt = 64, 2 * math.pi, 1e-3, 2.5e-3
    w0 = S.ns_power_law(n)[None]
    a = lib.Grid("ns", n, precision, lx=L, ly=L, dt=dt, nu=nu)
    a.set_state(w0)
    a.step(4)
    ck = a.checkpoint()
    a.step(4)
    b = lib.Grid("ns", n, precision, lx=L, ly=L, dt=dt, nu=nu)
    b.restore(ck)
    b.step(4)
    assert np.array_equal(a.get_state(), b.get_state())
    assert a.stats() == b.stats()


def test_non_convergence_is_reported_and_handle_stays_usable(lib, cuda_device):
    n, L = 32, 2 * math.pi
    g = lib.Grid("ns", n, "fp64", lx=L, ly=L, dt=2.5e-3, nu=1e-3, max_iter=1)
    g.set_state(S.ns_power_law(n)[None])
    # reported by step_n itself (direct launches) or by the next synchronising
    # call (a captured step graph loops on the device)
    with pytest.raises(lib.PssError) as e:
        g.step(3)
        g.sync()
    assert e.value.code == lib.PSS_E_NOT_CONVERGED
    assert np.isfinite(g.get_state()).all()
    assert g.stats()[1] == 3


def test_circulation_is_conserved_at_config4_size(lib, cuda_device):
    # 4096^2 FP32, the Navier-Stokes workload's grid: the mean vorticity is
    # conserved exactly by the scheme (J_hat(0) = 0); enstrophy only decays
    n, L = 4096, 2 * math.pi
    g = lib.Grid("ns", n, "fp32", lx=L, ly=L, dt=2.5e-4, nu=1e-3)
    g.set_state(S.ns_power_law(n)[None])
    (c0, z0, e0), = g.conserved()
    g.step(3)
    (c1, z1, e1), = g.conserved()
    assert abs(c1 - c0) <= 1e-9 * math.sqrt(z0) * L
    assert z1 <= z0 * (1 + 1e-6) and e1 <= e0 * (1 + 1e-6)


@pytest.mark.parametrize("eq", ["ns", "nls", "sg"])
def test_graph_and_direct_launches_agree_bitwise(lib, cuda_device, eq, monkeypatch):
    # the step as one captured CUDA graph (NS: a device-side WHILE loop over
    # the fixed-point updates) equals the step launched kernel by kernel
    n = 64
    if eq == "ns":
        kw, state = dict(lx=2 * math.pi, ly=2 * math.pi, dt=2.5e-3, nu=1e-3), (S.ns_power_law(n, batch=2),)
    elif eq == "nls":
        kw, state = dict(dt=1e-3), (S.nls_gaussian(n, batch=2),)
    else:
        kw, state = dict(lx=10 * math.pi, ly=10 * math.pi, dt=1e-3), S.sg_gaussian(n, batch=2)
    out = []
    for graphs in ("1", "0"):
        monkeypatch.setenv("PSS_GRAPHS", graphs)
        g = lib.Grid(eq, n, "fp32", batch=2, **kw)
        g.set_state(*state)
        g.step(7)
        g.step(7)
        r = g.get_state()
        out.append((r if isinstance(r, tuple) else (r,), g.stats()))
        g.close()
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)
    assert out[0][1] == out[1][1]


# ---------------------------------------------------------------------------
# Implicit-midpoint variant: the Jacobian of (w^k + w^n)/2 in place of the
# trapezoidal (J^k + J^n)/2, same Crank-Nicolson diffusion

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [64, 128])
def test_midpoint_matches_oracle(lib, orc, cuda_device, precision, n):
    L, nu, dt, steps = 2 * math.pi, 1e-3, 2.5e-3, 20
    w0 = S.ns_power_law(n)
    ref, iters, ok = orc.ns_run(orc.ns_init(w0, True), L, L, nu, dt, steps, scheme="midpoint")
    assert ok
    g = lib.Grid("ns", n, precision, lx=L, ly=L, dt=dt, nu=nu, tol=1e-10, dealias=1, scheme="midpoint")
    g.set_state(w0[None])
    g.step(steps)
    check(g.get_state()[0], orc.ns_field(ref), TOL64 if precision == "fp64" else 1e-5)
    if precision == "fp64":
        assert g.stats()[1] == int(iters.sum())


def test_midpoint_taylor_green_equals_cn_closed_form(lib, cuda_device):
    # J = 0: both schemes are the Crank-Nicolson amplification of Table 4's run
    g0 = _golden("ns_taylor_green_table4.txt")
    n, steps, dt, nu = 64, int(g0["steps"]), g0["dt"], g0["nu"]
    g = lib.Grid("ns", n, "fp64", lx=1.0, ly=1.0, dt=dt, nu=nu, tol=g0["tol"], dealias=0, scheme="midpoint")
    g.set_state(S.taylor_green_paper(n)[None])
    g.step(steps)
    err = np.abs(g.get_state()[0] - S.taylor_green_paper(n, t=steps * dt, nu=nu)).max()
    assert abs(err - _cn_error(4 * math.pi, 8 * math.pi ** 2, nu, dt, steps)) <= 1e-10


def test_midpoint_inviscid_keeps_energy_and_enstrophy(lib, cuda_device):
    # nu = 0 with the 2/3 rule: the midpoint rule conserves every quadratic
    # invariant of the truncated system, up to the fixed-point tolerance
    n, L, dt, steps = 64, 2 * math.pi, 1e-2, 20
    out = {}
    for scheme in ("midpoint", "cn"):
        g = lib.Grid("ns", n, "fp64", lx=L, ly=L, dt=dt, nu=0.0, tol=1e-24, max_iter=200, dealias=1,
                     scheme=scheme)
        g.set_state(S.ns_power_law(n)[None])
        (c0, z0, e0), = g.conserved()
        g.step(steps)
        (c1, z1, e1), = g.conserved()
        out[scheme] = (abs(z1 - z0) / z0, abs(e1 - e0) / e0)
    assert max(out["midpoint"]) <= 1e-11
    assert out["cn"][0] > 1e-9  # the trapezoidal rule does not conserve them


def test_midpoint_graph_direct_and_resume_agree_bitwise(lib, cuda_device, monkeypatch):
    n, L = 64, 2 * math.pi
    kw = dict(lx=L, ly=L, dt=2.5e-3, nu=1e-3, scheme="midpoint")
    w0 = S.ns_power_law(n, batch=2)
    out = []
    for graphs in ("1", "0"):
        monkeypatch.setenv("PSS_GRAPHS", graphs)
        g = lib.Grid("ns", n, "fp32", batch=2, **kw)
        g.set_state(w0)
        g.step(4)
        ck = g.checkpoint()
        g.step(5)
        out.append((g.get_state(), g.stats()))
        h = lib.Grid("ns", n, "fp32", batch=2, **kw)
        h.restore(ck)
        h.step(5)
        assert np.array_equal(h.get_state(), out[-1][0]) and h.stats() == out[-1][1]
        g.close()
        h.close()
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


# ---------------------------------------------------------------------------
# Half spectra (rfft = 1): the vorticity iterates and J_hat^n keep kx >= 0
# only; the derivative fields are written at kx and nx - kx

@pytest.mark.parametrize("scheme", ["cn", "midpoint"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [64, 128])
def test_half_spectrum_matches_oracle(lib, orc, cuda_device, scheme, precision, n):
    L, nu, dt, steps = 2 * math.pi, 1e-3, 2.5e-3, 20
    w0 = S.ns_power_law(n)
    ref, iters, ok = orc.ns_run(orc.ns_init(w0, True), L, L, nu, dt, steps, scheme=scheme)
    assert ok
    g = lib.Grid("ns", n, precision, lx=L, ly=L, dt=dt, nu=nu, tol=1e-10, dealias=1, scheme=scheme, rfft=1)
    g.set_state(w0[None])
    g.step(steps)
    check(g.get_state()[0], orc.ns_field(ref), TOL64 if precision == "fp64" else 1e-5)
    if precision == "fp64":
        assert g.stats()[1] == int(iters.sum())
    c0, z0, e0 = orc.ns_invariants(ref, L, L)
    (c, z, e), = g.conserved()
    assert abs(z - z0) / z0 <= (1e-10 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("n", [32, 64])
def test_half_spectrum_taylor_green_table4_without_dealiasing(lib, cuda_device, n):
    # the paper's mode (no 2/3 rule): the Nyquist column is visited and has
    # no mirror; Table 4's error as with full spectra
    g0 = _golden("ns_taylor_green_table4.txt")
    steps, dt, nu = int(g0["steps"]), g0["dt"], g0["nu"]
    g = lib.Grid("ns", n, "fp64", lx=1.0, ly=1.0, dt=dt, nu=nu, tol=g0["tol"], dealias=0, rfft=1)
    g.set_state(S.taylor_green_paper(n)[None])
    g.step(steps)
    err = np.abs(g.get_state()[0] - S.taylor_green_paper(n, t=steps * dt, nu=nu)).max()
    assert abs(err - _cn_error(4 * math.pi, 8 * math.pi ** 2, nu, dt, steps)) <= 1e-10


def test_half_spectrum_non_square_and_without_dealiasing_matches_oracle(lib, orc, cuda_device):
    nx, ny, L, nu, dt, steps = 128, 64, 2 * math.pi, 1e-3, 2.5e-3, 10
    x = S.grid_coords(nx, 0.0, L)
    y = S.grid_coords(ny, 0.0, L)
    X, Y = np.meshgrid(x, y, indexing="xy")
    w0 = np.sin(3 * X) * np.cos(2 * Y) + 0.5 * np.cos(X + Y) + 0.2 * np.sin(5 * X - 3 * Y)
    for dealias in (1, 0):
        ref, _, ok = orc.ns_run(orc.ns_init(w0, bool(dealias)), L, L, nu, dt, steps, dealias=bool(dealias))
        assert ok
        g = lib.Grid("ns", (nx, ny), "fp64", lx=L, ly=L, dt=dt, nu=nu, dealias=dealias, rfft=1)
        g.set_state(w0[None])
        g.step(steps)
        check(g.get_state()[0], orc.ns_field(ref), TOL64)


def test_half_spectrum_batch_resume_graphs_and_fields(lib, cuda_device, monkeypatch):
    # batch = solo, graph = direct launches and checkpoint resume bit for bit;
    # set_field / get_field of one slot
    n, L = 64, 2 * math.pi
    kw = dict(lx=L, ly=L, dt=2.5e-3, nu=1e-3, rfft=1)
    fields = np.stack([S.taylor_green_2pi(n), S.ns_power_law(n)])
    res = []
    for graphs in ("1", "0"):
        monkeypatch.setenv("PSS_GRAPHS", graphs)
        g = lib.Grid("ns", n, "fp32", batch=2, **kw)
        g.set_state(fields)
        g.step(3)
        ck = g.checkpoint()
        g.step(3)
        together = g.get_state()
        for i in range(2):
            h = lib.Grid("ns", n, "fp32", **kw)
            h.set_state(fields[i:i + 1])
            h.step(6)
            assert np.array_equal(h.get_state()[0], together[i])
            assert np.array_equal(g.get_field(i), together[i])
        r = lib.Grid("ns", n, "fp32", batch=2, **kw)
        r.restore(ck)
        r.step(3)
        assert np.array_equal(r.get_state(), together)
        g.set_field(0, fields[1])
        g.step(2)
        res.append((g.get_state(), g.stats()))
    assert np.array_equal(res[0][0], res[1][0]) and res[0][1] == res[1][1]

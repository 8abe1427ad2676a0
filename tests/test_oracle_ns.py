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


# --------------------------------------------------------------------------
# The nonlinear term of the update (Section 4.3): its sign, and the
# trapezoidal weighting (J^k + J^n)/2.  Taylor-Green has J = 0 and the
# invariants above are blind to the sign of J, so these pins look at the
# advection itself.

# the oracle's Crank-Nicolson update with the trapezoidal Jacobian
_CN_UPDATE = "wk1[i] = ((1.0 - a) * what[i] - 0.5 * dt * (jcur[i] + jn[i])) / (1.0 + a);"
# plausible mistakes: J entered with the wrong sign; the newest iterate's J alone
_MUTANTS = {
    "j_sign": [(_CN_UPDATE, _CN_UPDATE.replace("- 0.5 * dt", "+ 0.5 * dt"))],
    "jk_only": [(_CN_UPDATE, "wk1[i] = ((1.0 - a) * what[i] - dt * jcur[i]) / (1.0 + a);")],
}


def _two_mode(n):
    L = 2 * math.pi
    x = S.grid_coords(n, 0.0, L)
    X, Y = np.meshgrid(x, x)
    return L, X, Y, np.cos(X) + np.cos(2 * Y)


def _initial_rate_errors(o, dts=(4e-3, 2e-3, 1e-3)):
    # inviscid, omega0 = cos x + cos 2y: omega_t = -J = +1.5 sin x sin 2y at
    # t = 0; the one-step difference quotient of a consistent scheme tends to
    # it, with an error proportional to dt
    n = 32
    L, X, Y, w0 = _two_mode(n)
    rate = 1.5 * np.sin(X) * np.sin(2 * Y)
    wh0 = o.ns_init(w0, dealias=True)
    errs = []
    for dt in dts:
        wh, _, ok = o.ns_run(wh0, L, L, 0.0, dt, 1, tol=1e-28, max_iter=500)
        assert ok
        errs.append(np.abs((o.ns_field(wh) - w0) / dt - rate).max())
    return dts, errs


def _rk4_reference(w0, n, L, nu, T, h):
    """The semi-discrete 2/3-rule system d w_hat/dt = -D F[J] - nu |k|^2 w_hat
    integrated by classical RK4 with numpy's FFT (an independent integrator:
    fourth order, explicit, no fixed point), returned in physical space."""
    k = np.fft.fftfreq(n, d=L / n) * 2 * np.pi
    KX, KY = np.meshgrid(k, k)
    K2 = KX ** 2 + KY ** 2
    m = np.fft.fftfreq(n) * n
    MX, MY = np.meshgrid(m, m)
    D = ((3 * np.abs(MX) < n) & (3 * np.abs(MY) < n)).astype(float)

    def rhs(wh):
        ph = np.where(K2 > 0, wh / np.where(K2 > 0, K2, 1.0), 0.0)
        px, py = np.fft.ifft2(1j * KX * ph).real, np.fft.ifft2(1j * KY * ph).real
        wx, wy = np.fft.ifft2(1j * KX * wh).real, np.fft.ifft2(1j * KY * wh).real
        return -D * np.fft.fft2(py * wx - px * wy) - nu * K2 * wh

    wh = D * np.fft.fft2(w0)
    for _ in range(int(round(T / h))):
        a = rhs(wh)
        b = rhs(wh + 0.5 * h * a)
        c = rhs(wh + 0.5 * h * b)
        d = rhs(wh + h * c)
        wh = wh + h / 6 * (a + 2 * b + 2 * c + d)
    return np.fft.ifft2(wh).real


def _convergence_to_reference(o, n=32, nu=0.01, T=0.4, steps=(10, 20, 40)):
    L = 2 * math.pi
    w0 = S.ns_power_law(n)
    ref = _rk4_reference(w0, n, L, nu, T, T / 800)
    wh0 = o.ns_init(w0, dealias=True)
    errs = []
    for st in steps:
        wh, _, ok = o.ns_run(wh0, L, L, nu, T / st, st, tol=1e-28, max_iter=500)
        assert ok
        errs.append(np.abs(o.ns_field(wh) - ref).max())
    return errs, np.abs(ref).max()


def _rate_pin_holds(o):
    dts, errs = _initial_rate_errors(o)
    first_order = all(1.8 <= errs[i] / errs[i + 1] <= 2.2 for i in range(len(errs) - 1))
    return first_order and all(e <= 2.0 * dt for e, dt in zip(errs, dts))


def _second_order_pin_holds(o):
    errs, wmax = _convergence_to_reference(o)
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    return all(3.8 <= r <= 4.2 for r in ratios) and errs[-1] <= 1e-3 * wmax


def test_update_advects_with_minus_jacobian(orc):
    dts, errs = _initial_rate_errors(orc)
    # measured: error / dt = 1.2 at every dt (half the second derivative)
    for e, dt in zip(errs, dts):
        assert e <= 2.0 * dt, (e, dt)
    for i in range(len(errs) - 1):
        assert 1.8 <= errs[i] / errs[i + 1] <= 2.2


def test_trapezoidal_jacobian_is_second_order_against_rk4(orc):
    # ratio 4 per halving of dt (measured 4.01, 4.00); J^k or J^n alone would
    # be first order (ratio 2), a wrong sign converges to another solution
    errs, wmax = _convergence_to_reference(orc)
    for i in range(len(errs) - 1):
        assert 3.8 <= errs[i] / errs[i + 1] <= 4.2, errs
    assert errs[-1] <= 1e-3 * wmax, errs


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_planted_update_mistakes_fail_the_pins(orc, tmp_path, name):
    bad = orc.mutant(_MUTANTS[name], str(tmp_path))
    rate_ok, order_ok = _rate_pin_holds(bad), _second_order_pin_holds(bad)
    if name == "j_sign":
        assert not rate_ok and not order_ok
    else:  # consistent but first order: only the convergence pin sees it
        assert not order_ok
    # the unmodified oracle passes both
    assert _rate_pin_holds(orc) and _second_order_pin_holds(orc)

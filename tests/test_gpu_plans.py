"""Plans and the autotuner: the second launch shape of the FP32 passes (16
points per thread, four CTAs per SM) is as correct as the first, and tuning
leaves the grid's state untouched and every grid of a key on one plan."""
import math

import numpy as np
import pytest

import synthetic as S
from gpu_util import check

pytestmark = pytest.mark.gpu

L = 20 * math.pi


@pytest.mark.parametrize("plan", ["0", "1"])
@pytest.mark.parametrize("n", [512, 1024])
def test_each_shape_matches_oracle_nls(lib, orc, cuda_device, monkeypatch, plan, n):
    monkeypatch.setenv("PSS_PLAN", plan)
    dt, steps = 1e-3, 20
    p0 = S.nls_gaussian(n)
    g = lib.Grid("nls", n, "fp32", lx=L, ly=L, x0=-L / 2, y0=-L / 2, dt=dt)
    g.set_state(p0[None])
    g.step(steps)
    ref = orc.nls_run(p0, L, L, dt, steps, merged=True)
    check(g.get_state()[0], ref, 1e-5)


@pytest.mark.parametrize("plan", ["0", "1"])
@pytest.mark.parametrize("rfft", [0, 1])
def test_each_shape_matches_oracle_sg(lib, orc, cuda_device, monkeypatch, plan, rfft):
    monkeypatch.setenv("PSS_PLAN", plan)
    n, dt, steps, Ls = 1024, 1e-3, 20, 10 * math.pi
    u0, v0 = S.sg_gaussian(n)
    un, um = orc.sg_init(u0, v0, Ls, Ls, dt)
    un, um = orc.sg_run(un, um, Ls, Ls, dt, steps)
    ref, _ = orc.sg_fields(un, um)
    g = lib.Grid("sg", n, "fp32", lx=Ls, ly=Ls, x0=-Ls / 2, y0=-Ls / 2, dt=dt, rfft=rfft)
    g.set_state(u0[None], v0[None])
    g.step(steps)
    check(g.get_state()[0][0], ref, 2e-5)


@pytest.mark.parametrize("eq", ["nls", "sg"])
def test_autotune_keeps_state_and_one_plan_per_key(lib, cuda_device, eq):
    n = 512
    if eq == "nls":
        kw, state = dict(lx=L, ly=L, dt=1e-3), (S.nls_gaussian(n, batch=2),)
    else:
        kw, state = dict(lx=10 * math.pi, ly=10 * math.pi, dt=1e-3, rfft=1), S.sg_gaussian(n, batch=2)
    g = lib.Grid(eq, n, "fp32", batch=2, **kw)
    g.set_state(*state)
    g.step(3)
    before = g.get_state()
    changed = g.autotune(3)
    assert changed >= 0
    after = g.get_state()
    before = before if isinstance(before, tuple) else (before,)
    after = after if isinstance(after, tuple) else (after,)
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    assert g.stats()[0] == 3
    # the plan now in force is shared: a field run alone equals its slot
    g2 = lib.Grid(eq, n, "fp32", batch=2, **kw)
    g2.set_state(*state)
    g2.step(8)
    together = g2.get_state()
    together = together if isinstance(together, tuple) else (together,)
    h = lib.Grid(eq, n, "fp32", **kw)
    h.set_state(*(s[1:2] for s in state))
    h.step(8)
    alone = h.get_state()
    alone = alone if isinstance(alone, tuple) else (alone,)
    for a, b in zip(alone, together):
        assert np.array_equal(a[0], b[1])


@pytest.mark.parametrize("n", [256, 512, 1024, 2048, 4096])
def test_tensor_copy_staging_is_bitwise_equal(lib, cuda_device, monkeypatch, n):
    # The NLS column pass stages its tiles by tensor copies into a landing
    # buffer shared by two groups (default), by one tensor copy into a single
    # buffer (PSS_COL_LAND=0) or by per-point copies (PSS_TMA=0): the arithmetic is the
    # same, so the states agree bit for bit, including a batch whose tiles
    # wrap from one field to the next
    p0 = S.nls_gaussian(n, batch=3)
    out = []
    for tma, land in (("1", "1"), ("1", "0"), ("0", "0")):
        monkeypatch.setenv("PSS_TMA", tma)
        monkeypatch.setenv("PSS_COL_LAND", land)
        monkeypatch.setenv("PSS_PLAN", "0")
        g = lib.Grid("nls", n, "fp32", batch=3, lx=L, ly=L, x0=-L / 2, y0=-L / 2, dt=1e-3)
        g.set_state(p0)
        g.step(7)
        g.sync()
        out.append(g.get_state())
        g.close()
    assert np.array_equal(out[0].view(np.uint32), out[1].view(np.uint32))
    assert np.array_equal(out[0].view(np.uint32), out[2].view(np.uint32))


@pytest.mark.parametrize("rfft", [0, 1])
def test_tensor_copy_staging_is_bitwise_equal_sg(lib, cuda_device, monkeypatch, rfft):
    # the sine-Gordon column pass, also on half spectra (rows of nx/2 + 8
    # columns: a row stride that is not a power of two): landing-buffer,
    # one-buffer and per-point staging agree bit for bit
    n, Ls = 2048, 10 * math.pi
    u0, v0 = S.sg_gaussian(n, batch=2)
    out = []
    for tma, land in (("1", "1"), ("1", "0"), ("0", "0")):
        monkeypatch.setenv("PSS_TMA", tma)
        monkeypatch.setenv("PSS_COL_LAND", land)
        monkeypatch.setenv("PSS_PLAN", "0")
        g = lib.Grid("sg", n, "fp32", batch=2, lx=Ls, ly=Ls, x0=-Ls / 2, y0=-Ls / 2, dt=1e-3, rfft=rfft)
        g.set_state(u0, v0)
        g.step(5)
        g.sync()
        out.append(g.get_state())
        g.close()
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(np.ascontiguousarray(a).view(np.uint8), np.ascontiguousarray(b).view(np.uint8))


@pytest.mark.parametrize("rfft", [0, 1])
@pytest.mark.parametrize("scheme", ["cn", "midpoint"])
def test_tensor_copy_staging_is_bitwise_equal_ns(lib, cuda_device, monkeypatch, rfft, scheme):
    # the Navier-Stokes column pass: J staged from full-width rows while the
    # pass visits the (half-spectrum) vorticity columns and skips the column
    # groups the 2/3 rule zeroes; landing-buffer, one-buffer and per-point
    # staging agree bit for bit (also the fixed-point norm: same update count)
    n, Ln, nu, dt = 1024, 2 * math.pi, 1e-3, 2.5e-4
    w0 = S.ns_power_law(n, batch=2)
    out = []
    for tma, land in (("1", "1"), ("1", "0"), ("0", "0")):
        monkeypatch.setenv("PSS_TMA", tma)
        monkeypatch.setenv("PSS_COL_LAND", land)
        g = lib.Grid("ns", n, "fp32", batch=2, lx=Ln, ly=Ln, dt=dt, nu=nu, dealias=1, rfft=rfft,
                     scheme=scheme)
        g.set_state(w0)
        g.step(3)
        g.sync()
        out.append((g.get_state(), g.stats()[1]))
        g.close()
    for other in out[1:]:
        assert out[0][1] == other[1]
        assert np.array_equal(np.ascontiguousarray(out[0][0]).view(np.uint8), np.ascontiguousarray(other[0]).view(np.uint8))


@pytest.mark.parametrize("batch", [1, 2])
@pytest.mark.parametrize("scheme", ["cn", "midpoint"])
def test_split_column_pass_is_bitwise_equal_ns(lib, cuda_device, monkeypatch, batch, scheme):
    # 4096^2, half spectra: the column pass runs each tile in two parts claimed
    # from a counter (the second part, C2, waits for the first's stores); the
    # one-part tensor-copy pass (PSS_COL_SPLIT=0) and per-point staging
    # (PSS_TMA=0) agree with it bit for bit, also in the fixed-point
    # decisions.  Batch 2: the parts of one field's tiles and the next
    # field's interleave
    rfft = 1
    n, Ln, nu, dt = 4096, 2 * math.pi, 1e-3, 2.5e-4
    w0 = S.ns_power_law(n, batch=batch)
    out = []
    for tma, split in (("1", "1"), ("1", "0"), ("0", "0")):
        monkeypatch.setenv("PSS_TMA", tma)
        monkeypatch.setenv("PSS_COL_SPLIT", split)
        g = lib.Grid("ns", n, "fp32", batch=batch, lx=Ln, ly=Ln, dt=dt, nu=nu, dealias=1, rfft=rfft,
                     scheme=scheme)
        g.set_state(w0)
        g.step(3)
        g.sync()
        out.append((g.get_state(), g.stats()[1]))
        g.close()
    for other in out[1:]:
        assert out[0][1] == other[1]
        assert np.array_equal(np.ascontiguousarray(out[0][0]).view(np.uint8), np.ascontiguousarray(other[0]).view(np.uint8))


def test_split_column_pass_with_fields_converging_apart(lib, cuda_device, monkeypatch):
    # 4096^2 half spectra, two fields, the second 1e-4 times the first: its
    # fixed point converges in fewer updates, so later updates run the split
    # column pass with one field inactive (its parts skip their loads and
    # stores).  Split and one-part passes agree bit for bit, each field equals
    # its solo run, and the update counts differ between the fields
    n, Ln, nu, dt = 4096, 2 * math.pi, 1e-3, 2.5e-4
    w = S.ns_power_law(n, batch=1)[0]
    w0 = np.stack([w, 1e-4 * w])
    kw = dict(lx=Ln, ly=Ln, dt=dt, nu=nu, dealias=1, rfft=1, tol=1e-10)
    out = []
    for split in ("1", "0"):
        monkeypatch.setenv("PSS_COL_SPLIT", split)
        g = lib.Grid("ns", n, "fp32", batch=2, **kw)
        g.set_state(w0)
        g.step(2)
        g.sync()
        out.append((g.get_state(), g.stats()[1]))
        g.close()
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0].view(np.uint32), out[1][0].view(np.uint32))
    monkeypatch.setenv("PSS_COL_SPLIT", "1")
    solo_updates = []
    for f in range(2):
        g = lib.Grid("ns", n, "fp32", batch=1, **kw)
        g.set_state(w0[f][None])
        g.step(2)
        g.sync()
        assert np.array_equal(g.get_state()[0].view(np.uint32), out[0][0][f].view(np.uint32))
        solo_updates.append(g.stats()[1])
        g.close()
    assert sum(solo_updates) == out[0][1]
    assert solo_updates[0] != solo_updates[1]

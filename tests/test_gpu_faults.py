"""Host-side fault injection (PSS_FAULT): each injected failure comes back as
a status code through the C ABI, and the process and the handle stay usable.
Nothing here faults, traps or hangs the GPU: the tile-copy case announces
copies that are never started, so the kernels' bounded waits run out."""
import math

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

L = 20 * math.pi


def test_allocation_refused(lib, cuda_device, monkeypatch):
    monkeypatch.setenv("PSS_FAULT", "oom")
    with pytest.raises(lib.PssError) as e:
        lib.Grid("nls", 64, "fp32", lx=L, ly=L, dt=1e-3)
    assert e.value.code == lib.PSS_E_OOM
    monkeypatch.delenv("PSS_FAULT")
    g = lib.Grid("nls", 64, "fp32", lx=L, ly=L, dt=1e-3)
    g.set_state(S.nls_gaussian(64)[None])
    g.step(2)
    assert np.isfinite(g.get_state()).all()
    g.close()


def test_forced_non_convergence(lib, cuda_device, monkeypatch):
    monkeypatch.setenv("PSS_FAULT", "nonconv")
    n, Ln = 64, 2 * math.pi
    g = lib.Grid("ns", n, "fp32", lx=Ln, ly=Ln, dt=2.5e-3, nu=1e-3)
    g.set_state(S.ns_power_law(n)[None])
    with pytest.raises(lib.PssError) as e:
        g.step(2)
        g.sync()
    assert e.value.code == lib.PSS_E_NOT_CONVERGED
    assert np.isfinite(g.get_state()).all()
    g.close()


@pytest.mark.parametrize("land", ["1", "0"])
@pytest.mark.parametrize("n", [256, 1024])
def test_lost_tile_copy_is_reported_and_handle_recovers(lib, cuda_device, monkeypatch, n, land):
    # the column pass's tile copies never arrive: every CTA's bounded wait runs
    # out, it sets the grid's status word and returns; the next synchronising
    # call reports the state as lost, and the handle steps again once the
    # state is set again (the captured step graphs are rebuilt).  Both the
    # landing-buffer pass (a group that gives up stops the other group and
    # waits, bounded, for the copies issued) and the one-buffer pass
    p0 = S.nls_gaussian(n, batch=2)
    monkeypatch.setenv("PSS_PLAN", "0")
    monkeypatch.setenv("PSS_COL_LAND", land)
    monkeypatch.setenv("PSS_FAULT", "tma_timeout")
    g = lib.Grid("nls", n, "fp32", batch=2, lx=L, ly=L, x0=-L / 2, y0=-L / 2, dt=1e-3)
    g.set_state(p0)
    with pytest.raises(lib.PssError) as e:
        g.step(3)
        g.sync()
    assert e.value.code == lib.PSS_E_CUDA
    assert "tile copy" in str(e.value)
    monkeypatch.delenv("PSS_FAULT")
    g.set_state(p0)
    g.step(3)
    g.sync()
    got = g.get_state()
    ref = lib.Grid("nls", n, "fp32", batch=2, lx=L, ly=L, x0=-L / 2, y0=-L / 2, dt=1e-3)
    ref.set_state(p0)
    ref.step(3)
    assert np.array_equal(got.view(np.uint32), ref.get_state().view(np.uint32))
    g.close()
    ref.close()


def test_lost_tile_copy_in_the_split_column_pass(lib, cuda_device, monkeypatch):
    # Navier-Stokes at 4096^2 runs its column pass in two parts per tile: the
    # first parts' copies never arrive, so every CTA gives up on its first
    # item (no second part is claimed, nothing waits on it); the state is
    # reported lost, and the handle steps again, bit for bit as a fresh grid
    n, Ln = 4096, 2 * math.pi
    w0 = S.ns_power_law(n)
    kw = dict(lx=Ln, ly=Ln, dt=2.5e-4, nu=1e-3, dealias=1, rfft=1)
    monkeypatch.setenv("PSS_FAULT", "tma_timeout")
    g = lib.Grid("ns", n, "fp32", **kw)
    g.set_state(w0[None])
    with pytest.raises(lib.PssError) as e:
        g.step(2)
        g.sync()
    assert e.value.code == lib.PSS_E_CUDA
    assert "tile copy" in str(e.value)
    monkeypatch.delenv("PSS_FAULT")
    g.set_state(w0[None])
    g.step(2)
    g.sync()
    ref = lib.Grid("ns", n, "fp32", **kw)
    ref.set_state(w0[None])
    ref.step(2)
    assert np.array_equal(g.get_state().view(np.uint32), ref.get_state().view(np.uint32))
    assert g.stats()[1] == ref.stats()[1]  # set_state restarts the update count
    g.close()
    ref.close()

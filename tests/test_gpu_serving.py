"""Continuous batching: a mixed stream of NLS, sine-Gordon and Navier-Stokes
solves served through shared batched grids gives every request the result it
gets alone (SG and NS bit for bit; NLS within the FP32 tolerance, since the
split-step merges half steps inside each pss_step_n call and the server cuts
a solve into rounds)."""
import numpy as np
import pytest

import synthetic as S
from gpu_util import check

pytestmark = pytest.mark.gpu


def _check(results, reqs):
    from paper_1206_3215_gb300.serving import solve_alone
    for q in reqs:
        got = results[q.rid].state
        ref = solve_alone(q)
        got = got if isinstance(got, tuple) else (got,)
        ref = ref if isinstance(ref, tuple) else (ref,)
        for a, b in zip(got, ref):
            if q.eq == "nls":
                check(a, b, 1e-5)
            else:
                assert np.array_equal(a, b), q.rid


def test_mixed_stream_matches_solo_runs(lib, cuda_device):
    from paper_1206_3215_gb300.serving import Request, Server
    reqs = [Request.from_dict(d) for d in S.serving_mix(24, 1e6, sizes=(64, 128), steps=(20, 60))]
    srv = Server(slots=4, round_max=16)
    results, stats = srv.run(reqs, realtime=False)
    srv.close()
    assert len(results) == len(reqs)
    assert stats["rounds"] > 0 and stats["p99_latency_s"] >= stats["p50_latency_s"] > 0
    _check(results, reqs)


def test_one_pool_at_a_time_still_serves_everything(lib, cuda_device):
    # with room for a single pool, requests of other shapes wait and idle
    # pools are released to admit them
    from paper_1206_3215_gb300.serving import Request, Server
    reqs = [Request.from_dict(d) for d in S.serving_mix(10, 1e6, sizes=(64, 128), steps=(10, 30), seed=99)]
    srv = Server(slots=2, round_max=8, max_pools=1)
    results, stats = srv.run(reqs, realtime=False)
    srv.close()
    assert len(results) == len(reqs)
    _check(results, reqs)


def test_realtime_arrivals_report_latency(lib, cuda_device):
    from paper_1206_3215_gb300.serving import Request, Server
    reqs = [Request.from_dict(d) for d in S.serving_mix(12, 200.0, sizes=(64,), steps=(10, 20), seed=7)]
    srv = Server(slots=4, round_max=10)
    results, stats = srv.run(reqs, realtime=True, timeout=120)
    srv.close()
    assert len(results) == 12
    assert all(r.latency > 0 and r.queued >= 0 for r in results.values())


def test_set_and_get_field_round_trip(lib, cuda_device):
    n = 64
    for eq, state in (("nls", (S.nls_gaussian(n),)), ("sg", S.sg_gaussian(n)), ("ns", (S.taylor_green_2pi(n),))):
        g = lib.Grid(eq, n, "fp64", batch=3, lx=2 * np.pi, ly=2 * np.pi)
        g.set_field(1, *state)
        out = g.get_field(1)
        a = out[0] if isinstance(out, tuple) else out
        check(a, state[0], 1e-13)
        # the other slots hold zeros
        z = g.get_field(0)
        z = z[0] if isinstance(z, tuple) else z
        assert np.abs(z).max() == 0.0


def test_step_n_batch_equals_separate_calls(lib, cuda_device):
    # grids of different equations advanced by one pss_step_n_batch call
    # equal the same grids advanced one call each, bit for bit
    import math
    def make():
        g1 = lib.Grid("nls", 64, "fp32", dt=1e-3)
        g1.set_state(S.nls_gaussian(64)[None])
        g2 = lib.Grid("sg", 64, "fp32", lx=10 * math.pi, ly=10 * math.pi, dt=1e-3, rfft=1)
        g2.set_state(*(a[None] for a in S.sg_gaussian(64)))
        g3 = lib.Grid("ns", 64, "fp32", lx=2 * math.pi, ly=2 * math.pi, dt=2.5e-3, nu=1e-3)
        g3.set_state(S.ns_power_law(64)[None])
        return [g1, g2, g3]
    a, b = make(), make()
    lib.pss_step_n_batch([g.h for g in a], [7, 11, 5])
    for g, k in zip(b, [7, 11, 5]):
        g.step(k)
    for ga, gb in zip(a, b):
        ra, rb = ga.get_state(), gb.get_state()
        ra = ra if isinstance(ra, tuple) else (ra,)
        rb = rb if isinstance(rb, tuple) else (rb,)
        for x, y in zip(ra, rb):
            assert np.array_equal(x, y)
        assert ga.stats() == gb.stats()
    with pytest.raises(lib.PssError):
        lib.pss_step_n_batch([a[0].h, a[1].h], [1, -1])


def _oracle_result(orc, q):
    """The FP64 oracle's solve of request q from the same (rounded) initial field."""
    p = dict(q.params)
    L = p["lx"]
    if q.eq == "nls":
        return (orc.nls_run(q.state[0].astype(np.complex128), L, L, p["dt"], q.steps, merged=True),)
    if q.eq == "sg":
        un, um = orc.sg_init(q.state[0].astype(np.float64), q.state[1].astype(np.float64), L, L, p["dt"])
        un, um = orc.sg_run(un, um, L, L, p["dt"], q.steps)
        return orc.sg_fields(un, um)
    wh, _, ok = orc.ns_run(orc.ns_init(q.state[0].astype(np.float64), True), L, L, p["nu"], p["dt"], q.steps,
                           tol=1e-10)
    assert ok
    return (orc.ns_field(wh),)


def test_mix_up_to_1024_matches_solo_runs_and_oracle(lib, orc, cuda_device):
    # the serving workload's shapes up to 1024^2 (one pool per equation and
    # size, 1 to 8 slots each), requests admitted as slots free up; every
    # result equals its solo run, and for each equation the largest request
    # also matches the FP64 oracle (FP32 targets: 1e-5, sine-Gordon 2e-5)
    from paper_1206_3215_gb300.serving import Request, Server
    reqs = [Request.from_dict(d) for d in S.serving_mix(40, 1e6, sizes=(128, 256, 512, 1024), steps=(10, 40),
                                                         seed=S.SEED_BASE + 40, fields_per_shape=2)]
    srv = Server(slots=8, round_max=16)
    results, stats = srv.run(reqs, realtime=False)
    srv.close()
    assert len(results) == len(reqs) and stats["pools"] >= 6
    _check(results, reqs)
    for eq in ("nls", "sg", "ns"):
        mine = [q for q in reqs if q.eq == eq and q.n >= 512]
        assert mine, eq
        q = max(mine, key=lambda r: (r.n, -r.steps))
        got = results[q.rid].state
        got = got if isinstance(got, tuple) else (got,)
        for a, b in zip(got, _oracle_result(orc, q)):
            check(a, b, 2e-5 if eq == "sg" else 1e-5)

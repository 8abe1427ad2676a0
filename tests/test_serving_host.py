"""Host-side scheduling rules of the continuous-batching server (no GPU):
slots per pool, the device bytes a pool is admitted against, and the key
that decides which requests share a pool."""
from paper_1206_3215_gb300 import serving


def test_slots_per_pool_follow_the_grid_size():
    s = serving.Server(slots=8, pool_points=1 << 22)
    assert s._slots_for(("nls", 128, "fp32", ())) == 8
    assert s._slots_for(("nls", 1024, "fp32", ())) == 4
    assert s._slots_for(("sg", 2048, "fp32", ())) == 1
    assert s._slots_for(("ns", 4096, "fp32", ())) == 1  # at least one slot


def test_pool_bytes_count_every_slot():
    s = serving.Server(slots=8, pool_points=1 << 22)
    for eq in ("nls", "sg", "ns"):
        for prec in ("fp32", "fp64"):
            key = (eq, 512, prec, ())
            per_point = serving.BYTES_PER_POINT[(eq, prec)]
            assert s._pool_bytes(key) == per_point * 512 * 512 * s._slots_for(key) + (4 << 20)
    # FP64 doubles the bytes of every complex work array
    assert serving.BYTES_PER_POINT[("sg", "fp64")] == 2 * serving.BYTES_PER_POINT[("sg", "fp32")]


def test_requests_share_a_pool_only_with_equal_parameters():
    a = serving.Request.from_dict({"rid": 1, "eq": "sg", "n": 256, "steps": 10, "state": (0, 0),
                                   "params": {"dt": 1e-3, "rfft": 1}})
    b = serving.Request.from_dict({"rid": 2, "eq": "sg", "n": 256, "steps": 99, "state": (0, 0),
                                   "params": {"rfft": 1, "dt": 1e-3}})
    c = serving.Request.from_dict({"rid": 3, "eq": "sg", "n": 256, "steps": 10, "state": (0, 0),
                                   "params": {"dt": 2e-3, "rfft": 1}})
    assert a.key == b.key  # parameter order does not matter, step counts do not split pools
    assert a.key != c.key
    assert a.precision == "fp32" and a.arrival == 0.0

"""The bench's recorded profile data (no GPU): the DRAM traffic it reports
next to the roofline comes from profiles/traffic.json, keyed by the kernel
names the bench uses and by a hash of the kernel sources."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _records():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        return json.load(f)


def test_every_roofline_kernel_has_a_record():
    rec = _records()
    for name in bench.ROOFLINE_KERNELS.values():
        assert name in rec, name


def test_records_are_complete_and_plausible():
    # one read and one write of the 256 MiB state per pass: the measured DRAM
    # bytes of a launch cannot be far from that without re-reads (above) or
    # a kernel that skips work (below)
    algorithmic = 2 * 32 * 1024 * 1024 * 8
    for name, r in _records().items():
        assert set(r) >= {"dram_bytes_per_launch", "dram_read_bytes", "dram_write_bytes", "source_hash",
                          "source_files", "capture"}, name
        assert r["dram_bytes_per_launch"] == r["dram_read_bytes"] + r["dram_write_bytes"]
        assert 0.5 * algorithmic < r["dram_bytes_per_launch"] < 1.5 * algorithmic
        assert tuple(r["source_files"]) == bench.NLS_KERNEL_FILES
        assert os.path.exists(os.path.join(ROOT, r["capture"]))
        assert len(r["source_hash"]) == 16 and int(r["source_hash"], 16) >= 0


def test_source_hash_is_a_function_of_the_sources():
    h = bench.kernel_source_hash()
    assert h == bench.kernel_source_hash() and len(h) == 16
    assert bench.kernel_source_hash(bench.NLS_KERNEL_FILES[:-1]) != h

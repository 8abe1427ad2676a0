"""The bench's multi-GPU path is replicas (independent fields per rank, no
collective on the data path).  Its host-side logic -- the max-over-ranks
timing and the whole-job rate -- runs here as two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" 1.0 + r seconds for the same work
    t = bench.reduce_max(1.0 + rank)
    rate = bench.whole_job_rate(1e9, world, t)
    dist.barrier()
    q.put((rank, t, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in out:
        assert t == 2.0                      # the slowest rank's time on every rank
        assert rate == pytest.approx(1e9)    # 2 ranks x 1e9 units / 2 s


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0

"""Continuous-batching server for pseudospectral solves on one GPU.

Requests (an equation, a grid size, a number of steps and an initial state)
arrive over time.  Requests with the same equation, grid size, precision and
parameters share a *pool*: one batched grid whose fields are slots.  A pool
advances all its occupied slots together in *rounds* of
min(remaining steps over its slots, round_max) steps, enqueued on the pool's
own CUDA stream, so pools of different sizes and equations run concurrently
on the device.  Between rounds, finished slots are read back and freed and
waiting requests are admitted into free slots (continuous batching: a request
does not wait for the whole batch to finish).  A new pool is created only
when the device has room for it (free memory minus a reserve); otherwise the
request waits, and idle empty pools are released to make room.

A pool of N x N grids has min(slots, pool_points / N^2) slots: small grids
are batched to fill the GPU, while a 2048^2 field, which fills it alone,
does not wait for the steps of seven others.

Every field evolves exactly as it would alone: a batch does not couple its
fields (sine-Gordon and Navier-Stokes give bit-identical fields; the NLS
split-step merges the half steps inside one pss_step_n call, so a solve cut
into rounds differs from a single call by rounding only).

Host-side scheduling only: all arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses
import math
import time
from collections import deque

import numpy as np

from . import Grid, pss_step_n_batch

# device bytes per grid point of one slot (complex work arrays; sine-Gordon
# counts the half-spectrum copies as well)
BYTES_PER_POINT = {("nls", "fp32"): 3 * 8, ("nls", "fp64"): 3 * 16,
                   ("sg", "fp32"): 7 * 8, ("sg", "fp64"): 7 * 16,
                   ("ns", "fp32"): 7 * 8, ("ns", "fp64"): 7 * 16}


@dataclasses.dataclass
class Request:
    rid: int
    eq: str                      # "nls" | "sg" | "ns"
    n: int                       # grid points per side
    steps: int
    state: tuple                 # host arrays: (psi,) | (u0, v0) | (w0,)
    arrival: float = 0.0         # seconds after the start of the run
    precision: str = "fp32"
    params: tuple = ()           # sorted (name, value) pairs passed to the grid

    @property
    def key(self):
        return (self.eq, self.n, self.precision, self.params)

    @classmethod
    def from_dict(cls, d: dict) -> "Request":
        return cls(d["rid"], d["eq"], d["n"], d["steps"], tuple(d["state"]), d.get("arrival", 0.0),
                   d.get("precision", "fp32"), tuple(sorted(d.get("params", {}).items())))


@dataclasses.dataclass
class Result:
    rid: int
    state: object
    latency: float               # completion - arrival, seconds
    queued: float                # admission - arrival, seconds


class Pool:
    def __init__(self, key, slots: int):
        import torch
        eq, n, precision, params = key
        self.key = key
        self.stream = torch.cuda.Stream()
        self.grid = Grid(eq, n, precision, batch=slots, stream=self.stream.cuda_stream, **dict(params))
        self.slots: list = [None] * slots    # [request, remaining, admitted_at] or None
        self.event = None                    # completion event of the round in flight
        self.round = 0
        self.last_used = time.perf_counter()

    def free_slot(self):
        for i, s in enumerate(self.slots):
            if s is None:
                return i
        return None

    def occupied(self):
        return [i for i, s in enumerate(self.slots) if s is not None]

    def busy(self):
        return self.event is not None

    def close(self):
        self.grid.close()


class Server:
    """Admits, batches and advances requests; see the module docstring."""

    def __init__(self, slots: int = 8, round_max: int = 50, reserve_bytes: int = 2 << 30,
                 max_pools: int = 64, pool_points: int = 1 << 22):
        # a pool of N x N grids gets min(slots, pool_points / N^2) slots (at
        # least 1): one 2048^2 field already fills the GPU, and batching more of
        # them only makes each request wait for the others' steps
        self.slots = slots
        self.pool_points = pool_points
        self.round_max = round_max
        self.reserve = reserve_bytes
        self.max_pools = max_pools
        self.pools: dict = {}
        self.results: dict = {}
        self.rounds = 0
        self.point_steps = 0

    def _slots_for(self, key) -> int:
        n = key[1]
        return max(1, min(self.slots, self.pool_points // (n * n)))

    # -- memory admission --------------------------------------------------
    def _pool_bytes(self, key):
        eq, n, precision, _ = key
        return BYTES_PER_POINT[(eq, precision)] * n * n * self._slots_for(key) + (4 << 20)

    def _room_for(self, key) -> bool:
        import torch
        free, _ = torch.cuda.mem_get_info()
        return free - self._pool_bytes(key) >= self.reserve and len(self.pools) < self.max_pools

    def _release_idle(self):
        for k, p in list(self.pools.items()):
            if not p.busy() and not p.occupied():
                p.close()
                del self.pools[k]
                return True
        return False

    def _pool_for(self, key):
        p = self.pools.get(key)
        if p is not None:
            return p
        while not self._room_for(key):
            if not self._release_idle():
                return None
        p = Pool(key, self._slots_for(key))
        self.pools[key] = p
        return p

    # -- one scheduling pass -------------------------------------------------
    def _admit(self, waiting: deque, now: float, t0: float):
        blocked = set()
        for _ in range(len(waiting)):
            req = waiting.popleft()
            if req.key in blocked:
                waiting.append(req)
                continue
            pool = self._pool_for(req.key)
            if pool is None or pool.busy() or pool.free_slot() is None:
                blocked.add(req.key)
                waiting.append(req)
                continue
            i = pool.free_slot()
            pool.grid.set_field(i, *req.state)
            pool.slots[i] = [req, req.steps, now]

    def _launch(self):
        import torch
        ready = []
        for pool in self.pools.values():
            occ = pool.occupied()
            if pool.busy() or not occ:
                continue
            ready.append((pool, min(min(pool.slots[i][1] for i in occ), self.round_max)))
        if not ready:
            return
        # one call enqueues a round on every ready pool's stream
        pss_step_n_batch([p.grid.h for p, _ in ready], [r for _, r in ready])
        for pool, r in ready:
            ev = torch.cuda.Event()
            ev.record(pool.stream)
            pool.event = (ev, r)
            pool.round += 1
            pool.last_used = time.perf_counter()
            self.rounds += 1

    def _complete(self, t0: float):
        done = 0
        for pool in self.pools.values():
            if pool.event is None or not pool.event[0].query():
                continue
            _, r = pool.event
            pool.event = None
            now = time.perf_counter() - t0
            for i in pool.occupied():
                slot = pool.slots[i]
                slot[1] -= r
                self.point_steps += r * pool.grid.nx * pool.grid.ny
                if slot[1] == 0:
                    req = slot[0]
                    out = pool.grid.get_field(i)
                    t_done = time.perf_counter() - t0
                    self.results[req.rid] = Result(req.rid, out, t_done - req.arrival, slot[2] - req.arrival)
                    pool.slots[i] = None
                    done += 1
        return done

    def run(self, requests, realtime: bool = True, timeout: float = 600.0):
        """Serve `requests` (arrival offsets in seconds; ignored unless
        realtime).  Returns the results by request id and the run statistics."""
        pending = deque(sorted(requests, key=lambda q: q.arrival))
        waiting: deque = deque()
        total = len(pending)
        t0 = time.perf_counter()
        while len(self.results) < total:
            now = time.perf_counter() - t0
            if now > timeout:
                raise TimeoutError(f"served {len(self.results)} of {total} requests in {timeout} s")
            while pending and (not realtime or pending[0].arrival <= now):
                q = pending.popleft()
                if not realtime:
                    q = dataclasses.replace(q, arrival=now)
                waiting.append(q)
            self._complete(t0)
            self._admit(waiting, now, t0)
            self._launch()
            if not any(p.busy() for p in self.pools.values()) and not waiting and pending:
                time.sleep(min(0.001, max(0.0, pending[0].arrival - now)))
            else:
                time.sleep(0)
        wall = time.perf_counter() - t0
        lat = np.array([r.latency for r in self.results.values()])
        stats = {
            "requests": total, "wall_s": wall, "rounds": self.rounds, "pools": len(self.pools),
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_queue_s": float(np.mean([r.queued for r in self.results.values()])),
            "gpt_steps_per_s": self.point_steps / wall / 1e9,
        }
        return self.results, stats

    def close(self):
        for p in self.pools.values():
            p.close()
        self.pools.clear()


def solve_alone(req: Request):
    """The same solve on its own grid in one pss_step_n call."""
    g = Grid(req.eq, req.n, req.precision, batch=1, **dict(req.params))
    g.set_field(0, *req.state)
    g.step(req.steps)
    out = g.get_field(0)
    g.close()
    return out

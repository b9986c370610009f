"""Continuous-batching QP serving over the batched C ABI.

A pool of problem IDs stays resident on the GPU (scaled data, ρ̄, last
iterates).  Requests name a problem ID and bring new q, l, u (§6 vectors as
parameters); each warm-starts from that ID's previous solution (§6 warm
start).  The loop admits arrived requests onto free launch slots — each slot
is an independent stream, so requests that arrive while others are on the
GPU start as soon as CTAs free up and their work overlaps on the device —
as long as the device footprint of the work in flight stays within a budget.
Large problems (solved by clusters of CTAs, see osqp_batch_uses_cluster)
are launched alone on their slot, at most `large_slots` of them at a time,
so that the other slots stay free for small requests, which a launch takes
in arrival order up to `max_batch` (no cap by default).
A problem ID has at most one request in flight; later requests for it wait.
Host-side bookkeeping only: every numeric step runs in the library.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import _binding as B
from .solver import BatchSolver


@dataclasses.dataclass
class Request:
    pid: int
    t_arrival: float            # seconds after the start of the run
    q: np.ndarray | None = None
    l: np.ndarray | None = None
    u: np.ndarray | None = None
    t_launch: float = float("nan")
    t_done: float = float("nan")
    status: int = 0
    iter: int = 0
    x: np.ndarray | None = None

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


@dataclasses.dataclass
class RunStats:
    requests: int
    wall: float
    solves_per_s: float
    p50_ms: float
    p99_ms: float
    mean_queue_ms: float
    max_inflight_bytes: int
    launches: int
    dropped: int = 0
    host_launch_s: float = 0.0   # host time inside osqp_batch_launch
    host_result_s: float = 0.0   # host time reading results (osqp_batch_get)


class Server:
    def __init__(self, qps, slots: int = 4, footprint_budget: int | None = None,
                 stream: int | None = None, prime: bool = True, large_slots: int | None = None,
                 **settings):
        if not 1 <= slots <= B.OSQP_BATCH_MAX_SLOTS:
            raise ValueError(f"slots must be in 1..{B.OSQP_BATCH_MAX_SLOTS}")
        self.qps = qps
        self.slots = slots
        # slots that large requests may hold at once (the rest serve small ones)
        self.large_slots = max(1, slots // 2) if large_slots is None else max(1, large_slots)
        self.bs = BatchSolver(qps, stream=stream, **settings)
        self.h = self.bs.handle
        self.footprint = [B.osqp_batch_footprint(self.h, i) for i in range(len(qps))]
        # large problems run on clusters of CTAs: they are launched alone
        self.large = [B.osqp_batch_uses_cluster(self.h, i) for i in range(len(qps))]
        self.budget = footprint_budget if footprint_budget is not None else sum(self.footprint)
        if prime:  # cold solve of every resident problem (setup phase)
            self.bs.solve()

    def run(self, requests, max_batch: int | None = None, keep_x: bool = False,
            deadline: float | None = None, clock=time.perf_counter) -> RunStats:
        """Serve `requests` (arrival times relative to the start).  With a
        deadline (seconds), requests not launched by then are dropped (their
        status stays 0) and the run ends when the work in flight finishes —
        the way an overloaded server is measured."""
        reqs = sorted(requests, key=lambda r: r.t_arrival)
        for r in reqs:  # the library reads n (q) and m (l, u) values per request
            qp = self.qps[r.pid]
            for name, v, size in (("q", r.q, qp.n), ("l", r.l, qp.m), ("u", r.u, qp.m)):
                if v is not None and np.size(v) != size:
                    raise ValueError(f"request for problem {r.pid}: {name} has {np.size(v)} "
                                     f"entries, expected {size}")
        pending = collections.deque()
        free = list(range(self.slots))[::-1]
        busy = {}
        busy_large = 0
        host_launch = host_result = 0.0
        inflight_ids = set()
        inflight_bytes = 0
        max_inflight = 0
        launches = 0
        nxt = 0
        done = 0
        t0 = clock()
        dropped = 0
        while done + dropped < len(reqs):
            now = clock() - t0
            if deadline is not None and now > deadline:
                # stop admitting: drop what has not been launched
                dropped = len(reqs) - done - sum(len(v) for v in busy.values())
                pending.clear()
                nxt = len(reqs)
            while nxt < len(reqs) and reqs[nxt].t_arrival <= now:
                pending.append(reqs[nxt])
                nxt += 1
            progressed = False
            for slot in list(busy):
                if B.osqp_batch_slot_query(self.h, slot):
                    t_done = clock() - t0
                    for r in busy[slot]:
                        x, _, _, info = B.osqp_batch_get(self.h, r.pid, self.qps[r.pid].n,
                                                         self.qps[r.pid].m)
                        r.t_done, r.status, r.iter = t_done, info.status, info.iter
                        if keep_x:
                            r.x = x
                        inflight_ids.discard(r.pid)
                        inflight_bytes -= self.footprint[r.pid]
                    host_result += clock() - t0 - t_done
                    if len(busy[slot]) == 1 and self.large[busy[slot][0].pid]:
                        busy_large -= 1
                    done += len(busy[slot])
                    del busy[slot]
                    free.append(slot)
                    progressed = True
            if pending and free and (deadline is None or now <= deadline):
                take, ids, add = [], set(), 0
                for r in pending:
                    if r.pid in inflight_ids or r.pid in ids:
                        continue
                    if self.large[r.pid]:
                        # alone on its slot, and only while a large slot is free
                        if take or busy_large >= self.large_slots:
                            continue
                        if inflight_bytes + self.footprint[r.pid] > self.budget and inflight_bytes:
                            continue
                        take.append(r)
                        ids.add(r.pid)
                        add += self.footprint[r.pid]
                        break
                    fp = self.footprint[r.pid]
                    if inflight_bytes + add + fp > self.budget and (take or inflight_bytes):
                        continue
                    take.append(r)
                    ids.add(r.pid)
                    add += fp
                    if max_batch and len(take) >= max_batch:
                        break
                if take:
                    taken = set(id(r) for r in take)
                    pending = collections.deque(r for r in pending if id(r) not in taken)
                    slot = free.pop()
                    t_h = clock()
                    B.osqp_batch_launch(self.h, slot, [r.pid for r in take], [r.q for r in take],
                                        [r.l for r in take], [r.u for r in take])
                    host_launch += clock() - t_h
                    if len(take) == 1 and self.large[take[0].pid]:
                        busy_large += 1
                    t_l = clock() - t0
                    for r in take:
                        r.t_launch = t_l
                    busy[slot] = take
                    inflight_ids |= ids
                    inflight_bytes += add
                    max_inflight = max(max_inflight, inflight_bytes)
                    launches += 1
                    progressed = True
            if not progressed:
                time.sleep(0.0)
        wall = clock() - t0
        served = [r for r in reqs if r.t_done == r.t_done]  # completed (not NaN)
        lat = np.array([r.latency for r in served]) if served else np.zeros(1)
        queue = np.array([r.t_launch - r.t_arrival for r in served]) if served else np.zeros(1)
        return RunStats(len(served), wall, len(served) / wall, 1e3 * float(np.percentile(lat, 50)),
                        1e3 * float(np.percentile(lat, 99)), 1e3 * float(queue.mean()),
                        max_inflight, launches, len(reqs) - len(served), host_launch, host_result)

    def close(self):
        self.bs.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def poisson_requests(qps, rate: float, duration: float, seed: int = 0, perturb: float = 0.05):
    """Requests with exponential inter-arrival times (rate per second) over
    `duration` seconds; each picks a problem ID uniformly and perturbs its
    q, l, u around the pool problem's values."""
    from .problems import perturb_vectors
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        pid = int(rng.integers(len(qps)))
        q, l, u = perturb_vectors(rng, qps[pid], perturb)
        out.append(Request(pid, t, q, l, u))
    return out


def shard_requests(requests, mine):
    """The requests of a global stream that name this rank's problem IDs
    (`mine`, global indices as returned by dist.shard), renumbered to the
    rank's local problem list; arrival times and vectors unchanged."""
    local_of = {g: k for k, g in enumerate(mine)}
    return [Request(local_of[r.pid], r.t_arrival, r.q, r.l, r.u) for r in requests
            if r.pid in local_of]

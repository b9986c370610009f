"""Multi-GPU host logic: one process per GPU, problems sharded across ranks.

The solver has no data-path collective: independent problems (a batch, a
serving pool) are partitioned across ranks by estimated work, each rank
solves its share on its own GPU, and only host-side summaries (timings,
counts, per-problem statuses) are combined.  A single large problem runs as
independent replicas.  Everything here is plain torch.distributed and runs
with the gloo backend on CPU as well as with nccl on GPUs.
"""
from __future__ import annotations

import heapq
import os

import torch
import torch.distributed as dist


def env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str, device: torch.device | None = None):
    """Initialise the default process group (loopback rendezvous unless the
    launcher set MASTER_ADDR)."""
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    kw = {"device_id": device} if (backend == "nccl" and device is not None) else {}
    dist.init_process_group(backend, **kw)


def lpt_partition(weights, parts: int):
    """Longest-processing-time assignment of items to `parts` bins: items in
    decreasing weight go to the currently lightest bin (ties: lowest bin
    index, then lowest item index), which keeps the heaviest bin within 4/3
    of the optimum.  Returns one sorted index list per bin."""
    if parts < 1:
        raise ValueError("parts must be positive")
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    heap = [(0.0, b) for b in range(parts)]
    bins = [[] for _ in range(parts)]
    for i in order:
        load, b = heapq.heappop(heap)
        bins[b].append(i)
        heapq.heappush(heap, (load + float(weights[i]), b))
    return [sorted(b) for b in bins]


def shard(weights, rank: int, world: int):
    """Indices owned by `rank` under lpt_partition."""
    return lpt_partition(weights, world)[rank]


def _reduce(value: float, op, device) -> float:
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t[0])


def max_over_ranks(value: float, device=None) -> float:
    return _reduce(value, dist.ReduceOp.MAX, device or "cpu")


def sum_over_ranks(value: float, device=None) -> float:
    return _reduce(value, dist.ReduceOp.SUM, device or "cpu")


def gather_objects(obj):
    """All ranks' objects in rank order (host-side summaries only)."""
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out


class ShardedBatch:
    """One set of independent problems partitioned across ranks.

    Every rank holds the same list of work estimates (one per problem of the
    global set); lpt_partition assigns each problem to one rank, each rank
    generates and solves only its share on its own GPU, and results are
    combined on the host on request.  make_problem(i) builds global problem
    i; make_solver(problems) returns an object with solve(), result(k) (the
    k-th local problem) and close() — the batched GPU solver in the product
    path.  No collective touches the data path: the gather moves host
    objects after the solve."""

    def __init__(self, weights, make_problem, make_solver, rank: int | None = None,
                 world: int | None = None):
        if rank is None or world is None:
            ws, rk, _ = env()
            world = ws if world is None else world
            rank = rk if rank is None else rank
        self.rank, self.world = rank, world
        self.index = shard(weights, rank, world)
        self.problems = [make_problem(i) for i in self.index]
        self.solver = make_solver(self.problems) if self.problems else None

    def solve(self):
        if self.solver is not None:
            self.solver.solve()

    def local_results(self):
        """{global index: result} of this rank's problems."""
        if self.solver is None:
            return {}
        return {i: self.solver.result(k) for k, i in enumerate(self.index)}

    def gather(self, pick=lambda r: r):
        """{global index: pick(result)} of every rank's problems, on every
        rank (pick keeps the host objects small: e.g. status and x)."""
        merged = {}
        for part in gather_objects({i: pick(r) for i, r in self.local_results().items()}):
            merged.update(part)
        return merged

    def close(self):
        if self.solver is not None:
            self.solver.close()
            self.solver = None

"""Multi-rank host logic with two gloo ranks on CPU: problems are sharded by
work across ranks, each rank solves its share (here with the CPU oracle, so
no GPU is needed), and the gathered results equal a single-process solve;
timings combine as max over ranks, counts as sums."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_1711_08013_gb300 import dist as D
from paper_1711_08013_gb300 import problems as pb


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_lpt_partition_properties():
    rng = np.random.default_rng(0)
    w = rng.lognormal(0, 1.5, size=200)
    for parts in (1, 2, 3, 8):
        bins = D.lpt_partition(w, parts)
        flat = sorted(i for b in bins for i in b)
        assert flat == list(range(len(w)))
        loads = [w[b].sum() for b in bins]
        # LPT guarantee: the heaviest bin is within 4/3 of the optimum (≥ mean, ≥ max item)
        lower = max(w.sum() / parts, w.max())
        assert max(loads) <= 4.0 / 3.0 * lower + 1e-9
    assert D.lpt_partition([5.0, 1.0, 1.0], 2) == [[0], [1, 2]]


def test_lpt_within_grahams_bound_of_the_optimum():
    """Graham's bound for longest-processing-time scheduling: the heaviest
    bin is at most (4/3 − 1/(3m)) times the optimal makespan, the optimum
    found here by enumerating every assignment of up to 9 items."""
    import itertools
    rng = np.random.default_rng(5)
    for trial in range(40):
        parts = int(rng.integers(2, 4))
        w = rng.lognormal(0, 1.0, size=int(rng.integers(parts + 1, 10)))
        opt = min(max(np.bincount(a, weights=w, minlength=parts))
                  for a in itertools.product(range(parts), repeat=len(w)))
        lpt = max(w[b].sum() for b in D.lpt_partition(w, parts))
        assert lpt <= (4.0 / 3.0 - 1.0 / (3 * parts)) * opt + 1e-12, (trial, lpt, opt)


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from oracle import oracle as O
    D.init("gloo")
    qps = pb.mpc_batch(10, seed=3400, nx_range=(3, 6), T_range=(4, 8))
    weights = [q.A.nnz + q.n + q.m for q in qps]
    mine = D.shard(weights, rank, world)
    results = {i: O.solve(qps[i]).x.tolist() for i in mine}
    gathered = D.gather_objects(results)
    t = D.max_over_ranks(float(rank + 1))
    c = D.sum_over_ranks(float(len(mine)))
    if rank == 0:
        merged = {}
        for part in gathered:
            merged.update(part)
        np.save(os.path.join(out_dir, "merged.npy"),
                np.array([merged[i] for i in range(len(qps))], dtype=object), allow_pickle=True)
        with open(os.path.join(out_dir, "reduced.txt"), "w") as f:
            f.write(f"{t} {c}\n")
    import torch.distributed as dist
    dist.barrier()
    dist.destroy_process_group()


class _OracleBatch:
    """CPU stand-in for the batched GPU solver (same solve/result/close
    interface), so the sharding and gather of the product path run here."""

    def __init__(self, qps):
        self.qps = qps
        self.res = None

    def solve(self):
        from oracle import oracle as O
        self.res = [O.solve(q) for q in self.qps]

    def result(self, k):
        return self.res[k]

    def close(self):
        self.res = None


def _sharded_worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    D.init("gloo")
    spec = pb.mpc_batch_spec(12, seed=3500, nx_range=(3, 6), T_range=(4, 8))
    weights = [pb.mpc_spec_work(nx, T) for nx, T, _ in spec]
    sb = D.ShardedBatch(weights, lambda i: pb.mpc(spec[i][0], spec[i][1], seed=spec[i][2]),
                        _OracleBatch)
    sb.solve()
    merged = sb.gather(lambda r: (r.status, r.x.tolist()))
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(" ".join(map(str, sb.index)) + "\n")
    if rank == 0:
        np.save(os.path.join(out_dir, "sharded.npy"),
                np.array([merged[i][1] for i in range(len(spec))], dtype=object),
                allow_pickle=True)
    sb.close()
    import torch.distributed as dist
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_batch_product_path(tmp_path, oracle_mod):
    """The sharding object that bench.py uses for the batched workload: two
    ranks split one 12-problem set by LPT on the generator's work estimates,
    each builds and solves only its share (the batched solver replaced by
    the oracle on CPU), and the gathered results equal a single-process
    solve of the whole set; the two shares are disjoint and cover it."""
    port = _free_port()
    mp.spawn(_sharded_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    shares = [list(map(int, open(tmp_path / f"rank{r}.txt").read().split())) for r in range(2)]
    assert sorted(shares[0] + shares[1]) == list(range(12)) and shares[0] and shares[1]
    merged = np.load(tmp_path / "sharded.npy", allow_pickle=True)
    spec = pb.mpc_batch_spec(12, seed=3500, nx_range=(3, 6), T_range=(4, 8))
    for i, (nx, T, sd) in enumerate(spec):
        ref = oracle_mod.solve(pb.mpc(nx, T, seed=sd)).x
        assert np.array_equal(np.asarray(merged[i]), ref)


def test_two_rank_sharded_solve(tmp_path, oracle_mod):
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    merged = np.load(tmp_path / "merged.npy", allow_pickle=True)
    qps = pb.mpc_batch(10, seed=3400, nx_range=(3, 6), T_range=(4, 8))
    for i, qp in enumerate(qps):
        ref = oracle_mod.solve(qp).x
        assert np.array_equal(np.asarray(merged[i]), ref)
    t, c = map(float, open(tmp_path / "reduced.txt").read().split())
    assert t == 2.0 and c == 10.0


def _serve_worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_1711_08013_gb300.serve import poisson_requests, shard_requests
    D.init("gloo")
    qps = [pb.random_qp(n, seed=500 + n) for n in (4, 6, 9, 12, 5, 7)]
    weights = [q.A.nnz for q in qps]
    mine = D.shard(weights, rank, world)
    reqs = poisson_requests(qps, rate=3000.0, duration=0.02, seed=5)
    local = shard_requests(reqs, mine)
    rows = [(mine[r.pid], r.t_arrival, float(r.q.sum())) for r in local]
    for part_rank, part in enumerate(D.gather_objects(rows)):
        if rank == 0:
            with open(os.path.join(out_dir, f"serve{part_rank}.txt"), "w") as f:
                for g, t, qs in part:
                    f.write(f"{g} {t!r} {qs!r}\n")
    import torch.distributed as dist
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_serving_shards_one_request_stream(tmp_path):
    """The serving path of bench.py at two ranks: one pool of problem IDs
    split by LPT, one global request stream filtered by each rank to its IDs;
    the two local streams are disjoint and together are exactly the global
    stream (same IDs, arrival times and perturbed vectors)."""
    from paper_1711_08013_gb300.serve import poisson_requests
    port = _free_port()
    mp.spawn(_serve_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    got = []
    for r in range(2):
        for line in open(tmp_path / f"serve{r}.txt"):
            g, t, qs = line.split()
            got.append((int(g), float(t), float(qs)))
    qps = [pb.random_qp(n, seed=500 + n) for n in (4, 6, 9, 12, 5, 7)]
    ref = [(r.pid, r.t_arrival, float(r.q.sum()))
           for r in poisson_requests(qps, rate=3000.0, duration=0.02, seed=5)]
    assert len(ref) > 20
    assert sorted(got) == sorted(ref)

"""Host logic of the continuous-batching server (no GPU): the admission loop
of serve.Server driven against a fake batch backend and a fake clock.  Every
launch is checked for the server's invariants: at most one request per
problem ID in flight, the device footprint in flight within the budget
(a single request alone may exceed it), large problems launched alone, at
most `slots` launches in flight and at most `max_batch` requests per
launch; every request is served exactly once, after it arrived, or dropped
after the deadline without a launch."""
import types

import numpy as np
import pytest

from paper_1711_08013_gb300 import serve


class FakeBackend:
    OSQP_BATCH_MAX_SLOTS = 32

    def __init__(self, footprint, large, budget, slots, max_batch, finish_after):
        self.fp, self.lg, self.budget = footprint, large, budget
        self.nslots, self.max_batch, self.finish_after = slots, max_batch, finish_after
        self.running = {}      # slot -> [pids, queries]
        self.launched = []     # (slot, pids)

    def osqp_batch_footprint(self, h, i):
        return self.fp[i]

    def osqp_batch_uses_cluster(self, h, i):
        return int(self.lg[i])

    def osqp_batch_launch(self, h, slot, pids, qs, ls, us):
        assert 0 <= slot < self.nslots and slot not in self.running
        busy = [p for v in self.running.values() for p in v[0]]
        assert len(set(pids)) == len(pids) and not set(pids) & set(busy)
        if self.max_batch:
            assert len(pids) <= self.max_batch
        if any(self.lg[p] for p in pids):
            assert len(pids) == 1
        new = sum(self.fp[p] for p in pids)
        old = sum(self.fp[p] for p in busy)
        assert old + new <= self.budget or (len(pids) == 1 and old == 0)
        assert qs is None or len(qs) == len(pids)
        self.running[slot] = [list(pids), 0]
        self.launched.append((slot, list(pids)))

    def osqp_batch_slot_query(self, h, slot):
        st = self.running[slot]
        st[1] += 1
        if st[1] >= self.finish_after:
            del self.running[slot]
            return 1
        return 0

    def osqp_batch_get(self, h, pid, n, m):
        return np.full(n, float(pid)), np.zeros(m), np.zeros(m), types.SimpleNamespace(status=1, iter=7)


class FakeBatchSolver:
    def __init__(self, qps, stream=None, **settings):
        self.handle = object()
        self.solved = 0

    def solve(self):
        self.solved += 1

    def close(self):
        pass


def make_server(monkeypatch, nprob, slots, budget, large, max_batch, finish_after, seed):
    rng = np.random.default_rng(seed)
    fp = [int(v) for v in rng.integers(100, 1000, nprob)]
    lg = [i in large for i in range(nprob)]
    be = FakeBackend(fp, lg, budget if budget is not None else sum(fp), slots, max_batch,
                     finish_after)
    monkeypatch.setattr(serve, "B", be)
    monkeypatch.setattr(serve, "BatchSolver", FakeBatchSolver)
    qps = [types.SimpleNamespace(n=3 + i % 5, m=2 + i % 3) for i in range(nprob)]
    return serve.Server(qps, slots=slots, footprint_budget=budget), be, qps


def fake_clock(step):
    t = [0.0]

    def clock():
        t[0] += step
        return t[0]
    return clock


def requests(rng, nprob, count, rate):
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    return [serve.Request(int(rng.integers(nprob)), float(ti)) for ti in t]


@pytest.mark.parametrize("slots,budget,max_batch,large", [
    (4, None, None, ()),
    (2, 1500, None, ()),
    (8, 2500, 3, (1, 5)),
    (1, 800, None, (0,)),
])
def test_admission_invariants_and_every_request_served(monkeypatch, slots, budget, max_batch, large):
    srv, be, qps = make_server(monkeypatch, 12, slots, budget, large, max_batch, 4, seed=slots)
    rng = np.random.default_rng(7)
    reqs = requests(rng, 12, 200, rate=400.0)
    st = srv.run(reqs, max_batch=max_batch, keep_x=True, clock=fake_clock(1e-3))
    assert st.requests == len(reqs) and st.dropped == 0
    launched = [p for _, pids in be.launched for p in pids]
    assert sorted(launched) == sorted(r.pid for r in reqs)
    assert st.launches == len(be.launched)
    for r in reqs:
        assert r.status == 1 and r.iter == 7
        assert r.t_arrival <= r.t_launch <= r.t_done
        assert np.all(r.x == r.pid)          # the result of its own problem
    assert st.max_inflight_bytes <= max(srv.budget, max(be.fp))
    for p in large:
        assert all(len(pids) == 1 for _, pids in be.launched if p in pids)


def test_requests_for_one_problem_are_served_in_arrival_order(monkeypatch):
    srv, be, _ = make_server(monkeypatch, 3, 4, None, (), None, 3, seed=1)
    reqs = [serve.Request(1, 0.001 * k) for k in range(6)]
    srv.run(reqs, clock=fake_clock(1e-3))
    assert [pids for _, pids in be.launched] == [[1]] * 6
    launch_times = [r.t_launch for r in reqs]
    assert launch_times == sorted(launch_times)
    for a, b in zip(reqs, reqs[1:]):
        assert b.t_launch >= a.t_done      # never two requests of one ID in flight


def test_deadline_drops_unlaunched_requests(monkeypatch):
    srv, be, _ = make_server(monkeypatch, 4, 1, None, (), 1, 50, seed=2)
    rng = np.random.default_rng(3)
    reqs = requests(rng, 4, 100, rate=2000.0)
    st = srv.run(reqs, max_batch=1, deadline=0.2, clock=fake_clock(1e-3))
    served = [r for r in reqs if r.t_done == r.t_done]
    assert st.requests == len(served) and st.dropped == len(reqs) - len(served) > 0
    assert len(be.launched) == len(served)
    assert all(r.t_launch <= 0.2 + 1e-9 for r in served)
    assert all(r.status == 0 and r.t_launch != r.t_launch for r in reqs if r.t_done != r.t_done)


def test_requests_with_wrong_vector_lengths_are_refused(monkeypatch):
    srv, be, qps = make_server(monkeypatch, 3, 2, None, (), None, 3, seed=4)
    good = serve.Request(0, 0.0, np.zeros(qps[0].n), np.zeros(qps[0].m), np.zeros(qps[0].m))
    bad = serve.Request(2, 0.001, np.zeros(qps[2].n + 1), None, None)
    with pytest.raises(ValueError, match="q has"):
        srv.run([good, bad], clock=fake_clock(1e-3))
    assert be.launched == []          # refused before anything ran


def test_large_requests_leave_slots_for_small_ones(monkeypatch):
    """With many large (cluster) requests pending, at most large_slots of
    them hold a slot at any time, so small requests keep being launched on
    the other slots instead of waiting behind them."""
    nprob, slots = 10, 4
    srv, be, _ = make_server(monkeypatch, nprob, slots, None, (0, 1, 2, 3, 4), None, 6, seed=9)
    srv.large_slots = 1
    seen = []
    orig = be.osqp_batch_launch

    def launch(h, slot, pids, qs, ls, us):
        orig(h, slot, pids, qs, ls, us)
        running_large = sum(1 for v in be.running.values() if be.lg[v[0][0]] and len(v[0]) == 1)
        seen.append(running_large)

    be.osqp_batch_launch = launch
    reqs = [serve.Request(p, 0.0) for p in range(5)] + [serve.Request(5 + k % 5, 0.0005 * k)
                                                        for k in range(20)]
    st = srv.run(reqs, clock=fake_clock(1e-3))
    assert st.requests == len(reqs)
    assert max(seen) <= 1
    # small requests were launched while large ones were still waiting
    first_small = min(i for i, (_, pids) in enumerate(be.launched) if not be.lg[pids[0]])
    last_large = max(i for i, (_, pids) in enumerate(be.launched) if be.lg[pids[0]])
    assert first_small < last_large

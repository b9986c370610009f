"""Continuous-batching serving: requests overlap on the device, each result
equals the result of the same request served alone, results pass the
acceptance test against the perturbed problems, and the in-flight device
footprint stays within the admission budget."""
import numpy as np
import pytest

from paper_1711_08013_gb300 import _binding as B
from paper_1711_08013_gb300 import problems as pb
from tests.kkt_check import acceptance, objective, objective_interval

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_08013_gb300.serve import Request, Server, poisson_requests  # noqa: E402


def pool():
    qps = [pb.random_qp(int(n), seed=4100 + k) for k, n in enumerate((10, 16, 24, 40, 60, 90))]
    qps += [pb.huber(int(n), seed=4200 + k) for k, n in enumerate((3, 4, 6, 8, 10, 12))]
    return qps


def clone(reqs):
    return [Request(r.pid, r.t_arrival, r.q, r.l, r.u) for r in reqs]


def test_serving_overlap_matches_alone_and_oracle(oracle_mod):
    qps = pool()
    reqs = poisson_requests(qps, rate=2000.0, duration=0.05, seed=11)
    assert len(reqs) > 40
    # the rule's row partition in both servers (autotune = 0): the same
    # arithmetic for a problem whatever else is in flight
    with Server(qps, slots=4, autotune=0) as srv:
        mix = clone(reqs)
        st = srv.run(mix, keep_x=True)
    with Server(qps, slots=1, autotune=0) as srv1:
        alone = clone(reqs)
        st1 = srv1.run(alone, max_batch=1, keep_x=True)
    assert st.launches < st1.launches  # requests were batched / overlapped
    assert all(r.status == B.SOLVED for r in mix) and all(r.status == B.SOLVED for r in alone), \
        sorted({(r.pid, r.status) for r in mix + alone if r.status != B.SOLVED})
    for a, b in zip(sorted(mix, key=lambda r: r.t_arrival), sorted(alone, key=lambda r: r.t_arrival)):
        assert a.pid == b.pid
        # long rows too are summed in a fixed order: bit-identical results
        assert np.array_equal(a.x, b.x)
    # the last request of each problem ID: its (x, y) are still resident
    last = {}
    for r in sorted(mix, key=lambda r: r.t_arrival):
        last[r.pid] = r
    with Server(qps, slots=4) as srv:
        srv.run(clone(reqs))
        for pid, r in last.items():
            x, y, z, info = B.osqp_batch_get(srv.h, pid, qps[pid].n, qps[pid].m)
            qp2 = pb._finish("req", qps[pid].P, r.q, qps[pid].A, r.l, r.u)
            prim, dual, ep, ed = acceptance(qp2, x, y, 1e-3, 1e-3)
            assert prim <= 1.01 * ep and dual <= 1.01 * ed, (pid, prim, ep, dual, ed)
            o = oracle_mod.solve(qp2)
            assert o.status == oracle_mod.SOLVED
            # the served objective against the oracle's optimum of the same
            # perturbed QP: inside the convexity interval
            star = oracle_mod.solve(qp2, eps_abs=1e-9, eps_rel=1e-9, max_iter=800000)
            lo, hi = objective_interval(qp2, x, z, y, star.x, star.y)
            d = objective(qp2, x) - star.obj_val
            slack = 1e-9 * max(1.0, abs(star.obj_val))
            assert lo - slack <= d <= hi + slack, (pid, lo, d, hi)


def test_deadline_drops_unlaunched_requests():
    qps = pool()
    reqs = poisson_requests(qps, rate=50000.0, duration=0.05, seed=13)
    with Server(qps, slots=2) as srv:
        st = srv.run(clone(reqs), deadline=0.0)
    assert st.requests + st.dropped == len(reqs)


def test_footprint_budget_limits_inflight_work():
    qps = pool()
    reqs = poisson_requests(qps, rate=5000.0, duration=0.02, seed=12)
    with Server(qps, slots=4, prime=True) as srv:
        budget = max(srv.footprint) + min(srv.footprint)
        srv.budget = budget
        st = srv.run(clone(reqs))
    assert st.max_inflight_bytes <= budget
    assert st.requests == len(reqs)


def test_large_requests_on_clusters():
    """A large problem in the pool is solved by a cluster of CTAs on its own
    slot while small requests keep flowing; its results pass the acceptance
    test on the perturbed data, and it starts from its previous solution."""
    qps = pool() + [pb.random_qp(300, seed=4300)]
    big = len(qps) - 1
    rng = np.random.default_rng(22)
    reqs = poisson_requests(qps[:big], rate=1000.0, duration=0.05, seed=21)
    for t in (0.0, 0.02):
        q, l, u = pb.perturb_vectors(rng, qps[big], 0.05)
        reqs.append(Request(big, t, q, l, u))
    with Server(qps, slots=4) as srv:
        assert srv.large[big] and not any(srv.large[:big])
        st = srv.run(reqs, keep_x=True)
        assert st.requests == len(reqs)
        x, y, z, info = B.osqp_batch_get(srv.h, big, qps[big].n, qps[big].m)
        assert info.launch == 3
    for r in reqs:
        assert r.status == B.SOLVED, (r.pid, r.status)
    last = [r for r in reqs if r.pid == big][-1]
    qp2 = pb._finish("req", qps[big].P, last.q, qps[big].A, last.l, last.u)
    prim, dual, ep, ed = acceptance(qp2, last.x, y, 1e-3, 1e-3)
    assert prim <= 1.01 * ep and dual <= 1.01 * ed


def test_served_results_match_oracle_at_tight_eps(oracle_mod):
    """Served at ε = 1e-6 with overlapping slots: every request's objective
    is within 1e-4 (relative) of the oracle's solution of the same perturbed
    QP at the same ε, and passes the acceptance test at 1e-6."""
    qps = pool()
    reqs = poisson_requests(qps, rate=2000.0, duration=0.02, seed=17)
    assert len(reqs) >= 20
    with Server(qps, slots=4, eps_abs=1e-6, eps_rel=1e-6, max_iter=100000) as srv:
        mix = clone(reqs)
        srv.run(mix, keep_x=True)
    for r in mix:
        assert r.status == B.SOLVED, (r.pid, r.status)
        qp2 = pb._finish("req", qps[r.pid].P, r.q, qps[r.pid].A, r.l, r.u)
        o = oracle_mod.solve(qp2, eps_abs=1e-6, eps_rel=1e-6, max_iter=200000)
        assert o.status == oracle_mod.SOLVED
        f = objective(qp2, r.x)
        assert abs(f - o.obj_val) <= 1e-4 * max(1.0, abs(o.obj_val)), (r.pid, f, o.obj_val)

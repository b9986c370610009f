"""Batched solves through the C ABI: every problem of a ragged batch against
the oracle, and each result identical alone and among other problems."""
import numpy as np
import pytest

from paper_1711_08013_gb300 import _binding as B
from paper_1711_08013_gb300 import problems as pb
from tests.kkt_check import acceptance, objective, objective_interval

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_08013_gb300.solver import BatchSolver  # noqa: E402

HIGH_ORACLE = dict(eps_abs=1e-9, eps_rel=1e-9, max_iter=400000, check_interval=10)


def mixed_batch():
    qps = pb.mpc_batch(12, seed=3100, nx_range=(4, 12), T_range=(5, 12))
    qps += [pb.random_qp(30, 150, seed=3201), pb.portfolio(3, seed=3202), pb.lasso(5, seed=3203),
            pb.huber(4, seed=3204), pb.box_qp(25, seed=3205)]
    return qps


@pytest.mark.parametrize("precision", [B.FP64, B.FP32_MIXED], ids=["fp64", "fp32"])
def test_batch_against_oracle(oracle_mod, precision):
    qps = mixed_batch()
    with BatchSolver(qps, precision=precision) as bs:
        bs.solve()
        res = [bs.result(i) for i in range(len(qps))]
    for qp, g in zip(qps, res):
        star = oracle_mod.solve(qp, **HIGH_ORACLE)
        assert g.status == B.SOLVED, (qp.name, g.status, g.iter)
        prim, dual, ep, ed = acceptance(qp, g.x, g.y, 1e-3, 1e-3)
        assert prim <= ep * 1.01 and dual <= ed * 1.01, (qp.name, prim, ep, dual, ed)
        lo, hi = objective_interval(qp, g.x, g.z, g.y, star.x, star.y)
        d = objective(qp, g.x) - star.obj_val
        assert abs(g.obj_val - objective(qp, g.x)) <= 1e-6 * max(1.0, abs(g.obj_val))
        slack = 1e-7 * max(1.0, abs(star.obj_val))
        assert lo - slack <= d <= hi + slack, (qp.name, lo, d, hi)


@pytest.mark.parametrize("precision", [B.FP64, B.FP32_MIXED], ids=["fp64", "fp32"])
def test_batch_result_same_alone_and_in_mix(precision):
    """With the rule's row partition (autotune = 0) a problem's arithmetic,
    long rows included (chunk partials summed in chunk order), does not
    depend on the other problems of the batch: bit-identical results alone
    and in the mix.  (With the autotuner the partition of a shape class is a
    measured choice, which two batches may make differently.)"""
    qps = mixed_batch()
    with BatchSolver(qps, precision=precision, autotune=0) as bs:
        bs.solve()
        mix = [bs.result(i) for i in range(len(qps))]
    for i in (0, 5, len(qps) - 4, len(qps) - 1):
        with BatchSolver([qps[i]], precision=precision, autotune=0) as one:
            one.solve()
            alone = one.result(0)
        assert alone.status == mix[i].status
        assert alone.iter == mix[i].iter
        assert np.array_equal(alone.x, mix[i].x), qps[i].name
        assert np.array_equal(alone.y, mix[i].y), qps[i].name


GROUPS = [1, 2, 4, 8, 16, 32]


@pytest.mark.parametrize("precision", [B.FP64, B.FP32_MIXED], ids=["fp64", "fp32"])
def test_autotuner_uses_the_fastest_measured_partition(oracle_mod, precision):
    """The batch autotuner times every candidate group width on one matrix
    of each shape class and gives each class its fastest; the representative
    problems carry the chosen widths, and the tuned batch's results pass the
    acceptance test and lie in the convexity interval around the oracle's
    optimum, like the rule's."""
    qps = pb.mpc_batch(48, seed=3300) + mixed_batch()[12:]
    with BatchSolver(qps, precision=precision) as bs:
        table = B.osqp_batch_tuning(bs.handle)
        assert len(table) >= 2
        for kind, rb, mb, xb, rep, chosen, cyc in table:
            assert np.all(cyc > 0)
            assert chosen == GROUPS[int(np.argmin(cyc))], (kind, rb, mb, xb, cyc)
            assert B.osqp_batch_schedule(bs.handle, rep)[kind] == chosen
        bs.solve()
        res = [bs.result(i) for i in range(len(qps))]
    with BatchSolver(qps, precision=precision, autotune=0) as rule:
        assert B.osqp_batch_tuning(rule.handle) == []
    for qp, g in zip(qps, res):
        star = oracle_mod.solve(qp, **HIGH_ORACLE)
        assert g.status == B.SOLVED, (qp.name, g.status)
        prim, dual, ep, ed = acceptance(qp, g.x, g.y, 1e-3, 1e-3)
        assert prim <= ep * 1.01 and dual <= ed * 1.01, (qp.name, prim, ep, dual, ed)
        lo, hi = objective_interval(qp, g.x, g.z, g.y, star.x, star.y)
        d = objective(qp, g.x) - star.obj_val
        slack = 1e-7 * max(1.0, abs(star.obj_val))
        assert lo - slack <= d <= hi + slack, (qp.name, lo, d, hi)


def test_batch_matches_single_problem_solver(oracle_mod):
    """The batch kernel and the single-problem one-CTA solver run the same
    stages; with exact linear solves their iterates agree to rounding."""
    qps = mixed_batch()[:6]
    step = dict(adaptive_rho=0, eps_abs=0.0, eps_rel=0.0, eps_pinf=1e-300, eps_dinf=1e-300,
                pcg_tol_fraction=0.0, pcg_tol_floor=1e-14, pcg_max_iter=2000, check_interval=1,
                max_iter=30)
    with BatchSolver(qps, **step) as bs:
        bs.solve()
        for i, qp in enumerate(qps):
            g = bs.result(i)
            o = oracle_mod.solve(qp, adaptive_rho=0, eps_abs=0.0, eps_rel=0.0, eps_pinf=1e-300,
                                 eps_dinf=1e-300, check_interval=1, max_iter=30)
            scale = max(1.0, np.max(np.abs(o.x)))
            assert np.max(np.abs(g.x - o.x)) <= 1e-8 * scale, qp.name


def test_batch_update_vectors_subset_and_warm_start(oracle_mod):
    qps = mixed_batch()
    rng = np.random.default_rng(7)
    with BatchSolver(qps) as bs:
        bs.solve()
        first = [bs.result(i) for i in range(len(qps))]
        pick = [1, 4, len(qps) - 5]
        new = {}
        for i in pick:
            q2, l2, u2 = pb.perturb_vectors(rng, qps[i])
            new[i] = pb._finish("upd", qps[i].P, q2, qps[i].A, l2, u2)
            bs.update_vectors(i, q2, l2, u2)
        bs.solve(subset=pick)
        for i in pick:
            g = bs.result(i)
            qp2 = new[i]
            assert g.status == B.SOLVED
            prim, dual, ep, ed = acceptance(qp2, g.x, g.y, 1e-3, 1e-3)
            assert prim <= ep * 1.01 and dual <= ed * 1.01
        # problems outside the subset were not touched
        other = 0
        g = bs.result(other)
        assert np.array_equal(g.x, first[other].x)
        # a warm re-solve of an unchanged problem terminates at the first check
        bs.solve(subset=[other])
        assert bs.result(other).iter <= 25


def test_batch_reset_reproduces_cold_solve():
    qps = mixed_batch()[:5]
    with BatchSolver(qps) as bs:
        bs.solve()
        a = [bs.result(i) for i in range(len(qps))]
        bs.reset()
        bs.solve()
        b = [bs.result(i) for i in range(len(qps))]
    for ra, rb in zip(a, b):
        assert ra.iter == rb.iter and np.array_equal(ra.x, rb.x)


def test_batch_larger_mpc_mix():
    """A few hundred ragged MPC problems (the batched workload's generator)."""
    qps = pb.mpc_batch(300, seed=3300)
    with BatchSolver(qps, precision=B.FP32_MIXED) as bs:
        bs.solve()
        res = [bs.result(i) for i in range(len(qps))]
    bad = [i for i, r in enumerate(res) if r.status != B.SOLVED]
    assert not bad, bad[:10]
    for i in range(0, len(qps), 37):
        prim, dual, ep, ed = acceptance(qps[i], res[i].x, res[i].y, 1e-3, 1e-3)
        assert prim <= ep * 1.01 and dual <= ed * 1.01


def test_heavy_problems_on_clusters():
    """More problems than CTAs and one problem far slower than the fair share:
    once its time is known (second launch) it is solved by a cluster beside
    the one-CTA kernel; every result still passes the acceptance test, and
    the problems that stay on one CTA reproduce bit for bit."""
    qps = pb.mpc_batch(300, seed=3150, nx_range=(4, 8), T_range=(5, 8))
    qps.append(pb.mpc(32, 30, seed=5))
    heavy = len(qps) - 1
    with BatchSolver(qps) as bs:
        bs.solve()
        first = [bs.result(i) for i in range(len(qps))]
        B.osqp_batch_reset(bs.handle)
        bs.solve()
        second = [bs.result(i) for i in range(len(qps))]
    assert first[heavy].launch == 1 and second[heavy].launch == 3
    assert sum(r.launch == 3 for r in second) <= 32
    for i, r in enumerate(second):
        assert r.status == B.SOLVED, i
        prim, dual, ep, ed = acceptance(qps[i], r.x, r.y, 1e-3, 1e-3)
        assert prim <= 1.01 * ep and dual <= 1.01 * ed, i
        if r.launch == 1 and first[i].launch == 1:
            assert np.array_equal(r.x, first[i].x), i



def test_whole_batch_update_and_read_back_match_per_problem_calls():
    """osqp_batch_update_all / osqp_batch_get_all (one transfer per vector
    for the whole batch) give the same solves and solutions as the
    per-problem update and read-back calls, bit for bit."""
    qps = mixed_batch()
    rng = np.random.default_rng(17)
    new = [pb.perturb_vectors(rng, q) for q in qps]
    out = []
    for whole in (True, False):
        with BatchSolver(qps, autotune=0) as bs:
            bs.solve()
            if whole:
                B.osqp_batch_update_all(bs.handle, np.concatenate([v[0] for v in new]),
                                        np.concatenate([v[1] for v in new]),
                                        np.concatenate([v[2] for v in new]))
            else:
                for i, v in enumerate(new):
                    bs.update_vectors(i, *v)
            bs.solve()
            x = np.empty(sum(q.n for q in qps))
            y = np.empty(sum(q.m for q in qps))
            B.osqp_batch_get_all(bs.handle, x, y)
            per = [bs.result(i) for i in range(len(qps))]
            assert np.array_equal(x, np.concatenate([r.x for r in per]))
            assert np.array_equal(y, np.concatenate([r.y for r in per]))
            out.append(x)
    assert np.array_equal(out[0], out[1])
    with BatchSolver(qps[:2], autotune=0) as bs:
        bad_l = np.concatenate([new[0][1], new[1][1]])
        bad_u = bad_l - 1.0
        with pytest.raises(B.OsqpError):
            B.osqp_batch_update_all(bs.handle, None, bad_l, bad_u)

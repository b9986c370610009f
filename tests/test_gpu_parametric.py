"""Parametric sequences of §8.4 on the GPU: the data stay resident and are
updated in place between solves (vectors for the Lasso path and the MPC
loop, matrix values for the portfolio risk model).  Each step's result
passes the §8 acceptance test on the QP it solved, the oracle reaches the
same status on that QP, the MPC plant follows the applied inputs, and warm
starts cut the iteration count (§6)."""
import numpy as np
import pytest

from paper_1711_08013_gb300 import _binding as B
from paper_1711_08013_gb300 import parametric as pm
from paper_1711_08013_gb300 import problems as pb
from tests.kkt_check import acceptance, fp32_data_allowance, objective, objective_interval

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)


def replay(qp, trace):
    qs = []
    cur = qp
    for upd in trace:
        cur = pm.apply_update(cur, upd)
        qs.append(cur)
    return qs


def check(oracle_mod, qs, steps, eps=1e-3, precision=B.FP64):
    """Each step's result against the oracle on the QP that step solved: the
    acceptance test at ε, the oracle solving it too, and the GPU objective
    inside the convexity interval around the oracle's optimum (ε = 1e-9);
    at a tight ε (≤ 1e-6) also within 1e-4 (relative) of the oracle's
    objective at the same ε.  FP32-mixed mode keeps the matrices in FP32 and
    meets ε on that rounding of the problem: its acceptance test on the
    problem as given allows the bound on the rounding's effect
    (fp32_data_allowance), which only matters at a tight ε."""
    for k, (q, st) in enumerate(zip(qs, steps)):
        assert st.status == B.SOLVED, (k, st.status)
        prim, dual, ep, ed = acceptance(q, st.x, st.y, eps, eps)
        ap, ad = fp32_data_allowance(q, st.x, st.y) if precision == B.FP32_MIXED else (0.0, 0.0)
        assert prim <= 1.01 * ep + ap and dual <= 1.01 * ed + ad, (k, prim, ep, ap, dual, ed, ad)
        o = oracle_mod.solve(q, eps_abs=eps, eps_rel=eps, max_iter=200000)
        assert o.status == oracle_mod.SOLVED
        star = oracle_mod.solve(q, eps_abs=1e-9, eps_rel=1e-9, max_iter=800000)
        lo, hi = objective_interval(q, st.x, st.z, st.y, star.x, star.y)
        d = objective(q, st.x) - star.obj_val
        slack = 1e-9 * max(1.0, abs(star.obj_val))
        assert lo - slack <= d <= hi + slack, (k, lo, d, hi)
        if eps <= 1e-6:
            assert abs(objective(q, st.x) - o.obj_val) <= 1e-4 * max(1.0, abs(o.obj_val)), k


@pytest.mark.parametrize("precision", [B.FP64, B.FP32_MIXED], ids=["fp64", "fp32"])
@pytest.mark.parametrize("launch", [1, 2], ids=["block", "grid"])
def test_lasso_path(oracle_mod, precision, launch):
    qp = pb.lasso(10, seed=1)
    trace = []
    with pm.GpuSession(qp, precision=precision, launch=launch) as s:
        ws = pm.run(s, pm.lasso_path(qp, 8), trace=trace)
    check(oracle_mod, replay(qp, trace), ws, precision=precision)
    with pm.GpuSession(qp, precision=precision, launch=launch) as s:
        cold = pm.run(s, pm.lasso_path(qp, 8), warm=False)
    check(oracle_mod, replay(qp, trace), cold, precision=precision)
    assert sum(st.iter for st in ws) < sum(st.iter for st in cold)


def test_mpc_closed_loop(oracle_mod):
    qp = pb.mpc_paper(8, T=10, seed=2)
    nx, nu, T = qp.meta["nx"], qp.meta["nu"], qp.meta["T"]
    trace = []
    with pm.GpuSession(qp) as s:
        steps = pm.run(s, pm.mpc_closed_loop(qp, 10), trace=trace)
    qs = replay(qp, trace)
    check(oracle_mod, qs, steps)
    u0 = [st.x[nx * (T + 1): nx * (T + 1) + nu] for st in steps]
    xs = pm.mpc_states(qp, u0[:-1])
    for k, (q, st) in enumerate(zip(qs, steps)):
        assert np.array_equal(q.l[:nx], -xs[k])
        assert np.max(np.abs(st.x[:nx] - xs[k])) <= 1e-2, k


def test_portfolio_backtest(oracle_mod):
    qp = pb.portfolio(3, seed=5)
    n = qp.meta["F"].shape[0]
    trace = []
    with pm.GpuSession(qp) as s:
        steps = pm.run(s, pm.portfolio_backtest(qp, days=6, days_per_month=2, seed=3), trace=trace)
    assert sum("A_val" in t for t in trace) == 2
    qs = replay(qp, trace)
    check(oracle_mod, qs, steps)
    for st in steps:
        assert abs(st.x[:n].sum() - 1.0) <= 1e-2 and st.x[:n].min() >= -1e-2


@pytest.mark.parametrize("precision", [B.FP64, B.FP32_MIXED], ids=["fp64", "fp32"])
def test_lasso_path_tight_eps(oracle_mod, precision):
    """The warm-started λ-path at ε = 1e-6: every step's objective within
    1e-4 of the oracle's on the same QP."""
    qp = pb.lasso(10, seed=3)
    trace = []
    with pm.GpuSession(qp, precision=precision, eps_abs=1e-6, eps_rel=1e-6, max_iter=100000) as s:
        ws = pm.run(s, pm.lasso_path(qp, 6), trace=trace)
    check(oracle_mod, replay(qp, trace), ws, eps=1e-6, precision=precision)


def test_mpc_closed_loop_tight_eps(oracle_mod):
    qp = pb.mpc_paper(8, T=10, seed=4)
    trace = []
    with pm.GpuSession(qp, eps_abs=1e-6, eps_rel=1e-6, max_iter=100000) as s:
        steps = pm.run(s, pm.mpc_closed_loop(qp, 6), trace=trace)
    check(oracle_mod, replay(qp, trace), steps, eps=1e-6)

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
from tests.kkt_check import acceptance

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


def check(oracle_mod, qs, steps, eps=1e-3):
    for k, (q, st) in enumerate(zip(qs, steps)):
        assert st.status == B.SOLVED, (k, st.status)
        prim, dual, ep, ed = acceptance(q, st.x, st.y, eps, eps)
        assert prim <= 1.01 * ep and dual <= 1.01 * ed, (k, prim, ep, dual, ed)
        assert oracle_mod.solve(q).status == oracle_mod.SOLVED


@pytest.mark.parametrize("precision", [B.FP64, B.FP32_MIXED], ids=["fp64", "fp32"])
@pytest.mark.parametrize("launch", [1, 2], ids=["block", "grid"])
def test_lasso_path(oracle_mod, precision, launch):
    qp = pb.lasso(10, seed=1)
    trace = []
    with pm.GpuSession(qp, precision=precision, launch=launch) as s:
        ws = pm.run(s, pm.lasso_path(qp, 8), trace=trace)
    check(oracle_mod, replay(qp, trace), ws)
    with pm.GpuSession(qp, precision=precision, launch=launch) as s:
        cold = pm.run(s, pm.lasso_path(qp, 8), warm=False)
    check(oracle_mod, replay(qp, trace), cold)
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

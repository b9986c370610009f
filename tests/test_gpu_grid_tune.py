"""Row-partition autotuning of a single problem on the whole-GPU grid team:
every candidate group width of both matrices is timed at setup, the choice
follows the timings, and the tuned solve passes the same checks against the
oracle as the row-length rule's."""
import numpy as np
import pytest

from paper_1711_08013_gb300 import _binding as B
from paper_1711_08013_gb300 import problems as pb
from tests.kkt_check import acceptance, objective, objective_interval

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_08013_gb300.solver import Solver  # noqa: E402

GROUPS = [1, 2, 4, 8, 16, 32]
HIGH_ORACLE = dict(eps_abs=1e-9, eps_rel=1e-9, max_iter=400000, check_interval=10)
CASES = [
    ("lasso_long", lambda: pb.lasso(2, seed=7, m=1500)),  # columns beyond the chunk length
    ("portfolio", lambda: pb.portfolio(3, seed=5)),       # a 300-entry budget row
    ("random_qp", lambda: pb.random_qp(30, 120, seed=3)),
]


def _chosen_ok(ms, chosen, rule):
    """The width used is the fastest, or the rule's when that is within 3 %."""
    best = GROUPS[int(np.argmin(ms))]
    if chosen == best:
        return True
    return chosen == rule and ms[GROUPS.index(rule)] <= 1.03 * ms.min() * (1 + 1e-6)


@pytest.mark.parametrize("precision", [B.FP64, B.FP32_MIXED], ids=["fp64", "fp32"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_grid_autotuner(oracle_mod, name, make, precision):
    qp = make()
    with Solver(qp, launch=2, precision=precision, autotune=0) as rule:
        gk0, ga0, tuned0, ms_kn0, ms_a0 = B.osqp_diag_schedule(rule.handle)
        assert tuned0 == 0 and not ms_kn0.any() and not ms_a0.any()
    with Solver(qp, launch=2, precision=precision) as s:
        gk, ga, tuned, ms_kn, ms_a = B.osqp_diag_schedule(s.handle)
        assert tuned == 1
        assert np.all(ms_kn > 0) and np.all(ms_a > 0)
        assert _chosen_ok(ms_kn, gk, gk0), (gk, gk0, ms_kn)
        assert _chosen_ok(ms_a, ga, ga0), (ga, ga0, ms_a)
        g = s.solve()
    star = oracle_mod.solve(qp, **HIGH_ORACLE)
    assert g.status == B.SOLVED, (name, g.status)
    prim, dual, ep, ed = acceptance(qp, g.x, g.y, 1e-3, 1e-3)
    assert prim <= ep * 1.01 and dual <= ed * 1.01, (name, prim, ep, dual, ed)
    lo, hi = objective_interval(qp, g.x, g.z, g.y, star.x, star.y)
    d = objective(qp, g.x) - star.obj_val
    slack = 1e-7 * max(1.0, abs(star.obj_val))
    assert lo - slack <= d <= hi + slack, (name, lo, d, hi)


def test_other_teams_keep_the_rule():
    """The one-CTA and cluster teams use the row-length rule with autotuning
    on (their products are too short for a launch-level timing)."""
    qp = pb.random_qp(30, 120, seed=3)
    for launch in (1, 3):
        with Solver(qp, launch=launch) as s:
            assert B.osqp_diag_schedule(s.handle)[2] == 0, launch

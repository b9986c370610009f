"""Solution polishing (§4) on the GPU against the oracle: an accepted polish
reaches the high-accuracy solution (acceptance test at ε = 1e-8, objective
of a 1e-10 oracle run), in both precision modes (polishing runs in FP64 on
the raw data) and all team shapes; a rejected polish leaves the ADMM
solution bit for bit; the batch kernel polishes too."""
import numpy as np
import pytest

from paper_1711_08013_gb300 import _binding as B
from paper_1711_08013_gb300 import problems as pb
from tests.kkt_check import acceptance, objective

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_08013_gb300.solver import BatchSolver, Solver  # noqa: E402

HIGH = dict(eps_abs=1e-10, eps_rel=1e-10, max_iter=400000, check_interval=10)
CASES = [
    ("random", lambda: pb.random_qp(40, seed=3)),
    ("mpc", lambda: pb.mpc(6, 8, seed=4)),
    ("lasso", lambda: pb.lasso(20, seed=1)),
    ("box", lambda: pb.box_qp(30, seed=1)),
    ("eq", lambda: pb.eq_qp(30, seed=30_001, density=0.5)),
]


_BLOCK64 = {}


@pytest.mark.parametrize("precision", [B.FP64, B.FP32_MIXED], ids=["fp64", "fp32"])
@pytest.mark.parametrize("launch", [1, 2, 3], ids=["block", "grid", "cluster"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_polish_reaches_high_accuracy(oracle_mod, name, make, launch, precision):
    """Every case polishes on the one-CTA FP64 solver, and every other team
    shape and precision polishes it too (its ADMM point differs at the
    rounding level, not in the active set that the signs of y give)."""
    qp = make()
    hi = oracle_mod.solve(qp, **HIGH)
    if name not in _BLOCK64:
        with Solver(qp, launch=1, precision=B.FP64, polish=1) as s:
            _BLOCK64[name] = s.solve().polished
    with Solver(qp, launch=launch, precision=precision, polish=1) as s:
        g = s.solve()
    assert g.status == B.SOLVED
    assert _BLOCK64[name] == 1, name
    assert g.polished == 1, (name, g.polished)
    if g.polished == 1:
        prim, dual, ep, ed = acceptance(qp, g.x, g.y, 1e-8, 1e-8)
        assert prim <= ep and dual <= ed, (name, prim, ep, dual, ed)
        f, f_hi = objective(qp, g.x), objective(qp, hi.x)
        assert abs(f - f_hi) <= 1e-7 * max(1.0, abs(f_hi)), (name, f, f_hi)
        assert abs(g.obj_val - f) <= 1e-9 * max(1.0, abs(f))


def test_rejected_polish_keeps_admm_solution(oracle_mod):
    qp = pb.svm(10, seed=1)
    with Solver(qp, launch=1, polish=1) as s:
        g = s.solve()
    with Solver(qp, launch=1) as s:
        plain = s.solve()
    assert g.polished == -1 and plain.polished == 0
    assert np.array_equal(g.x, plain.x) and np.array_equal(g.y, plain.y)


def test_batch_polish(oracle_mod):
    """The batch kernel polishes each problem as the one-CTA solver does (same
    stages on the same team shape): same polish outcome, same solution."""
    qps = [pb.random_qp(int(n), int(2 * n), seed=600 + k) for k, n in enumerate((8, 15, 30, 45))]
    qps += [pb.box_qp(20, seed=700), pb.mpc(6, 8, seed=4)]
    with BatchSolver(qps, polish=1, autotune=0) as bs:  # the one-CTA solver's partition
        bs.solve()
        res = [bs.result(i) for i in range(len(qps))]
    for qp, r in zip(qps, res):
        with Solver(qp, launch=1, polish=1) as s:
            one = s.solve()
        with Solver(qp, launch=1) as s:
            plain = s.solve()
        assert r.status == B.SOLVED and r.polished == one.polished
        assert np.max(np.abs(r.x - one.x)) <= 1e-12 * max(1.0, np.max(np.abs(one.x)))
        if r.polished == 1:  # accepted only when no worse than the ADMM point
            prim, dual, _, _ = acceptance(qp, r.x, r.y, 0.0, 0.0)
            prim0, dual0, _, _ = acceptance(qp, plain.x, plain.y, 0.0, 0.0)
            assert prim <= 1.01 * prim0 + 1e-12 and dual <= 1.01 * dual0 + 1e-12
    assert sum(r.polished == 1 for r in res) >= 3

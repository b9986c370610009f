"""The FP32 data-rounding allowance of the acceptance test (no GPU): rounding
every entry of a diagonally scaled P and A to FP32 and scaling back moves the
residuals of any point by no more than fp32_data_allowance says, and the
bound is not vacuous (it is within a small factor of the worst movement
that independent roundings produce)."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1711_08013_gb300 import problems as pb
from tests.kkt_check import U32, acceptance, fp32_data_allowance, full_P


def rounded(M, r, c):
    """diag(1/r)·fl32(diag(r)·M·diag(c))·diag(1/c): FP32 storage of a scaled matrix."""
    S = sp.diags(r) @ M @ sp.diags(c)
    S = sp.csc_matrix(S)
    S.data = S.data.astype(np.float32).astype(np.float64)
    return sp.csc_matrix(sp.diags(1.0 / r) @ S @ sp.diags(1.0 / c))


@pytest.mark.parametrize("seed", range(4))
def test_allowance_bounds_rounded_residuals(seed):
    rng = np.random.default_rng(seed)
    qp = pb.random_qp(40, 200, seed=seed)
    P, A = full_P(qp), qp.A
    D = np.exp(rng.uniform(-3, 3, qp.n))
    E = np.exp(rng.uniform(-3, 3, qp.m))
    c = float(np.exp(rng.uniform(-2, 2)))
    Pr = rounded(c * P, D, D) / c
    Ar = rounded(A, E, D)
    assert U32 == 2.0 ** -24
    for _ in range(5):
        x = rng.standard_normal(qp.n) * 10.0 ** rng.uniform(-2, 2)
        y = rng.standard_normal(qp.m) * 10.0 ** rng.uniform(-2, 2)
        ap, ad = fp32_data_allowance(qp, x, y)
        dp = np.max(np.abs((Ar - A) @ x))
        dd = np.max(np.abs((Pr - P) @ x + (Ar - A).T @ y))
        assert dp <= ap * (1 + 1e-9) and dd <= ad * (1 + 1e-9)
        # the acceptance residuals of the true and the rounded problem differ
        # by no more than the allowance
        rq = pb.QP(qp.name, sp.triu(Pr, format="csc"), qp.q, Ar, qp.l, qp.u, qp.meta)
        p0, d0, _, _ = acceptance(qp, x, y, 0.0, 0.0)
        p1, d1, _, _ = acceptance(rq, x, y, 0.0, 0.0)
        assert abs(p0 - p1) <= ap * (1 + 1e-9) and abs(d0 - d1) <= ad * (1 + 1e-9)
        # not vacuous: the bound is a worst case over signs, the actual
        # movement of random roundings is a sizeable fraction of it
        assert dd >= 1e-3 * ad

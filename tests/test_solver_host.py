"""Host-side argument checks of the Python solver objects (no GPU): arrays
whose length differs from what the C ABI will read behind the pointer are
refused before the library is called."""
import numpy as np
import pytest

from paper_1711_08013_gb300 import solver as S


def _solver(monkeypatch, calls):
    for name in ("osqp_update_vectors", "osqp_update_matrices", "osqp_warm_start",
                 "osqp_batch_update_vectors"):
        monkeypatch.setattr(S.B, name, lambda *a, _n=name: calls.append((_n, a)))
    s = object.__new__(S.Solver)
    s.n, s.m, s.nnz_p, s.nnz_a, s.handle = 3, 2, 4, 5, None
    b = object.__new__(S.BatchSolver)
    b.sizes, b.handle = [(3, 2), (6, 1)], None
    return s, b


def test_wrong_lengths_refused(monkeypatch):
    calls = []
    s, b = _solver(monkeypatch, calls)
    with pytest.raises(ValueError, match="q has 4 entries, expected 3"):
        s.update_vectors(q=np.zeros(4))
    with pytest.raises(ValueError, match="u has"):
        s.update_vectors(u=np.zeros(3))
    with pytest.raises(ValueError, match="A_val"):
        s.update_matrices(A_val=np.zeros(4))
    with pytest.raises(ValueError, match="y has"):
        s.warm_start(x=np.zeros(3), y=np.zeros(1))
    with pytest.raises(ValueError, match="l has"):
        b.update_vectors(1, l=np.zeros(2))
    assert calls == []


def test_right_lengths_and_none_pass_through(monkeypatch):
    calls = []
    s, b = _solver(monkeypatch, calls)
    s.update_vectors(q=np.zeros(3), l=np.zeros(2))
    s.update_matrices(P_val=np.zeros(4))
    s.warm_start(x=np.zeros(3))
    b.update_vectors(1, q=np.zeros(6), u=np.zeros(1))
    assert [c[0] for c in calls] == ["osqp_update_vectors", "osqp_update_matrices",
                                     "osqp_warm_start", "osqp_batch_update_vectors"]
    assert calls[0][1][3] is None and calls[2][1][2] is None

"""The algorithmic-bytes model behind every roofline figure of bench.py
(no GPU): linear in the iteration counts, and one PCG iteration streams the
matrices of Kn = [P̄ Āᵀ] and Ā once each, (nnz(P) + 2·nnz(A))·(s_v + 4)
bytes plus row pointers, with vector traffic of a few vectors per row."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_model", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("sv", [8, 4])
def test_pcg_iteration_streams_each_matrix_once(bench, sv):
    n, m, nnz_p, nnz_a = 1000, 3000, 5000, 20000
    nnz_kn = nnz_p + nnz_a
    f = lambda K, J, C: bench.admm_bytes(n, m, nnz_kn, nnz_a, sv, K, J, C)
    per_pcg = f(10, 41, 0) - f(10, 40, 0)
    matrix = (nnz_p + 2 * nnz_a) * (sv + 4) + 4 * (n + 1) + 4 * (m + 1)
    vectors = per_pcg - matrix
    assert 5 * (n + m) * sv <= vectors <= 20 * (n + m) * 8


def test_linear_in_iteration_counts(bench):
    args = (500, 800, 9000, 6000, 8)
    f = lambda K, J, C: bench.admm_bytes(*args, K, J, C)
    assert f(0, 0, 0) == 0
    assert f(20, 120, 2) == pytest.approx(2 * f(10, 60, 1))
    assert f(10, 60, 2) - f(10, 60, 1) == pytest.approx(f(10, 60, 1) - f(10, 60, 0))
    # a check streams both matrices at least once in FP64 work
    assert f(10, 60, 1) - f(10, 60, 0) > 9000 * 12 + 6000 * 12


def test_workload_text_states_its_parameters(bench):
    """The serving line names the offered rate and the size cap it ran with,
    in the bench's own line and in the reference arm's."""
    import argparse
    a = argparse.Namespace(nmax=500, rate=5.0)
    text = bench.workload_desc(a, "serve")
    assert "at 5 req/s" in text and "logU[10,500]" in text
    assert "RATE" not in text and "NMAX" not in text
    assert bench.workload_desc(a, "lasso") == bench.WORKLOADS["lasso"][1]

"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every function that include/*.h declares, and rejects invalid input
with the documented codes before any device work."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1711_08013_gb300 import _binding as B
from paper_1711_08013_gb300 import build as BLD
from paper_1711_08013_gb300 import problems as pb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    BLD.build()
    return B.lib()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names += re.findall(r"^\s*(?:int32_t|int64_t|void|const char\s*\*)\s+(osqp_\w+)\s*\(", text,
                            re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("osqp_setup", "osqp_solve", "osqp_update_vectors", "osqp_update_rho",
                     "osqp_cleanup", "osqp_warm_start", "osqp_get_solution"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_defaults(lib):
    s = B.osqp_set_default_settings()
    assert (s.rho, s.sigma, s.alpha) == (0.1, 1e-6, 1.6)
    assert (s.eps_abs, s.eps_rel, s.eps_pinf, s.eps_dinf) == (1e-3, 1e-3, 1e-4, 1e-4)
    assert s.adaptive_rho == 1 and s.check_interval == 25 and s.scaling_iters == 10
    assert s.precision == B.FP64


def _setup_rc(qp, **settings):
    try:
        h = B.osqp_setup(qp.P, qp.q, qp.A, qp.l, qp.u, B.osqp_set_default_settings(**settings))
    except B.OsqpError as e:
        return e.code
    B.osqp_cleanup(h)
    return 0


def test_rejects_lower_triangle_P(lib):
    qp = pb.unconstrained_qp(6, seed=1)  # dense P
    qp.P = sp.csc_matrix(qp.P_full().toarray())  # full, not upper
    qp.P.sort_indices()
    assert _setup_rc(qp) == B.OSQP_ERR_CSC


def test_rejects_l_greater_than_u(lib):
    qp = pb.random_qp(6, 10, seed=1)
    qp.l = qp.u + 1.0
    assert _setup_rc(qp) == B.OSQP_ERR_LGTU


def test_rejects_nonfinite(lib):
    qp = pb.random_qp(6, 10, seed=1)
    qp.q = qp.q.copy()
    qp.q[2] = np.nan
    assert _setup_rc(qp) == B.OSQP_ERR_NONFINITE


def test_rejects_bad_settings(lib):
    qp = pb.random_qp(6, 10, seed=1)
    assert _setup_rc(qp, alpha=2.0) == B.OSQP_ERR_SETTINGS
    assert _setup_rc(qp, rho=0.0) == B.OSQP_ERR_SETTINGS
    assert _setup_rc(qp, check_interval=0) == B.OSQP_ERR_SETTINGS
    assert _setup_rc(qp, precision=7) == B.OSQP_ERR_SETTINGS


def test_rejects_unsorted_rows(lib):
    qp = pb.random_qp(6, 10, seed=1)
    A = qp.A.copy()
    j = next(c for c in range(A.shape[1]) if A.indptr[c + 1] - A.indptr[c] >= 2)
    a, b = A.indptr[j], A.indptr[j + 1]
    A.indices[a:b] = A.indices[a:b][::-1].copy()
    A.has_sorted_indices = False
    qp.A = A
    assert _setup_rc(qp) == B.OSQP_ERR_CSC


def test_null_arguments(lib):
    assert lib.osqp_solve(None) == B.OSQP_ERR_ARG
    assert lib.osqp_cleanup(None) == B.OSQP_ERR_ARG
    assert lib.osqp_update_rho(None, C.c_double(1.0)) == B.OSQP_ERR_ARG


def _batch_rc(qps, **settings):
    try:
        h = B.osqp_batch_setup(qps, B.osqp_set_default_settings(**settings))
    except B.OsqpError as e:
        return e.code
    B.osqp_batch_cleanup(h)
    return 0


def test_batch_setup_validates_every_problem_on_the_host(lib):
    """osqp_batch_setup checks each problem as osqp_setup does, before any
    device work: the first invalid problem decides the error code."""
    good = pb.random_qp(5, 12, seed=1)
    lgtu = pb._finish("lgtu", good.P, good.q, good.A, good.u + 1.0, good.u)
    nan_q = pb._finish("nan", good.P, np.where(np.arange(good.n) == 1, np.nan, good.q), good.A,
                       good.l, good.u)
    full_p = pb.unconstrained_qp(6, seed=1)
    full_p.P = sp.csc_matrix(full_p.P_full().toarray())
    full_p.P.sort_indices()
    assert _batch_rc([good, lgtu]) == B.OSQP_ERR_LGTU
    assert _batch_rc([nan_q, good]) == B.OSQP_ERR_NONFINITE
    assert _batch_rc([good, full_p]) == B.OSQP_ERR_CSC
    assert _batch_rc([good], alpha=2.0) == B.OSQP_ERR_SETTINGS
    assert _batch_rc([]) == B.OSQP_ERR_ARG

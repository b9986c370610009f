"""Failure detection without a GPU fault: a grid barrier whose wait runs out
(one CTA never arrives) returns an error status that the host reads, and the
context stays usable for a normal solve afterwards."""
import pytest

from paper_1711_08013_gb300 import _binding as B
from paper_1711_08013_gb300 import problems as pb

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_08013_gb300.solver import Solver  # noqa: E402


def test_barrier_timeout_reported_and_context_usable():
    assert B.lib().osqp_diag_barrier_timeout(0.05) == B.OSQP_OK
    assert B.lib().osqp_diag_barrier_timeout(0.0) == B.OSQP_ERR_ARG
    qp = pb.random_qp(20, 60, seed=1)
    with Solver(qp, launch=2) as s:
        assert s.solve().status == B.SOLVED

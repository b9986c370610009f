"""The seeded synthetic inputs against the recipe of each benchmark workload
(App. A classes with the sizes and ranges of the workloads): dimensions,
sparsity, value ranges and structure, so that every measured number refers
to the stated workload.  No generator stores zero entries: every stored
entry is a nonzero the kernels and the oracle must process."""
import numpy as np
import pytest

from paper_1711_08013_gb300 import problems as pb


def _no_stored_zeros(qp):
    return not np.any(qp.A.data == 0) and not np.any(qp.P.data == 0)


@pytest.mark.parametrize("make", [
    lambda: pb.random_qp(20, seed=1), lambda: pb.eq_qp(20, seed=1), lambda: pb.mpc(7, 9, seed=1),
    lambda: pb.mpc_paper(6, seed=1), lambda: pb.portfolio(2, seed=1), lambda: pb.lasso(5, seed=1),
    lambda: pb.huber(4, seed=1), lambda: pb.svm(4, seed=1), lambda: pb.box_qp(6, seed=1),
])
def test_no_stored_zeros_and_valid_bounds(make):
    qp = make()
    assert _no_stored_zeros(qp)
    assert np.all(qp.l <= qp.u)
    assert qp.P.shape == (qp.n, qp.n) and qp.A.shape == (qp.m, qp.n)


def test_config0_random_qp():
    """n = 50, m = 500; P = MMᵀ + 1e-2·I; A at 15% N(0,1); q ~ N(0,1);
    l = −U[0,1], u = U[0,1]."""
    qp = pb.config_problem(0)
    assert (qp.n, qp.m) == (50, 500)
    assert 0.13 <= qp.A.nnz / (500 * 50) <= 0.17
    assert np.linalg.eigvalsh(qp.P_full().toarray()).min() >= 1e-2 - 1e-9
    assert np.all((qp.l >= -1) & (qp.l <= 0)) and np.all((qp.u >= 0) & (qp.u <= 1))
    assert abs(qp.q.mean()) < 0.5 and 0.6 < qp.q.std() < 1.4


def test_config1_lasso():
    """A_d 20000 × 200 at 15%; variables (x, y, t), n = m = 20400; rows
    A_d x − y = b, x − t ≤ 0, x + t ≥ 0; P = diag(0, 2I, 0); q = (0, 0, λ1)
    with λ = 0.2‖A_dᵀb‖∞."""
    qp = pb.config_problem(1)
    nf, md = 200, 20000
    assert (qp.n, qp.m) == (nf + md + nf, md + 2 * nf)
    Ad = qp.A[:md, :nf]
    assert 0.145 <= Ad.nnz / (md * nf) <= 0.155
    assert qp.A.nnz == Ad.nnz + md + 4 * nf
    b = qp.l[:md]
    assert np.array_equal(qp.l[:md], qp.u[:md])
    lam = 0.2 * np.max(np.abs(Ad.T @ b))
    assert np.allclose(qp.q, np.concatenate([np.zeros(nf + md), np.full(nf, lam)]), rtol=1e-12)
    assert np.array_equal(qp.P.diagonal(), np.concatenate([np.zeros(nf), np.full(md, 2.0), np.zeros(nf)]))
    assert np.all(np.isinf(qp.l[md:md + nf])) and np.all(qp.u[md:md + nf] == 0)
    assert np.all(qp.l[md + nf:] == 0) and np.all(np.isinf(qp.u[md + nf:]))


def test_config2_portfolio():
    """n = 10000 assets, k = 100 factors: F at 50% N(0,1), D_ii ~ U[0, √k];
    rows Fᵀx − y = 0, 1ᵀx = 1, x ≥ 0."""
    qp = pb.config_problem(2)
    na, k = 10000, 100
    assert (qp.n, qp.m) == (na + k, k + 1 + na)
    F = qp.meta["F"]
    assert 0.49 <= F.nnz / (na * k) <= 0.51
    D = qp.meta["D"]
    assert D.min() >= 0 and D.max() <= 10 and 4.5 < D.mean() < 5.5
    assert np.all(qp.l[:k] == 0) and np.all(qp.u[:k] == 0)
    assert qp.l[k] == 1 and qp.u[k] == 1
    assert np.all(qp.l[k + 1:] == 0) and np.all(np.isinf(qp.u[k + 1:]))


def test_config3_mpc_batch():
    """nx ~ U{4..32}, nu = ⌊nx/2⌋, T ~ U{10..30}; spectral radius of A_d at
    most 0.99; Q diagonal at 10% U[0,10]; R = 0.1·I; |x| ≤ U[1,2],
    |u| ≤ U[0.5,1.5], x₀ ~ U[−½, ½]; A holds the dense A_d and B_d blocks,
    the identities and the boxes, nothing else."""
    qps = pb.mpc_batch(256, seed=3000)
    nnz, qdens = [], []
    for qp in qps:
        nx, nu, T = qp.meta["nx"], qp.meta["nu"], qp.meta["T"]
        assert 4 <= nx <= 32 and nu == nx // 2 and 10 <= T <= 30
        assert np.max(np.abs(np.linalg.eigvals(qp.meta["Ad"]))) <= 0.99 + 1e-12
        assert qp.n == nx * (T + 1) + nu * T and qp.m == nx * (T + 1) + qp.n
        assert qp.A.nnz == T * nx * nx + T * nx * nu + nx * (T + 1) + qp.n
        pd = qp.P.diagonal()
        assert np.allclose(pd[nx * (T + 1):], 0.2)          # 2·R, objective without ½
        qd = pd[:nx] / 2.0
        assert np.all((qd >= 0) & (qd <= 10))
        qdens.append(np.mean(qd > 0))
        xbar, ubar, x0 = qp.meta["xbar"], qp.meta["ubar"], qp.meta["x0"]
        assert np.all((xbar >= 1) & (xbar <= 2)) and np.all((ubar >= 0.5) & (ubar <= 1.5))
        assert np.all(np.abs(x0) <= 0.5)
        nnz.append(qp.A.nnz)
    assert 0.07 <= np.mean(qdens) <= 0.13
    assert 1.1e4 <= np.mean(nnz) <= 1.45e4


def test_config4_serving_pool():
    """256 random QPs (m = 10n) and 256 Huber problems (data 100n × n), n
    log-uniform on [10, nmax]."""
    spec = pb.serving_pool_spec(seed=4000, pool=256, n_range=(10, 500))
    assert len(spec) == 512
    for cls in ("random_qp", "huber"):
        ns = np.array([n for c, n, _ in spec if c == cls])
        assert len(ns) == 256 and ns.min() >= 10 and ns.max() <= 500
        # log-uniform: the median sits near the geometric mean of the range
        assert 40 <= np.median(ns) <= 110
    qp = pb.random_qp(30, seed=1)
    assert qp.m == 300
    h = pb.huber(6, seed=1)
    assert h.meta["m_data"] == 600


def test_svm_workload():
    """App. A.7 (bench workload svm: 100 features, 10⁴ points): labels +1 on
    the first half, −1 on the rest; features N(±1/n, 1/n) at 15%; rows
    t ≥ diag(b)A_d x + 1 and t ≥ 0; P = blockdiag(2I, 0), q = (0, λ1)."""
    qp = pb.svm(100, seed=7000)
    n, m = 100, 10000
    assert (qp.n, qp.m) == (n + m, 2 * m)
    D = qp.A[:m, :n].toarray()          # diag(b)·A_d
    assert np.allclose(qp.A[:m, n:].toarray(), -np.eye(m))
    top, bot = D[: m // 2], -D[m // 2:]  # undo the labels: rows of A_d
    for half, mean in ((top, 1.0 / n), (bot, -1.0 / n)):
        vals = half[half != 0]
        assert 0.145 <= vals.size / half.size <= 0.155
        assert abs(vals.mean() - mean) < 0.1 / np.sqrt(n)
        assert abs(vals.std() - 1.0 / np.sqrt(n)) < 0.05 / np.sqrt(n)
    assert np.all(np.isinf(qp.l[:m])) and np.all(qp.u[:m] == -1)
    assert np.all(qp.l[m:] == 0) and np.all(np.isinf(qp.u[m:]))
    assert np.array_equal(qp.P.diagonal()[:n], np.full(n, 2.0)) and qp.P.nnz == n
    assert np.all(qp.q[:n] == 0) and np.all(qp.q[n:] == 1.0)


def test_eq_qp_workload():
    """App. A.2 (bench workload eqqp, n = 1000): m = n/2 equality rows
    l = u = b; P = MMᵀ + 1e-2·I with M at 15%."""
    qp = pb.eq_qp(1000, seed=8000)
    assert (qp.n, qp.m) == (1000, 500)
    assert np.array_equal(qp.l, qp.u)
    assert 0.14 <= qp.A.nnz / (500 * 1000) <= 0.16
    assert np.linalg.eigvalsh(qp.P_full().toarray()).min() >= 1e-2 - 1e-8

"""Parametric sequences of §8.4 (host logic) replayed on the FP64 CPU
oracle: every step's data is the update the sequence prescribes, and the
results satisfy properties the paper and the mathematics fix — the §8
acceptance test, the Lasso path's zero solution above 2‖A_dᵀb‖∞ and its
ℓ1 norm growing as λ falls, the MPC plant following the applied inputs
inside its bounds, and the budget and sign constraints of the portfolio."""
import numpy as np
import pytest

from paper_1711_08013_gb300 import parametric as pm
from paper_1711_08013_gb300 import problems as pb
from tests.kkt_check import acceptance

HIGH = dict(eps_abs=1e-9, eps_rel=1e-9, max_iter=400000, check_interval=10)


class OracleSession:
    """The oracle as a session: the current QP on the host, solved cold."""

    def __init__(self, oracle_mod, qp, **settings):
        self.O, self.qp, self.settings = oracle_mod, qp, settings
        self.solved = []

    def update(self, **upd):
        self.qp = pm.apply_update(self.qp, upd)

    def solve(self, warm=True):
        r = self.O.solve(self.qp, **self.settings)
        self.solved.append(self.qp)
        return pm.Step(r.x, r.y, r.status, r.iter, 0, 0.0, 0.0)


def check_steps(sess, steps, eps):
    for qp, st in zip(sess.solved, steps):
        assert st.status == 1
        prim, dual, ep, ed = acceptance(qp, st.x, st.y, eps, eps)
        assert prim <= ep and dual <= ed, (prim, ep, dual, ed)


def test_lasso_lambda_grid():
    qp = pb.lasso(8, seed=1)
    lam = pm.lasso_lambdas(qp, 100)
    assert lam[0] == pytest.approx(qp.meta["lam_max"]) and lam[-1] == pytest.approx(0.01 * lam[0])
    assert np.allclose(np.diff(np.log(lam)), np.log(0.01) / 99)
    ups = list(pm.lasso_path(qp, 5))
    off = qp.meta["n_feat"] + qp.meta["m_data"]
    for u, l_ in zip(ups, pm.lasso_lambdas(qp, 5)):
        assert np.all(u["q"][off:] == l_) and np.all(u["q"][:off] == 0.0)


def test_lasso_path_on_oracle(oracle_mod):
    qp = pb.lasso(8, seed=1)
    sess = OracleSession(oracle_mod, qp, **HIGH)
    steps = pm.run(sess, pm.lasso_path(qp, 6))
    assert len(steps) == 6
    check_steps(sess, steps, 1e-7)
    n = qp.meta["n_feat"]
    l1 = [np.abs(st.x[:n]).sum() for st in steps]
    # the ℓ1 norm of the Lasso solution does not decrease as λ decreases
    assert all(b >= a - 1e-6 * max(1.0, a) for a, b in zip(l1, l1[1:])), l1
    assert l1[-1] > l1[0]


def test_lasso_zero_above_threshold(oracle_mod):
    """With the objective ‖A_dx − b‖² + λ‖x‖₁ of App. A.5, x = 0 is optimal
    exactly when λ ≥ 2‖A_dᵀb‖∞ (the subgradient condition at x = 0)."""
    qp = pb.lasso(8, seed=1)
    n, m = qp.meta["n_feat"], qp.meta["m_data"]
    q = qp.q.copy()
    q[n + m:] = 2.05 * qp.meta["lam_max"]
    r = oracle_mod.solve(pm.apply_update(qp, {"q": q}), **HIGH)
    assert np.max(np.abs(r.x[:n])) <= 1e-6
    q[n + m:] = 1.5 * qp.meta["lam_max"]
    r = oracle_mod.solve(pm.apply_update(qp, {"q": q}), **HIGH)
    assert np.max(np.abs(r.x[:n])) > 1e-4


def test_mpc_closed_loop_on_oracle(oracle_mod):
    qp = pb.mpc_paper(4, T=5, seed=2)
    nx, nu, T = qp.meta["nx"], qp.meta["nu"], qp.meta["T"]
    sess = OracleSession(oracle_mod, qp, **HIGH)
    steps = pm.run(sess, pm.mpc_closed_loop(qp, 6))
    assert len(steps) == 6
    check_steps(sess, steps, 1e-7)
    u0 = [st.x[nx * (T + 1): nx * (T + 1) + nu] for st in steps]
    xs = pm.mpc_states(qp, u0[:-1])
    for k, (st, qk) in enumerate(zip(steps, sess.solved)):
        # the solved QP starts from the plant state, and so does its solution
        assert np.array_equal(qk.l[:nx], -xs[k]) and np.array_equal(qk.u[:nx], -xs[k])
        assert np.allclose(st.x[:nx], xs[k], atol=1e-6)
        assert np.all(np.abs(u0[k]) <= qp.meta["ubar"] + 1e-6)
        assert np.all(np.abs(xs[k]) <= qp.meta["xbar"] + 1e-6)


def test_mpc_paper_instance():
    """App. A.3 ranges: q at 70% density, ū in [0, 0.1], x_init inside
    ±x̄/2, terminal cost from the Riccati equation (P's x_T block solves
    Q_T = Q + AᵀQ_TA − AᵀQ_TB(R + BᵀQ_TB)⁻¹BᵀQ_TA)."""
    qp = pb.mpc_paper(6, T=4, seed=3)
    nx, nu, T = 6, 3, 4
    Ad, Bd, xbar = qp.meta["Ad"], qp.meta["Bd"], qp.meta["xbar"]
    assert np.all(qp.meta["ubar"] <= 0.1) and np.all(np.abs(qp.meta["x0"]) <= 0.5 * xbar)
    P = qp.P_full().toarray()
    QT = 0.5 * P[nx * T: nx * (T + 1), nx * T: nx * (T + 1)]
    Q = np.diag(0.5 * np.diag(P)[:nx])
    R = 0.1 * np.eye(nu)
    rhs = Q + Ad.T @ QT @ Ad - Ad.T @ QT @ Bd @ np.linalg.solve(R + Bd.T @ QT @ Bd, Bd.T @ QT @ Ad)
    assert np.allclose(QT, rhs, rtol=1e-8, atol=1e-8)
    assert np.max(np.abs(np.linalg.eigvals(Ad))) <= 0.99 + 1e-12


def test_portfolio_backtest_on_oracle(oracle_mod):
    qp = pb.portfolio(2, seed=4)
    k = qp.meta["k"]
    sess = OracleSession(oracle_mod, qp, **HIGH)
    trace = []
    steps = pm.run(sess, pm.portfolio_backtest(qp, days=5, days_per_month=2, seed=7), trace=trace)
    assert len(steps) == 5
    assert "A_val" not in trace[1] and "A_val" in trace[2] and "A_val" in trace[4]
    check_steps(sess, steps, 1e-7)
    n = qp.meta["F"].shape[0]
    for st, qk in zip(steps, sess.solved):
        x = st.x[:n]
        assert abs(x.sum() - 1.0) <= 1e-6 and x.min() >= -1e-6
        F = qk.A[:k, :n]
        assert np.allclose(st.x[n:], F @ x, atol=1e-6)   # y = Fᵀx (rows of A hold Fᵀ)
    # a month's risk-model update keeps D > 0 and the pattern of F
    F0 = qp.meta["F"]
    F2 = sess.solved[2].A[:k, :n].T
    assert F2.nnz == F0.nnz


def test_sequences_are_deterministic():
    qp = pb.portfolio(2, seed=4)
    a = list(pm.portfolio_backtest(qp, days=4, days_per_month=2, seed=9))
    b = list(pm.portfolio_backtest(qp, days=4, days_per_month=2, seed=9))
    for x, y in zip(a, b):
        assert x.keys() == y.keys()
        for key in x:
            assert np.array_equal(x[key], y[key])

"""Pins of the CPU oracle against what the paper and the mathematics fix
(closed forms, brute force, definitions, invariants, hand-derived fixtures).
None of these re-types the oracle's own formulas."""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1711_08013_gb300 import problems as pb
from tests.kkt_check import acceptance, dual_cert_ok, objective, primal_cert_ok

HIGH = dict(eps_abs=1e-9, eps_rel=1e-9, max_iter=200000, check_interval=10)


def dense_qp(P, q, A, l, u, name="dense"):
    P = np.asarray(P, float)
    A = np.asarray(A, float).reshape(-1, P.shape[0])
    return pb._finish(name, sp.csc_matrix(np.triu(P)), q, sp.csc_matrix(A), l, u)


# ----------------------------------------------------------------------------
# LDLᵀ and ordering (§3.1 direct method)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(6))
def test_ldl_matches_dense_solve(oracle_mod, seed):
    """Quasi-definite K = [H Bᵀ; B −G] (H, G ≻ 0): the LDLᵀ solve equals a
    dense LU solve, and D has n positive and m negative entries."""
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(1, 90)), int(rng.integers(0, 110))
    H = pb.sprandn(rng, n, n, 0.1)
    H = (H @ H.T + sp.diags(rng.uniform(0.1, 2.0, n))).toarray()
    B = pb.sprandn(rng, m, n, 0.15).toarray()
    G = np.diag(rng.uniform(0.01, 3.0, m))
    K = np.block([[H, B.T], [B, -G]])
    g = rng.standard_normal((n + m, 3))
    t, D, nnzL = oracle_mod.ldl_solve(sp.csc_matrix(np.triu(K)), g)
    ref = np.linalg.solve(K, g)
    assert np.max(np.abs(t - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref)))
    assert int(np.sum(D > 0)) == n and int(np.sum(D < 0)) == m


def test_ldl_arrow_fill(oracle_mod):
    """Arrowhead matrix with the hub first: minimum degree moves the hub to
    one of the last two pivots (the last leaf and the hub tie at degree 1),
    so L has exactly N−1 off-diagonal entries (no fill)."""
    N = 200
    K = np.eye(N) * 4.0
    K[0, :] = K[:, 0] = 1.0
    K[0, 0] = N + 1.0
    perm = oracle_mod.min_degree(sp.csc_matrix(K))
    assert sorted(perm.tolist()) == list(range(N))
    assert 0 in perm[-2:].tolist()
    t, D, nnzL = oracle_mod.ldl_solve(sp.csc_matrix(np.triu(K)), np.ones(N))
    assert nnzL == N - 1
    assert np.allclose(K @ t, np.ones(N), atol=1e-12)


# ----------------------------------------------------------------------------
# Closed forms
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(40))
def test_eq_qp_closed_form(oracle_mod, seed):
    """App. A.2: the solution of an equality-constrained QP solves
    [P Aᵀ; A 0][x; ν] = [−q; b] (Eq. eq_constr_qp_optimality)."""
    rng = np.random.default_rng(10_000 + seed)
    n = int(rng.integers(2, 61))
    # A sparse draw can have an empty or dependent row (an infeasible system);
    # such draws are replaced by a denser one of the same size.
    for density in (0.15, 0.5, 1.0):
        qp = pb.eq_qp(n, seed=10_000 + seed, density=density)
        P = qp.P_full().toarray()
        A = qp.A.toarray()
        m = A.shape[0]
        K = np.block([[P, A.T], [A, np.zeros((m, m))]])
        if np.linalg.cond(K) < 1e8:
            break
    sol = np.linalg.solve(K, np.concatenate([-qp.q, qp.l]))
    r = oracle_mod.solve(qp, **HIGH)
    assert r.status == oracle_mod.SOLVED
    scale = max(1.0, np.max(np.abs(sol)))
    assert np.max(np.abs(r.x - sol[:n])) <= 1e-6 * scale
    assert np.max(np.abs(r.y - sol[n:])) <= 1e-6 * scale


@pytest.mark.parametrize("seed", range(10))
def test_unconstrained_closed_form(oracle_mod, seed):
    """All bounds infinite: x = −P⁻¹q and y = 0."""
    qp = pb.unconstrained_qp(int(5 + 3 * seed), seed=seed)
    x_ref = -np.linalg.solve(qp.P_full().toarray(), qp.q)
    r = oracle_mod.solve(qp, **HIGH)
    assert r.status == oracle_mod.SOLVED
    assert np.max(np.abs(r.x - x_ref)) <= 1e-6 * max(1, np.max(np.abs(x_ref)))
    assert np.max(np.abs(r.y)) <= 1e-8


@pytest.mark.parametrize("seed", range(10))
def test_separable_box_closed_form(oracle_mod, seed):
    """Diagonal P ≻ 0 and A = I: x_i = clip(−q_i/P_ii, l_i, u_i),
    y = −(Px + q) (Eqs. dual_feas, compl_slack)."""
    qp = pb.box_qp(30 + seed, seed=seed)
    pd = qp.P.diagonal()
    x_ref = np.clip(-qp.q / pd, qp.l, qp.u)
    y_ref = -(pd * x_ref + qp.q)
    r = oracle_mod.solve(qp, **HIGH)
    assert r.status == oracle_mod.SOLVED
    assert np.max(np.abs(r.x - x_ref)) <= 1e-7
    assert np.max(np.abs(r.y - y_ref)) <= 1e-7


def _brute_force_active_set(qp):
    """Enumerate every (lower / upper / inactive) label of the m rows, solve
    the resulting equality-constrained KKT system and keep the point that is
    primal feasible with dual signs y_L ≤ 0, y_U ≥ 0 (Eq. compl_slack).  With
    P ≻ 0 the primal solution is unique."""
    P = qp.P_full().toarray()
    A = qp.A.toarray()
    n, m = A.shape[1], A.shape[0]
    best = None
    for labels in itertools.product((0, 1, 2), repeat=m):
        act = [i for i in range(m) if labels[i] != 0]
        b = np.array([qp.l[i] if labels[i] == 1 else qp.u[i] for i in act])
        if np.any(~np.isfinite(b)):
            continue
        As = A[act, :]
        k = len(act)
        K = np.block([[P, As.T], [As, np.zeros((k, k))]])
        try:
            sol = np.linalg.solve(K, np.concatenate([-qp.q, b]))
        except np.linalg.LinAlgError:
            continue
        if not np.all(np.isfinite(sol)):
            continue
        x = sol[:n]
        y = np.zeros(m)
        y[act] = sol[n:]
        Ax = A @ x
        if np.any(Ax < qp.l - 1e-9) or np.any(Ax > qp.u + 1e-9):
            continue
        if any(labels[i] == 1 and y[i] > 1e-9 for i in range(m)):
            continue
        if any(labels[i] == 2 and y[i] < -1e-9 for i in range(m)):
            continue
        best = (x, y)
        break
    return best


@pytest.mark.parametrize("seed", range(8))
def test_brute_force_active_set(oracle_mod, seed):
    """n ≤ 8, m ≤ 8: the oracle's x equals the enumerated active-set solution."""
    rng = np.random.default_rng(20_000 + seed)
    n = int(rng.integers(2, 9))
    m = int(rng.integers(1, 9))
    qp = pb.random_qp(n, m, seed=20_000 + seed, density=0.6)
    bf = _brute_force_active_set(qp)
    assert bf is not None
    r = oracle_mod.solve(qp, **HIGH)
    assert r.status == oracle_mod.SOLVED
    assert np.max(np.abs(r.x - bf[0])) <= 1e-6
    assert abs(objective(qp, r.x) - objective(qp, bf[0])) <= 1e-6 * max(1, abs(objective(qp, bf[0])))


# ----------------------------------------------------------------------------
# Hand-derived fixtures
# ----------------------------------------------------------------------------
def _load_golden():
    with open(os.path.join(os.path.dirname(__file__), "golden", "tiny_qps.json")) as f:
        data = json.load(f)
    conv = lambda v: [float(a) if not isinstance(a, str) else float(a) for a in v]
    cases = []
    for c in data["cases"]:
        qp = dense_qp(c["P"], c["q"], c["A"], conv(c["l"]), conv(c["u"]), c["name"])
        cases.append((c, qp))
    return cases


@pytest.mark.parametrize("case,qp", _load_golden(), ids=lambda v: getattr(v, "name", None) or v.get("name"))
def test_golden_tiny(oracle_mod, case, qp):
    if case["status"] == "solved":
        r = oracle_mod.solve(qp, **HIGH)
        assert r.status == oracle_mod.SOLVED
        assert np.allclose(r.x, case["x"], atol=1e-7)
        assert np.allclose(r.y, case["y"], atol=1e-7)
        assert abs(r.obj_val - case["obj"]) <= 1e-7
    elif case["status"] == "primal_infeasible":
        r = oracle_mod.solve(qp)
        assert r.status == oracle_mod.PRIMAL_INFEASIBLE
        d = r.prim_cert / np.linalg.norm(r.prim_cert)
        assert np.allclose(d, case["cert_dir"], atol=1e-3)
    else:
        r = oracle_mod.solve(qp)
        assert r.status == oracle_mod.DUAL_INFEASIBLE
        d = r.dual_cert / np.linalg.norm(r.dual_cert)
        assert np.allclose(d, case["cert_dir"], atol=1e-3)


# ----------------------------------------------------------------------------
# Certificates (§2.1, §3.4)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(5))
def test_primal_infeasibility_certificate(oracle_mod, seed):
    qp = pb.primal_infeasible_qp(4, seed=seed)
    r = oracle_mod.solve(qp)
    assert r.status == oracle_mod.PRIMAL_INFEASIBLE
    assert primal_cert_ok(qp, r.prim_cert, eps=1e-3)


@pytest.mark.parametrize("seed", range(5))
def test_dual_infeasibility_certificate(oracle_mod, seed):
    qp = pb.dual_infeasible_lp(3 + seed, seed=seed)
    r = oracle_mod.solve(qp)
    assert r.status == oracle_mod.DUAL_INFEASIBLE
    assert dual_cert_ok(qp, r.dual_cert, eps=1e-3)


# Certificates and reported residuals are unscaled (§5.1): pinned on badly
# scaled data, where a missing D, E or c changes the answer.
def _resid(qp, x, y, z):
    P = qp.P_full()
    return (float(np.max(np.abs(qp.A @ x - z), initial=0.0)),
            float(np.max(np.abs(P @ x + qp.q + qp.A.T @ y))))


@pytest.mark.parametrize("make", [lambda: pb.random_qp(30, seed=5), lambda: pb.mpc(5, 6, seed=2),
                                  lambda: pb.lasso(4, seed=3), lambda: pb.portfolio(2, seed=1)])
def test_reported_residuals_match_returned_point(oracle_mod, make):
    qp = make()
    r = oracle_mod.solve(qp)
    rp, rd = _resid(qp, r.x, r.y, r.z)
    assert r.prim_res == pytest.approx(rp, rel=1e-9, abs=1e-14)
    assert r.dual_res == pytest.approx(rd, rel=1e-9, abs=1e-14)


def _scaled_rows(qp, seed):
    rng = np.random.default_rng(seed)
    f = np.exp(rng.uniform(-3, 3, qp.m))
    Fm = sp.diags(f)
    return pb._finish(qp.name + "_rs", qp.P, qp.q, sp.csc_matrix(Fm @ qp.A), qp.l * f, qp.u * f)


def _scaled_cols(qp, seed):
    rng = np.random.default_rng(seed)
    g = np.exp(rng.uniform(-3, 3, qp.n))
    G = sp.diags(g)
    P = sp.csc_matrix(sp.triu(G @ qp.P_full() @ G))
    return pb._finish(qp.name + "_cs", P, g * qp.q, sp.csc_matrix(qp.A @ G), qp.l, qp.u)


@pytest.mark.parametrize("seed", range(4))
def test_primal_certificate_on_badly_scaled_rows(oracle_mod, seed):
    qp = _scaled_rows(pb.primal_infeasible_qp(4, seed=seed), 50 + seed)
    r = oracle_mod.solve(qp)
    assert r.status == oracle_mod.PRIMAL_INFEASIBLE
    assert primal_cert_ok(qp, r.prim_cert, eps=1e-3)


@pytest.mark.parametrize("seed", range(4))
def test_dual_certificate_on_badly_scaled_columns(oracle_mod, seed):
    qp = _scaled_cols(pb.dual_infeasible_lp(4 + seed, seed=seed), 60 + seed)
    r = oracle_mod.solve(qp)
    assert r.status == oracle_mod.DUAL_INFEASIBLE
    assert dual_cert_ok(qp, r.dual_cert, eps=1e-3)


def _coupled_dinf(seed):
    """min −x₁ − x₂ + q₃x₃ s.t. x₁ − x₂ = 0, x₁ ≥ 0, x₃ ∈ [−1, 1], columns
    scaled by random factors: unbounded along G⁻¹(1, 1, 0)."""
    rng = np.random.default_rng(seed)
    g = np.exp(rng.uniform(-2, 2, 3))
    A = sp.csc_matrix(np.array([[1.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]]) @ np.diag(g))
    q = np.array([-1.0, -1.0, rng.uniform(-1, 1)]) * g
    return pb._finish("dinf_coupled", sp.csc_matrix((3, 3)), q, A,
                      np.array([0.0, 0.0, -1.0]), np.array([0.0, np.inf, 1.0])), g


@pytest.mark.parametrize("seed", range(4))
def test_dual_certificate_couples_scaled_columns(oracle_mod, seed):
    qp, g = _coupled_dinf(seed)
    r = oracle_mod.solve(qp)
    assert r.status == oracle_mod.DUAL_INFEASIBLE
    assert dual_cert_ok(qp, r.dual_cert, eps=1e-3)
    d = r.dual_cert / np.linalg.norm(r.dual_cert)
    ref = np.array([1.0 / g[0], 1.0 / g[1], 0.0])
    assert np.allclose(d, ref / np.linalg.norm(ref), atol=1e-3)


def test_primal_certificate_with_one_sided_rows(oracle_mod):
    rng = np.random.default_rng(4)
    n = 5
    rows = [np.eye(1, n, 0).ravel(), np.eye(1, n, 0).ravel()]
    A = np.vstack(rows + [rng.standard_normal((6, n))])
    l = np.array([1.0, -np.inf] + [-5.0, -np.inf, -5.0, -np.inf, -5.0, -np.inf])
    u = np.array([np.inf, 0.0] + [np.inf, 5.0, np.inf, 5.0, np.inf, 5.0])
    qp = pb._finish("pinf_onesided", sp.eye(n), rng.standard_normal(n), sp.csc_matrix(A), l, u)
    r = oracle_mod.solve(qp)
    assert r.status == oracle_mod.PRIMAL_INFEASIBLE
    assert primal_cert_ok(qp, r.prim_cert, eps=1e-3)


def test_primal_infeasibility_with_active_one_sided_rows(oracle_mod):
    """x₁ ≥ 1 and x₁ ≤ 0 conflict while one-sided rows (x₂ ≥ 1, x₃ ≤ −1,
    x₄ ≥ 0.5) are held at their finite bounds by the cost.  Their multipliers
    settle at finite values, so a difference δy on such a row can carry the
    sign of its infinite side; paired with ±∞ it would make the support
    function of §3.4 infinite and hide the certificate.  Every instance must
    be declared primal infeasible with a valid certificate (reading R17)."""
    for seed in range(30):
        rng = np.random.default_rng(seed)
        n = 4
        A = np.vstack([np.eye(1, n, 0).ravel(), np.eye(1, n, 0).ravel(), np.eye(n)[1:],
                       rng.standard_normal((2, n))])
        l = np.array([1.0, -np.inf, 1.0, -np.inf, 0.5, -np.inf, -np.inf])
        u = np.array([np.inf, 0.0, np.inf, -1.0, np.inf, 3.0, 3.0])
        q = np.array([0.0, 5.0, -5.0, 5.0]) + 0.3 * rng.standard_normal(n)
        qp = pb._finish("pinf_active_onesided", sp.eye(n) * 0.1, q, sp.csc_matrix(A), l, u)
        r = oracle_mod.solve(qp, max_iter=4000)
        assert r.status == oracle_mod.PRIMAL_INFEASIBLE, (seed, r.status, r.iter)
        assert primal_cert_ok(qp, r.prim_cert, eps=1e-3), seed


def test_feasible_problems_are_not_flagged(oracle_mod):
    for seed in range(10):
        r = oracle_mod.solve(pb.random_qp(20, seed=seed))
        assert r.status == oracle_mod.SOLVED


# ----------------------------------------------------------------------------
# Invariants (§3.3): z ∈ [l, u], y_i > 0 ⇒ z_i = u_i, y_i < 0 ⇒ z_i = l_i
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("iters", [1, 2, 7, 40])
def test_iterate_invariants_exact(oracle_mod, iters):
    qp = pb.random_qp(15, seed=iters)
    r = oracle_mod.solve(qp, max_iter=iters, scaling_iters=0, eps_abs=0, eps_rel=0)
    assert np.all(r.z >= qp.l) and np.all(r.z <= qp.u)
    assert np.all(r.z[r.y > 0] == qp.u[r.y > 0])
    assert np.all(r.z[r.y < 0] == qp.l[r.y < 0])


def test_iterate_invariants_scaled(oracle_mod):
    qp = pb.random_qp(15, seed=3)
    r = oracle_mod.solve(qp, max_iter=30, eps_abs=0, eps_rel=0)
    tol = 1e-13 * (1 + np.abs(qp.u))
    assert np.all(np.abs(r.z[r.y > 0] - qp.u[r.y > 0]) <= tol[r.y > 0])
    assert np.all(np.abs(r.z[r.y < 0] - qp.l[r.y < 0]) <= 1e-13 * (1 + np.abs(qp.l[r.y < 0])))


# ----------------------------------------------------------------------------
# Eq-QP ADMM with α = 1 equals iterative refinement (App. A.2)
# ----------------------------------------------------------------------------
def test_eq_qp_is_iterative_refinement(oracle_mod):
    """With α = 1, no scaling and a fixed ρ, the iterates (x^k, y^k) for k ≥ 1
    follow t^{k+1} = t^k + (K+ΔK)⁻¹(g − K t^k) with K = [P Aᵀ; A 0],
    ΔK = diag(σI, −ρ⁻¹I), g = (−q, b)."""
    qp = pb.eq_qp(12, seed=5)
    n, m = qp.n, qp.m
    sigma, rho = 1e-2, 0.1 * 1e3  # equality rows use 10³ρ̄ (§5.2)
    kw = dict(alpha=1.0, rho=0.1, sigma=sigma, scaling_iters=0, adaptive_rho=0, eps_abs=0,
              eps_rel=0)
    r1 = oracle_mod.solve(qp, max_iter=1, **kw)
    P = qp.P_full().toarray()
    A = qp.A.toarray()
    K = np.block([[P, A.T], [A, np.zeros((m, m))]])
    dK = np.diag(np.concatenate([np.full(n, sigma), np.full(m, -1.0 / rho)]))
    g = np.concatenate([-qp.q, qp.l])
    t = np.concatenate([r1.x, r1.y])
    for k in range(2, 9):
        t = t + np.linalg.solve(K + dK, g - K @ t)
        rk = oracle_mod.solve(qp, max_iter=k, **kw)
        assert np.allclose(rk.x, t[:n], rtol=1e-9, atol=1e-10)
        assert np.allclose(rk.y, t[n:], rtol=1e-9, atol=1e-10)


# ----------------------------------------------------------------------------
# Ruiz equilibration (Alg. 2, Eq. pb:scaled_qp)
# ----------------------------------------------------------------------------
def test_ruiz_scaled_data_consistent(oracle_mod):
    """The scaled data equal P̄ = cDPD, q̄ = cDq, Ā = EAD, (l̄, ū) = (El, Eu)
    for the returned D, E, c (Eq. pb:scaled_qp)."""
    qp = pb.random_qp(30, seed=7)
    Pf = qp.P_full()
    s = oracle_mod.ruiz(Pf, qp.q, qp.A, qp.l, qp.u, scaling_iters=10, eps_equil=1e-3)
    D, E, c = s["D"], s["E"], s["c"]
    Pbar = sp.csc_matrix((s["P_x"], Pf.indices, Pf.indptr), shape=Pf.shape)
    Abar = sp.csc_matrix((s["A_x"], qp.A.indices, qp.A.indptr), shape=qp.A.shape)
    assert np.allclose(Pbar.toarray(), c * np.diag(D) @ Pf.toarray() @ np.diag(D), rtol=1e-12, atol=1e-14)
    assert np.allclose(Abar.toarray(), np.diag(E) @ qp.A.toarray() @ np.diag(D), rtol=1e-12, atol=1e-14)
    assert np.allclose(s["q"], c * D * qp.q, rtol=1e-12)
    assert np.allclose(s["l"], E * qp.l, rtol=1e-12) and np.allclose(s["u"], E * qp.u, rtol=1e-12)
    assert s["passes"] == 10


def test_ruiz_equilibrates_rows_and_columns(oracle_mod):
    """With P = 0 and q = 0 (so γ stays 1), repeated passes drive every row
    and column ∞-norm of Ā to 1 (Ruiz's fixed point)."""
    rng = np.random.default_rng(3)
    A = pb.sprandn(rng, 40, 25, 0.3)
    A = sp.diags(np.exp(rng.uniform(-4, 4, 40))) @ A @ sp.diags(np.exp(rng.uniform(-4, 4, 25)))
    A = sp.csc_matrix(A)
    keep = np.asarray((abs(A) > 0).sum(axis=1)).ravel() > 0
    A = sp.csc_matrix(A[keep])
    m = A.shape[0]
    Pf = sp.csc_matrix((25, 25))
    s = oracle_mod.ruiz(Pf, np.zeros(25), A, -np.ones(m), np.ones(m), scaling_iters=200,
                        eps_equil=1e-12)
    Abar = sp.csc_matrix((s["A_x"], A.indices, A.indptr), shape=A.shape)
    rn = abs(Abar).max(axis=1).toarray().ravel()
    cn = abs(Abar).max(axis=0).toarray().ravel()
    assert np.allclose(rn, 1.0, atol=1e-6) and np.allclose(cn[cn > 0], 1.0, atol=1e-6)
    assert s["c"] == 1.0


@pytest.mark.parametrize("seed", range(3))
def test_ruiz_cost_normalised_after_last_pass(oracle_mod, seed):
    """Alg. 2 ends each pass by scaling the cost with γ = 1/max(mean_j
    ‖P̄_:j‖∞, ‖q̄‖∞), so after the last pass that maximum is 1 (the data
    here keep both norms inside the clamp of reading R3)."""
    qp = pb.random_qp(30, seed=40 + seed)
    Pf = qp.P_full()
    s = oracle_mod.ruiz(Pf, qp.q, qp.A, qp.l, qp.u, scaling_iters=7, eps_equil=0.0)
    Pbar = sp.csc_matrix((s["P_x"], Pf.indices, Pf.indptr), shape=Pf.shape)
    mean_col = float(np.mean(abs(Pbar).max(axis=0).toarray()))
    assert max(mean_col, float(np.max(np.abs(s["q"])))) == pytest.approx(1.0, rel=1e-12)
    assert s["passes"] == 7


def test_ruiz_cost_scale_bounded_without_linear_cost(oracle_mod):
    """Reading R3: with q = 0 the vanishing ‖q̄‖∞ counts as 1 in the max, so
    γ ≤ 1 every pass and c stays at most 1 however many passes run (taken
    literally, 1/mean_j ‖P̄_:j‖∞ with mostly-zero columns of P̄ would grow c
    pass after pass)."""
    qp = pb.mpc(6, 10, seed=3)
    assert not np.any(qp.q)
    Pf = qp.P_full()
    cs = [oracle_mod.ruiz(Pf, qp.q, qp.A, qp.l, qp.u, scaling_iters=k, eps_equil=0.0)["c"]
          for k in (5, 10, 30)]
    assert all(0.0 < c <= 1.0 for c in cs)
    assert cs[2] >= 0.5 * cs[1]


def test_scaling_does_not_change_solution(oracle_mod):
    qp = pb.random_qp(25, seed=11)
    a = oracle_mod.solve(qp, scaling_iters=0, **HIGH)
    b = oracle_mod.solve(qp, scaling_iters=10, **HIGH)
    assert a.status == b.status == oracle_mod.SOLVED
    assert np.max(np.abs(a.x - b.x)) <= 1e-6


# ----------------------------------------------------------------------------
# ρ̄ adaptation direction (§5.2): the rule raises ρ̄ when the normalised primal
# residual dominates and lowers it when the dual one does.
# ----------------------------------------------------------------------------
def test_rho_update_gated_by_tolerance_factor(oracle_mod):
    """Reading R6: a new ρ̄ is applied only when it is more than the
    tolerance factor away.  ρ̄ stays in [1e-6, 1e6], so no proposal can be
    1e13 times away (no update ever), while with factor 1 any proposal that
    differs at all is applied."""
    qp = pb.random_qp(30, seed=2)
    never = oracle_mod.solve(qp, adaptive_rho_tolerance=1e13, max_iter=400)
    always = oracle_mod.solve(qp, adaptive_rho_tolerance=1.0, max_iter=400)
    assert never.rho_updates == 0 and never.rho_bar == 0.1
    assert always.rho_updates >= 1 and always.rho_bar != 0.1


def test_rho_adaptation_direction(oracle_mod):
    qp = pb.random_qp(30, seed=2)
    lo = oracle_mod.solve(qp, rho=1e-5, max_rho_updates=1)
    hi = oracle_mod.solve(qp, rho=1e3, max_rho_updates=1)
    assert lo.rho_updates == 1 and lo.rho_bar > 1e-5
    assert hi.rho_updates == 1 and hi.rho_bar < 1e3


# ----------------------------------------------------------------------------
# The paper's problem classes: acceptance test of §8 at ε = 1e-3 and 1e-5
# ----------------------------------------------------------------------------
CLASSES = [
    ("random_qp", lambda: pb.random_qp(40, seed=1)),
    ("eq_qp", lambda: pb.eq_qp(40, seed=1)),
    ("mpc", lambda: pb.mpc(8, 10, seed=1)),
    ("portfolio", lambda: pb.portfolio(5, seed=1)),
    ("lasso", lambda: pb.lasso(8, seed=1)),
    ("huber", lambda: pb.huber(6, seed=1)),
    ("svm", lambda: pb.svm(6, seed=1)),
]


@pytest.mark.parametrize("eps", [1e-3, 1e-5])
@pytest.mark.parametrize("name,make", CLASSES, ids=[c[0] for c in CLASSES])
def test_problem_classes_acceptance(oracle_mod, name, make, eps):
    qp = make()
    r = oracle_mod.solve(qp, eps_abs=eps, eps_rel=eps, max_iter=100000)
    assert r.status == oracle_mod.SOLVED, (name, r.status, r.iter)
    prim, dual, ep, ed = acceptance(qp, r.x, r.y, eps, eps)
    assert prim <= ep and dual <= ed
    assert abs(objective(qp, r.x) - r.obj_val) <= 1e-9 * max(1.0, abs(r.obj_val))


def test_warm_start_from_solution_converges_immediately(oracle_mod):
    """Warm start (§6) from the solution of the same problem terminates at the
    first check."""
    qp = pb.random_qp(30, seed=4)
    r = oracle_mod.solve(qp, eps_abs=1e-6, eps_rel=1e-6, max_iter=100000)
    w = oracle_mod.solve(qp, x0=r.x, y0=r.y, check_interval=1, eps_abs=1e-3, eps_rel=1e-3)
    assert w.status == oracle_mod.SOLVED and w.iter <= 2


def test_invalid_inputs_rejected(oracle_mod):
    qp = pb.random_qp(5, seed=0)
    bad = pb.random_qp(5, seed=0)
    bad.l = bad.u + 1.0
    with pytest.raises(ValueError):
        oracle_mod.solve(bad)
    with pytest.raises(ValueError):
        oracle_mod.solve(qp, alpha=2.5)

"""Solution polishing (§4) in the oracle, pinned against solutions that do
not come from the polishing code: the enumerated active-set solution (brute
force, n, m ≤ 8), the closed forms of equality-constrained and separable box
QPs, and high-accuracy ADMM runs.  A polished point replaces the ADMM point
only when it is at least as good, so a wrong active-set guess must leave the
solution untouched."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1711_08013_gb300 import problems as pb
from tests.kkt_check import acceptance, objective
from tests.test_oracle_pins import _brute_force_active_set

HIGH = dict(eps_abs=1e-10, eps_rel=1e-10, max_iter=400000, check_interval=10)


@pytest.mark.parametrize("seed", range(8))
def test_polish_reaches_brute_force_solution(oracle_mod, seed):
    """At the default ε = 1e-3 the ADMM point is only approximate; when the
    sign pattern of y names the right active set, polishing returns the
    enumerated active-set solution to rounding level."""
    rng = np.random.default_rng(20_000 + seed)
    n = int(rng.integers(2, 9))
    m = int(rng.integers(1, 9))
    qp = pb.random_qp(n, m, seed=20_000 + seed, density=0.6)
    bf = _brute_force_active_set(qp)
    assert bf is not None
    r = oracle_mod.solve(qp, polish=1)
    plain = oracle_mod.solve(qp)
    assert r.status == oracle_mod.SOLVED and r.polished in (1, -1)
    if r.polished == 1:
        assert np.max(np.abs(r.x - bf[0])) <= 1e-9 * max(1.0, np.max(np.abs(bf[0])))
        assert r.prim_res <= plain.prim_res and r.dual_res <= plain.dual_res
    else:
        assert np.array_equal(r.x, plain.x)


@pytest.mark.parametrize("seed", range(6))
def test_polish_eq_qp_closed_form(oracle_mod, seed):
    """Equality rows are active with either sign: polishing solves the KKT
    system [P Aᵀ; A 0][x; ν] = [−q; b] of App. A.2 up to refinement error."""
    qp = pb.eq_qp(20 + 5 * seed, seed=30_000 + seed, density=0.5)
    P = qp.P_full().toarray()
    A = qp.A.toarray()
    m = A.shape[0]
    sol = np.linalg.solve(np.block([[P, A.T], [A, np.zeros((m, m))]]),
                          np.concatenate([-qp.q, qp.l]))
    r = oracle_mod.solve(qp, polish=1)
    assert r.status == oracle_mod.SOLVED and r.polished == 1
    scale = max(1.0, np.max(np.abs(sol)))
    assert np.max(np.abs(r.x - sol[:qp.P.shape[0]])) <= 1e-9 * scale
    assert np.max(np.abs(r.y - sol[qp.P.shape[0]:])) <= 1e-8 * scale


@pytest.mark.parametrize("seed", range(5))
def test_polish_box_closed_form(oracle_mod, seed):
    """Separable box QP: x = clip(−q/P_ii, l, u) exactly after polishing."""
    qp = pb.box_qp(30 + seed, seed=seed)
    pd = qp.P.diagonal()
    x_ref = np.clip(-qp.q / pd, qp.l, qp.u)
    r = oracle_mod.solve(qp, polish=1)
    assert r.polished == 1
    assert np.max(np.abs(r.x - x_ref)) <= 1e-10


@pytest.mark.parametrize("name,make", [
    ("random", lambda: pb.random_qp(40, seed=3)),
    ("mpc", lambda: pb.mpc(6, 8, seed=4)),
    ("lasso", lambda: pb.lasso(20, seed=1)),
])
def test_polish_matches_high_accuracy(oracle_mod, name, make):
    qp = make()
    r = oracle_mod.solve(qp, polish=1)
    hi = oracle_mod.solve(qp, **HIGH)
    assert r.polished == 1, name
    prim, dual, ep, ed = acceptance(qp, r.x, r.y, 1e-9, 1e-9)
    assert prim <= ep and dual <= ed, (name, prim, dual)
    f, f_hi = objective(qp, r.x), objective(qp, hi.x)
    assert abs(f - f_hi) <= 1e-8 * max(1.0, abs(f_hi)), name


def test_polish_rejected_leaves_admm_solution(oracle_mod):
    """A wrong active-set guess (App. A.7 SVM at ε = 1e-3) is rejected and
    the returned point is the ADMM point."""
    qp = pb.svm(10, seed=1)
    r = oracle_mod.solve(qp, polish=1)
    plain = oracle_mod.solve(qp)
    assert r.polished == -1
    assert np.array_equal(r.x, plain.x) and np.array_equal(r.y, plain.y)


def test_polish_not_run_unless_solved(oracle_mod):
    qp = pb.random_qp(30, seed=2)
    r = oracle_mod.solve(qp, polish=1, max_iter=5)
    assert r.status == oracle_mod.MAX_ITER and r.polished == 0


def test_polish_with_dependent_active_rows(oracle_mod):
    """Every bound row of a box QP appears twice: the active rows are linearly
    dependent, so the unregularised reduced KKT matrix is singular; the δ
    regularisation still polishes to the clip formula."""
    n = 12
    qp0 = pb.box_qp(n, seed=3)
    A = sp.vstack([qp0.A, qp0.A]).tocsc()
    qp = pb._finish("box_dup", qp0.P, qp0.q, A, np.concatenate([qp0.l, qp0.l]),
                    np.concatenate([qp0.u, qp0.u]))
    r = oracle_mod.solve(qp, polish=1)
    x_ref = np.clip(-qp.q / qp.P.diagonal(), qp0.l, qp0.u)
    assert r.polished == 1
    assert np.max(np.abs(r.x - x_ref)) <= 1e-9


def test_polish_lp_with_zero_cost_free_direction(oracle_mod):
    """LP whose optimal face is not a vertex: min x₁ s.t. x₁ ≥ 0, x₂ ∈ [−1, 1]
    with no cost on x₂.  The reduced KKT matrix without the δ of Eq.
    (kkt_polish_reg) is singular along x₂; with it, polishing returns x₁ = 0
    at the bound and a feasible x₂."""
    A = sp.csc_matrix(np.eye(2))
    qp = pb._finish("lp_face", sp.csc_matrix((2, 2)), np.array([1.0, 0.0]), A,
                    np.array([0.0, -1.0]), np.array([np.inf, 1.0]))
    r = oracle_mod.solve(qp, polish=1)
    assert r.status == oracle_mod.SOLVED and r.polished == 1
    assert abs(r.x[0]) <= 1e-12 and -1.0 <= r.x[1] <= 1.0


def test_polish_qp_with_zero_curvature_face(oracle_mod):
    """min ½(x₁ + x₂)² s.t. x₁ + x₂ ≥ 1, x₁ − x₂ ∈ [−1, 1]: the optimal set
    is a segment along (1, −1), where P (diagonal stored) has no curvature
    and q no cost.  Only the δ of Eq. (kkt_polish_reg) makes the reduced
    system solvable; the polished point lies on the face."""
    P = sp.csc_matrix(np.array([[1.0, 1.0], [0.0, 1.0]]))
    A = sp.csc_matrix(np.array([[1.0, 1.0], [1.0, -1.0]]))
    qp = pb._finish("qp_face", P, np.zeros(2), A, np.array([1.0, -1.0]), np.array([np.inf, 1.0]))
    r = oracle_mod.solve(qp, polish=1)
    assert r.status == oracle_mod.SOLVED and r.polished == 1
    assert abs(r.x[0] + r.x[1] - 1.0) <= 1e-10 and abs(r.x[0] - r.x[1]) <= 1.0 + 1e-12


def test_polished_points_keep_the_sign_invariant(oracle_mod):
    """Every returned point, polished or not, satisfies the invariant of §3.3
    that ADMM iterates satisfy exactly: y_i > 0 only at an upper bound and
    y_i < 0 only at a lower bound (Eq. compl_slack).  Polishing guesses its
    active set from the signs of a loose (ε = 1e-2) ADMM point, so over
    these 400 small QPs some guesses yield multipliers of the wrong sign;
    those points must be rejected."""
    polished = 0
    for seed in range(400):
        rng = np.random.default_rng(90_000 + seed)
        n, m = int(rng.integers(2, 7)), int(rng.integers(2, 9))
        qp = pb.random_qp(n, m, seed=90_000 + seed, density=0.7)
        r = oracle_mod.solve(qp, polish=1, eps_abs=1e-2, eps_rel=1e-2)
        assert r.status == oracle_mod.SOLVED
        polished += r.polished == 1
        tol = 1e-9 * (1.0 + np.abs(r.z))
        up = r.y > 0
        lo = r.y < 0
        assert np.all(np.abs(r.z[up] - qp.u[up]) <= tol[up]), seed
        assert np.all(np.abs(r.z[lo] - qp.l[lo]) <= tol[lo]), seed
    assert polished >= 350

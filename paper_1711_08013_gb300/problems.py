"""Seeded synthetic QP generators shaped like the paper's problem classes (App. A).

Every generator returns a :class:`QP` in the boundary's input format: the upper
triangle of P and the full A as CSC matrices (scipy.sparse, sorted indices,
int32 indices, float64 values), and dense float64 vectors q, l, u.  Infinite
bounds are IEEE ``±inf``.

This module draws random numbers and assembles matrices; it holds none of the
solver's arithmetic.  It is the one module that both the CPU oracle tests and
the CUDA path import.

Objectives printed in App. A without the factor 1/2 of the standard form
(MPC Eq. in App. A.3, portfolio App. A.4, Lasso App. A.5, Huber App. A.6) are
taken literally, so P is twice the printed quadratic block.  Random sparsity
"with 15% nonzero elements" is an independent Bernoulli mask per entry with
N(0,1) values on the mask.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

__all__ = [
    "QP", "random_qp", "eq_qp", "lasso", "portfolio", "mpc", "mpc_batch", "huber",
    "svm", "box_qp", "unconstrained_qp", "primal_infeasible_qp", "dual_infeasible_lp",
    "config_problem", "perturb_vectors", "serving_pool_spec",
]


@dataclasses.dataclass
class QP:
    """minimize ½xᵀPx + qᵀx subject to l ≤ Ax ≤ u (Eq. pb:qp, §1.1)."""
    name: str
    P: sp.csc_matrix          # upper triangle, n × n
    q: np.ndarray
    A: sp.csc_matrix          # m × n
    l: np.ndarray
    u: np.ndarray
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.P.shape[0]

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def nnz(self) -> int:
        """N = nnz(P) + nnz(A) of the size tuple (n, m, N), §1.1."""
        return int(self.P.nnz + self.A.nnz)

    def P_full(self) -> sp.csc_matrix:
        U = self.P
        return (U + sp.triu(U, k=1).T).tocsc()


def _csc(M) -> sp.csc_matrix:
    """CSC with int32 indices, sorted, duplicates summed and stored zeros
    dropped (block constructions such as the MPC dynamics, a block-sparse
    Kronecker product minus an identity, store whole blocks with their
    zeros)."""
    M = sp.csc_matrix(M)
    M.sum_duplicates()
    M.eliminate_zeros()
    M.sort_indices()
    M.indices = M.indices.astype(np.int32)
    M.indptr = M.indptr.astype(np.int32)
    M.data = M.data.astype(np.float64)
    return M


def _finish(name, P, q, A, l, u, **meta) -> QP:
    Pu = _csc(sp.triu(sp.csc_matrix(P)))
    A = _csc(A)
    return QP(name, Pu, np.asarray(q, np.float64), A,
              np.asarray(l, np.float64), np.asarray(u, np.float64), dict(meta))


def sprandn(rng: np.random.Generator, rows: int, cols: int, density: float,
            scale: float = 1.0, loc: float = 0.0, chunk_entries: int = 1 << 24) -> sp.csc_matrix:
    """rows × cols matrix with an independent Bernoulli(density) mask and
    N(loc, scale²) values on the mask.  Drawn row-block by row-block so that
    very large instances need no dense rows × cols array."""
    if rows == 0 or cols == 0:
        return sp.csc_matrix((rows, cols))
    rb = max(1, chunk_entries // max(cols, 1))
    r_idx, c_idx, vals = [], [], []
    for r0 in range(0, rows, rb):
        r1 = min(rows, r0 + rb)
        mask = rng.random((r1 - r0, cols)) < density
        rr, cc = np.nonzero(mask)
        r_idx.append(rr + r0)
        c_idx.append(cc)
        vals.append(loc + scale * rng.standard_normal(rr.size))
    r = np.concatenate(r_idx)
    c = np.concatenate(c_idx)
    v = np.concatenate(vals)
    return sp.csc_matrix((v, (r, c)), shape=(rows, cols))


# ----------------------------------------------------------------------------
# App. A.1: random QP
# ----------------------------------------------------------------------------
def random_qp(n: int, m: int | None = None, seed: int = 0, density: float = 0.15) -> QP:
    """App. A.1: P = MMᵀ + 1e-2·I with M at 15% N(0,1); A (m × n, default
    m = 10n) at 15% N(0,1); q ~ N(0,1); l = −U(0,1), u = U(0,1)."""
    rng = np.random.default_rng(seed)
    m = 10 * n if m is None else m
    M = sprandn(rng, n, n, density)
    P = (M @ M.T + 1e-2 * sp.eye(n)).tocsc()
    A = sprandn(rng, m, n, density)
    q = rng.standard_normal(n)
    l = -rng.random(m)
    u = rng.random(m)
    return _finish(f"random_qp_n{n}_m{m}_s{seed}", P, q, A, l, u, cls="random_qp", seed=seed)


# ----------------------------------------------------------------------------
# App. A.2: equality-constrained QP
# ----------------------------------------------------------------------------
def eq_qp(n: int, seed: int = 0, density: float = 0.15) -> QP:
    """App. A.2: m = ⌊n/2⌋ equality rows Ax = b encoded as l = u = b."""
    rng = np.random.default_rng(seed)
    m = n // 2
    M = sprandn(rng, n, n, density)
    P = (M @ M.T + 1e-2 * sp.eye(n)).tocsc()
    A = sprandn(rng, m, n, density)
    q = rng.standard_normal(n)
    b = rng.standard_normal(m)
    return _finish(f"eq_qp_n{n}_s{seed}", P, q, A, b, b.copy(), cls="eq_qp", seed=seed)


# ----------------------------------------------------------------------------
# App. A.3: optimal control (MPC), with the ranges of the batched workload
# ----------------------------------------------------------------------------
def mpc(nx: int, T: int, seed: int = 0, nu: int | None = None, q_density: float = 0.10,
        xbar_range=(1.0, 2.0), ubar_range=(0.5, 1.5), x0_range=(-0.5, 0.5),
        x0_scale: float | None = None, terminal: str = "Q") -> QP:
    """App. A.3 MPC QP in z = (x_0..x_T, u_0..u_{T-1}).

    Dynamics A_d = I + 0.1·N(0,1), scaled by 0.99/ρ(A_d) when its spectral
    radius exceeds 0.99; B_d ~ N(0,1); Q = diag(q) with q at `q_density`
    U[0,10]; R = 0.1·I; terminal cost Q_T = Q, or with terminal="dare" the
    LQR cost-to-go of (A_d, B_d, Q, R) from the discrete algebraic Riccati
    equation; |x_t| ≤ x̄, |u_t| ≤ ū; x_0 = x_init with x_init ~ U(x0_range),
    or U(−s·x̄, s·x̄) for x0_scale = s.  Rows: x_0 = x_init, A_d x_t + B_d u_t
    − x_{t+1} = 0 (equalities), then the state and input boxes.  meta keeps
    A_d, B_d, x̄, ū and x_init for closed-loop simulation.
    """
    rng = np.random.default_rng(seed)
    nu = nx // 2 if nu is None else nu
    Ad = np.eye(nx) + 0.1 * rng.standard_normal((nx, nx))
    rad = float(np.max(np.abs(np.linalg.eigvals(Ad))))
    if rad > 0.99:
        Ad *= 0.99 / rad
    Bd = rng.standard_normal((nx, nu))
    qd = np.where(rng.random(nx) < q_density, 10.0 * rng.random(nx), 0.0)
    xbar = rng.uniform(*xbar_range, size=nx)
    ubar = rng.uniform(*ubar_range, size=nu)
    if x0_scale is None:
        x0 = rng.uniform(*x0_range, size=nx)
    else:
        x0 = rng.uniform(-1.0, 1.0, size=nx) * x0_scale * xbar

    nX = nx * (T + 1)
    n = nX + nu * T
    # P = 2·blockdiag(Q, …, Q, Q_T, R, …, R), objective read without the ½.
    if terminal == "Q":
        pdiag = np.concatenate([np.tile(qd, T + 1), np.full(nu * T, 0.1)]) * 2.0
        P = sp.diags(pdiag, format="csc")
    elif terminal == "dare":
        import scipy.linalg as sla
        QT = sla.solve_discrete_are(Ad, Bd, np.diag(qd), 0.1 * np.eye(nu))
        QT = 0.5 * (QT + QT.T)
        P = 2.0 * sp.block_diag([sp.diags(np.tile(qd, T)), sp.csc_matrix(QT),
                                 sp.diags(np.full(nu * T, 0.1))], format="csc")
    else:
        raise ValueError("terminal must be 'Q' or 'dare'")
    q = np.zeros(n)

    # Equality block: rows 0..nx-1: x_0 = x0; rows nx(t+1)..: A_d x_t + B_d u_t - x_{t+1} = 0
    Ad_s = sp.csc_matrix(Ad)
    Bd_s = sp.csc_matrix(Bd)
    Sx = sp.kron(sp.eye(T + 1, k=-1), Ad_s) - sp.eye(nX)
    Su = sp.kron(sp.vstack([sp.csc_matrix((1, T)), sp.eye(T)]), Bd_s)
    Aeq = sp.hstack([Sx, Su])
    beq = np.concatenate([-x0, np.zeros(nx * T)])
    Abox = sp.eye(n)
    lbox = np.concatenate([np.tile(-xbar, T + 1), np.tile(-ubar, T)])
    ubox = -lbox
    A = sp.vstack([Aeq, Abox]).tocsc()
    l = np.concatenate([beq, lbox])
    u = np.concatenate([beq, ubox])
    return _finish(f"mpc_nx{nx}_T{T}_s{seed}", P, q, A, l, u, cls="mpc", nx=nx, nu=nu, T=T,
                   seed=seed, Ad=Ad, Bd=Bd, xbar=xbar, ubar=ubar, x0=x0)


def mpc_paper(nx: int, T: int = 10, seed: int = 0) -> QP:
    """App. A.3 with the paper's own instance ranges (the parametric
    closed-loop workload of §8.4): q at 70% density, ū ~ U(0, 0.1),
    x_init ~ U(−0.5x̄, 0.5x̄), Q_T from the Riccati equation."""
    return mpc(nx, T, seed=seed, q_density=0.7, ubar_range=(0.0, 0.1), x0_scale=0.5,
               terminal="dare")


def mpc_batch_spec(count: int = 4096, seed: int = 3000, nx_range=(4, 32),
                   T_range=(10, 30)) -> list[tuple[int, int, int]]:
    """(nx, T, seed) of every problem of the batched ragged MPC workload:
    nx ~ U{4..32} and T ~ U{10..30} drawn from seed `seed`, problem i then
    generated with seed `seed`+1+i (so any subset can be generated alone)."""
    rng = np.random.default_rng(seed)
    nxs = rng.integers(nx_range[0], nx_range[1] + 1, size=count)
    Ts = rng.integers(T_range[0], T_range[1] + 1, size=count)
    return [(int(nxs[i]), int(Ts[i]), seed + 1 + i) for i in range(count)]


def mpc_spec_work(nx: int, T: int) -> float:
    """Estimated matrix entries of one batched MPC problem (dense dynamics
    blocks, identity couplings and boxes): the weight by which problems are
    ordered and sharded before they are generated."""
    nu = nx // 2
    n = nx * (T + 1) + nu * T
    return float(T * nx * (nx + nu + 1) + nx + 2 * n)


def mpc_batch(count: int = 4096, seed: int = 3000, nx_range=(4, 32), T_range=(10, 30)) -> list[QP]:
    """Batched ragged MPC workload: problem i draws nx ~ U{4..32},
    T ~ U{10..30} from seed `seed`, then is generated with seed `seed`+1+i."""
    return [mpc(nx, T, seed=sd) for nx, T, sd in mpc_batch_spec(count, seed, nx_range, T_range)]


# ----------------------------------------------------------------------------
# App. A.4: portfolio optimisation (factor model)
# ----------------------------------------------------------------------------
def portfolio_data(F: sp.csc_matrix, Dd: np.ndarray, mu: np.ndarray, gamma: float = 1.0):
    """(P, q, A, l, u) of App. A.4 in variables (x, y), y = Fᵀx: P =
    blockdiag(2D, 2I), q = (−μ/γ, 0); rows Fᵀx − y = 0, 1ᵀx = 1, x ≥ 0."""
    n, k = F.shape
    P = sp.diags(np.concatenate([2.0 * Dd, 2.0 * np.ones(k)]), format="csc")
    q = np.concatenate([-mu / gamma, np.zeros(k)])
    A = sp.vstack([
        sp.hstack([F.T, -sp.eye(k)]),
        sp.hstack([sp.csc_matrix(np.ones((1, n))), sp.csc_matrix((1, k))]),
        sp.hstack([sp.eye(n), sp.csc_matrix((n, k))]),
    ]).tocsc()
    l = np.concatenate([np.zeros(k), [1.0], np.zeros(n)])
    u = np.concatenate([np.zeros(k), [1.0], np.full(n, np.inf)])
    return P, q, A, l, u


def portfolio(k: int, seed: int = 0, n: int | None = None, gamma: float = 1.0) -> QP:
    """App. A.4 in variables (x, y), y = Fᵀx (see portfolio_data); n = 100k
    assets, F at 50% N(0,1), D_ii ~ U[0, √k], μ ~ N(0,1).  meta keeps F, D
    and μ for the back test of §8.4."""
    rng = np.random.default_rng(seed)
    n = 100 * k if n is None else n
    F = sprandn(rng, n, k, 0.5)
    Dd = rng.uniform(0.0, math.sqrt(k), size=n)
    mu = rng.standard_normal(n)
    P, q, A, l, u = portfolio_data(F, Dd, mu, gamma)
    return _finish(f"portfolio_k{k}_n{n}_s{seed}", P, q, A, l, u, cls="portfolio", k=k,
                   seed=seed, F=F, D=Dd, mu=mu, gamma=gamma)


# ----------------------------------------------------------------------------
# App. A.5: Lasso
# ----------------------------------------------------------------------------
def lasso(n: int, seed: int = 0, m: int | None = None, lam_frac: float = 0.2) -> QP:
    """App. A.5 in variables (x, y, t): minimise yᵀy + λ1ᵀt subject to
    y = A_d x − b and −t ≤ x ≤ t; A_d is m × n (m = 100n) at 15% N(0,1),
    v_i = 0 w.p. 0.5 else N(0, 1/n), b = A_d v + N(0,1), λ = ‖A_dᵀb‖∞/5."""
    rng = np.random.default_rng(seed)
    m = 100 * n if m is None else m
    Ad = sprandn(rng, m, n, 0.15)
    v = np.where(rng.random(n) < 0.5, 0.0, rng.standard_normal(n) / math.sqrt(n))
    b = Ad @ v + rng.standard_normal(m)
    lam = lam_frac * float(np.max(np.abs(Ad.T @ b)))
    In = sp.eye(n)
    P = sp.block_diag([sp.csc_matrix((n, n)), 2.0 * sp.eye(m), sp.csc_matrix((n, n))]).tocsc()
    q = np.concatenate([np.zeros(n + m), lam * np.ones(n)])
    A = sp.vstack([
        sp.hstack([Ad, -sp.eye(m), sp.csc_matrix((m, n))]),
        sp.hstack([In, sp.csc_matrix((n, m)), -In]),
        sp.hstack([In, sp.csc_matrix((n, m)), In]),
    ]).tocsc()
    l = np.concatenate([b, np.full(n, -np.inf), np.zeros(n)])
    u = np.concatenate([b, np.zeros(n), np.full(n, np.inf)])
    return _finish(f"lasso_n{n}_m{m}_s{seed}", P, q, A, l, u, cls="lasso", lam=lam,
                   lam_max=lam / lam_frac, n_feat=n, m_data=m, seed=seed)


# ----------------------------------------------------------------------------
# App. A.6: Huber fitting
# ----------------------------------------------------------------------------
def huber(n: int, seed: int = 0, m: int | None = None, M: float = 1.0) -> QP:
    """App. A.6 in variables (x, u, r, s): minimise uᵀu + 2M1ᵀ(r + s)
    subject to A_d x − u − r + s = b, r ≥ 0, s ≥ 0; A_d is m × n (m = 100n)
    at 15% N(0,1); v ~ N(0, 1/n); noise N(0, 1/4) w.p. 0.95 else U[0, 10]."""
    rng = np.random.default_rng(seed)
    m = 100 * n if m is None else m
    Ad = sprandn(rng, m, n, 0.15)
    v = rng.standard_normal(n) / math.sqrt(n)
    noise = np.where(rng.random(m) < 0.95, 0.5 * rng.standard_normal(m), 10.0 * rng.random(m))
    b = Ad @ v + noise
    Im = sp.eye(m)
    P = sp.block_diag([sp.csc_matrix((n, n)), 2.0 * Im, sp.csc_matrix((2 * m, 2 * m))]).tocsc()
    q = np.concatenate([np.zeros(n + m), 2.0 * M * np.ones(2 * m)])
    Z = sp.csc_matrix((m, m))
    A = sp.vstack([
        sp.hstack([Ad, -Im, -Im, Im]),
        sp.hstack([sp.csc_matrix((m, n)), Z, Im, Z]),
        sp.hstack([sp.csc_matrix((m, n)), Z, Z, Im]),
    ]).tocsc()
    l = np.concatenate([b, np.zeros(2 * m)])
    u = np.concatenate([b, np.full(2 * m, np.inf)])
    return _finish(f"huber_n{n}_m{m}_s{seed}", P, q, A, l, u, cls="huber", n_feat=n, m_data=m,
                   seed=seed)


# ----------------------------------------------------------------------------
# App. A.7: support vector machine
# ----------------------------------------------------------------------------
def svm(n: int, seed: int = 0, m: int | None = None, lam: float = 1.0) -> QP:
    """App. A.7 in variables (x, t): minimise xᵀx + λ1ᵀt subject to
    t ≥ diag(b)A_d x + 1, t ≥ 0; labels b = +1 for the first half of the
    m = 100n points and −1 for the rest; A_d entries N(±1/n, 1/n) at 15%."""
    rng = np.random.default_rng(seed)
    m = 100 * n if m is None else m
    mh = m // 2
    A1 = sprandn(rng, mh, n, 0.15, scale=1.0 / math.sqrt(n), loc=1.0 / n)
    A2 = sprandn(rng, m - mh, n, 0.15, scale=1.0 / math.sqrt(n), loc=-1.0 / n)
    Ad = sp.vstack([A1, A2]).tocsc()
    b = np.concatenate([np.ones(mh), -np.ones(m - mh)])
    P = sp.block_diag([2.0 * sp.eye(n), sp.csc_matrix((m, m))]).tocsc()
    q = np.concatenate([np.zeros(n), lam * np.ones(m)])
    A = sp.vstack([
        sp.hstack([sp.diags(b) @ Ad, -sp.eye(m)]),
        sp.hstack([sp.csc_matrix((m, n)), sp.eye(m)]),
    ]).tocsc()
    l = np.concatenate([np.full(m, -np.inf), np.zeros(m)])
    u = np.concatenate([-np.ones(m), np.full(m, np.inf)])
    return _finish(f"svm_n{n}_m{m}_s{seed}", P, q, A, l, u, cls="svm", seed=seed)


# ----------------------------------------------------------------------------
# Small families used by the tests
# ----------------------------------------------------------------------------
def box_qp(n: int, seed: int = 0) -> QP:
    """Separable QP: diagonal P ≻ 0, A = I, finite boxes (some rows free or
    one-sided).  Its solution is clip(−q/P_ii, l, u) coordinate-wise."""
    rng = np.random.default_rng(seed)
    pd = rng.uniform(0.5, 3.0, size=n)
    q = 2.0 * rng.standard_normal(n)
    l = -rng.uniform(0.1, 1.0, size=n)
    u = rng.uniform(0.1, 1.0, size=n)
    kind = rng.integers(0, 4, size=n)
    l[kind == 1] = -np.inf
    u[kind == 2] = np.inf
    return _finish(f"box_qp_n{n}_s{seed}", sp.diags(pd), q, sp.eye(n), l, u, cls="box_qp")


def unconstrained_qp(n: int, seed: int = 0, m: int = 3) -> QP:
    """P ≻ 0 with m constraint rows whose bounds are all infinite."""
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    P = M @ M.T + n * np.eye(n)
    A = sprandn(rng, m, n, 0.5)
    return _finish(f"unc_qp_n{n}_s{seed}", sp.csc_matrix(P), rng.standard_normal(n), A,
                   np.full(m, -np.inf), np.full(m, np.inf), cls="unconstrained")


def primal_infeasible_qp(n: int = 4, seed: int = 0) -> QP:
    """x_1 ≥ 1 and x_1 ≤ 0 as two rows, plus random feasible box rows."""
    rng = np.random.default_rng(seed)
    P = sp.eye(n)
    rows = [np.eye(1, n, 0).ravel(), np.eye(1, n, 0).ravel()]
    A = np.vstack(rows + [rng.standard_normal((2, n))])
    l = np.array([1.0, -np.inf, -10.0, -10.0])
    u = np.array([np.inf, 0.0, 10.0, 10.0])
    return _finish(f"pinf_qp_n{n}_s{seed}", P, rng.standard_normal(n), sp.csc_matrix(A), l, u,
                   cls="primal_infeasible")


def dual_infeasible_lp(n: int = 3, seed: int = 0) -> QP:
    """minimise −x_1 subject to x_1 ≥ 0 and box rows on the other coordinates:
    unbounded below along e_1."""
    rng = np.random.default_rng(seed)
    P = sp.csc_matrix((n, n))
    q = np.zeros(n)
    q[0] = -1.0
    A = sp.eye(n)
    l = np.concatenate([[0.0], -np.ones(n - 1)])
    u = np.concatenate([[np.inf], np.ones(n - 1)])
    q[1:] = rng.standard_normal(n - 1)
    return _finish(f"dinf_lp_n{n}_s{seed}", P, q, A, l, u, cls="dual_infeasible")


# ----------------------------------------------------------------------------
# Workload recipes (seed = 1000·config + instance)
# ----------------------------------------------------------------------------
def config_problem(config: int, instance: int = 0, **kw) -> QP:
    """The single-problem workloads: 0 random QP n=50 m=500; 1 Lasso with a
    20000 × 200 data matrix; 2 portfolio n=10000 k=100."""
    seed = 1000 * config + instance
    if config == 0:
        return random_qp(kw.get("n", 50), kw.get("m", 500), seed=seed)
    if config == 1:
        return lasso(kw.get("n", 200), seed=seed, m=kw.get("m", 20000))
    if config == 2:
        return portfolio(kw.get("k", 100), seed=seed, n=kw.get("n", 10000))
    raise ValueError(f"no single-problem recipe for config {config}")


def perturb_vectors(rng: np.random.Generator, qp: QP, scale: float = 0.05):
    """Serving-request perturbation: q_j + scale·N(0,1)·(1+|q_j|); each row's
    bounds are multiplied by one factor max(0.5, 1 + scale·N(0,1)), which
    keeps l ≤ u, equality rows equal, infinite bounds infinite and 0 inside
    [l, u] wherever it was."""
    q = qp.q + scale * rng.standard_normal(qp.n) * (1.0 + np.abs(qp.q))
    f = np.maximum(0.5, 1.0 + scale * rng.standard_normal(qp.m))
    l = np.where(np.isfinite(qp.l), qp.l * f, qp.l)
    u = np.where(np.isfinite(qp.u), qp.u * f, qp.u)
    return q, l, u


def serving_pool_spec(seed: int = 4000, pool: int = 256, n_range=(10, 5000)):
    """Problem-ID pool of the serving stream: per class, `pool` IDs with
    n ~ logU[n_range]; returns a list of (class, n, seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for cls in ("random_qp", "huber"):
        ns = np.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1]), size=pool))
        for i in range(pool):
            out.append((cls, int(round(ns[i])), seed + 1 + len(out)))
    return out

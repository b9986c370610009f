"""Parametric programs (§8.4): sequences of related QPs solved with the data
kept on the GPU, each solve starting from the previous solution (§6 warm
start) unless ``warm`` is off, in which case it starts from zero iterates
with ρ̄ reset to its initial value.

* Lasso regularisation path: λ runs over ``nlam`` values logarithmically
  spaced from λ_max = ‖A_dᵀb‖∞ down to 0.01·λ_max; only q changes.
* MPC closed loop: at every step the QP is solved for the current initial
  state, the first input is applied to the plant x⁺ = A_d x + B_d u₀, and the
  initial-state rows (l = u = −x_init) are updated; only l and u change.
* Portfolio back test: every day μ ← 0.9μ + N(0, 0.1); at the start of every
  month of ``days_per_month`` trading days D_ii ← 0.9D_ii + U[0, 0.1√k] and
  the nonzeros F_ij ← 0.9F_ij + N(0, 0.1), same sparsity, so the matrices
  are updated in place and the scaling and Jacobi diagonal are rebuilt on
  the device (no structural work).

A sequence is a generator of data updates (dicts with any of q, l, u,
P_val, A_val, where P_val and A_val are CSC value arrays in the pattern of
the first QP's upper-triangular P and A).  It receives each step's primal
solution through ``send``, so closed-loop sequences can react to it.
``run`` replays a sequence on a session; ``GpuSession`` is the session over
the GPU solver.  Host-side bookkeeping only: every solve runs in the library.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import problems as pb
from .solver import Solver


@dataclasses.dataclass
class Step:
    x: np.ndarray
    y: np.ndarray
    status: int
    iter: int
    pcg_iters: int
    solve_time: float      # device seconds of the solve
    wall: float            # host seconds of update + solve + result read-back
    z: np.ndarray | None = None


class GpuSession:
    """One QP resident on the GPU, updated and re-solved in place."""

    def __init__(self, qp, stream: int | None = None, **settings):
        settings.setdefault("warm_start", 1)
        self.rho = settings.get("rho", 0.1)
        self.solver = Solver(qp, stream=stream, **settings)
        self.n, self.m = self.solver.n, self.solver.m

    def update(self, q=None, l=None, u=None, P_val=None, A_val=None):
        if P_val is not None or A_val is not None:
            self.solver.update_matrices(P_val, A_val)
        if q is not None or l is not None or u is not None:
            self.solver.update_vectors(q, l, u)

    def solve(self, warm: bool = True) -> Step:
        t0 = time.perf_counter()
        if not warm:
            self.solver.update_rho(self.rho)
            self.solver.warm_start(np.zeros(self.n), np.zeros(self.m))
        r = self.solver.solve()
        return Step(r.x, r.y, r.status, r.iter, r.pcg_iters, r.solve_time,
                    time.perf_counter() - t0, r.z)

    def close(self):
        self.solver.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run(session, sequence, warm: bool = True, limit: int | None = None,
        trace: list | None = None) -> list[Step]:
    """Apply each update of ``sequence`` to ``session`` and solve; the step's
    primal solution is sent back to the sequence.  ``trace`` collects the
    updates in order."""
    steps = []
    try:
        upd = next(sequence)
        while True:
            if trace is not None:
                trace.append(upd)
            session.update(**upd)
            st = session.solve(warm)
            steps.append(st)
            if limit is not None and len(steps) >= limit:
                break
            upd = sequence.send(st.x)
    except StopIteration:
        pass
    return steps


# ----------------------------------------------------------------------------
# the three sequences of §8.4
# ----------------------------------------------------------------------------
def lasso_lambdas(qp, nlam: int = 100, lo_frac: float = 0.01) -> np.ndarray:
    lam_max = qp.meta["lam_max"]
    return np.logspace(np.log10(lam_max), np.log10(lo_frac * lam_max), nlam)


def lasso_path(qp, nlam: int = 100, lo_frac: float = 0.01):
    """Updates of q = (0, 0, λ1) along the regularisation path."""
    off = qp.meta["n_feat"] + qp.meta["m_data"]
    for lam in lasso_lambdas(qp, nlam, lo_frac):
        q = qp.q.copy()
        q[off:] = lam
        yield {"q": q}


def mpc_closed_loop(qp, steps: int = 100):
    """Updates of the initial-state rows; the plant is propagated with the
    first input of each solution."""
    nx, nu, T = qp.meta["nx"], qp.meta["nu"], qp.meta["T"]
    Ad, Bd = qp.meta["Ad"], qp.meta["Bd"]
    x = np.array(qp.meta["x0"], dtype=np.float64)
    u0_at = nx * (T + 1)
    for _ in range(steps):
        l = qp.l.copy()
        u = qp.u.copy()
        l[:nx] = -x
        u[:nx] = -x
        z = yield {"l": l, "u": u}
        x = Ad @ x + Bd @ z[u0_at:u0_at + nu]


def mpc_states(qp, inputs) -> np.ndarray:
    """Plant states x_0, x_1, … under the given first inputs (for checks)."""
    Ad, Bd = qp.meta["Ad"], qp.meta["Bd"]
    xs = [np.array(qp.meta["x0"], dtype=np.float64)]
    for u0 in inputs:
        xs.append(Ad @ xs[-1] + Bd @ u0)
    return np.array(xs)


def portfolio_backtest(qp, days: int = 960, days_per_month: int = 20, seed: int = 0):
    """Daily μ updates and monthly risk-model (D, F) updates."""
    rng = np.random.default_rng(seed)
    k, gamma = qp.meta["k"], qp.meta["gamma"]
    F = qp.meta["F"].copy()
    D = np.array(qp.meta["D"], dtype=np.float64)
    mu = np.array(qp.meta["mu"], dtype=np.float64)
    for day in range(days):
        upd = {}
        if day > 0 and day % days_per_month == 0:
            D = 0.9 * D + rng.uniform(0.0, 0.1 * np.sqrt(k), size=D.shape)
            F.data = 0.9 * F.data + rng.normal(0.0, 0.1, size=F.data.shape)
            P, _, A, _, _ = pb.portfolio_data(F, D, mu, gamma)
            Pu, Ac = pb._csc(P), pb._csc(A)
            if not (np.array_equal(Pu.indptr, qp.P.indptr) and np.array_equal(Pu.indices, qp.P.indices)
                    and np.array_equal(Ac.indptr, qp.A.indptr)
                    and np.array_equal(Ac.indices, qp.A.indices)):
                raise RuntimeError("risk-model update changed the sparsity pattern")
            upd["P_val"], upd["A_val"] = Pu.data, Ac.data
        if day > 0:
            mu = 0.9 * mu + rng.normal(0.0, 0.1, size=mu.shape)
            upd["q"] = np.concatenate([-mu / gamma, np.zeros(k)])
        yield upd


def apply_update(qp, upd: dict):
    """The QP that an update turns ``qp`` into (host copy, for checks)."""
    P, A = qp.P.copy(), qp.A.copy()
    if upd.get("P_val") is not None:
        P.data = np.asarray(upd["P_val"], np.float64).copy()
    if upd.get("A_val") is not None:
        A.data = np.asarray(upd["A_val"], np.float64).copy()
    q = np.asarray(upd["q"], np.float64) if upd.get("q") is not None else qp.q
    l = np.asarray(upd["l"], np.float64) if upd.get("l") is not None else qp.l
    u = np.asarray(upd["u"], np.float64) if upd.get("u") is not None else qp.u
    return pb.QP(qp.name, P, q.copy(), A, l.copy(), u.copy(), dict(qp.meta))

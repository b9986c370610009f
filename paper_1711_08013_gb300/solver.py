"""Convenience object over the C ABI (one solver = one QP resident on the GPU)."""
from __future__ import annotations

import dataclasses

import numpy as np

from . import _binding as B


@dataclasses.dataclass
class Result:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    status: int
    iter: int
    pcg_iters: int
    rho_updates: int
    obj_val: float
    prim_res: float
    dual_res: float
    rho_estimate: float
    setup_time: float
    solve_time: float
    launch: int
    polished: int = 0


def _sized(name, v, size):
    """The C ABI reads exactly `size` values behind each pointer: refuse
    arrays of another length before they reach it."""
    if v is not None and np.size(v) != size:
        raise ValueError(f"{name} has {np.size(v)} entries, expected {size}")
    return v


class Solver:
    """``Solver(qp, **settings)`` with ``qp`` exposing P (upper CSC), q, A, l, u."""

    def __init__(self, qp, stream: int | None = None, **settings):
        self.n, self.m = qp.P.shape[0], qp.A.shape[0]
        self.nnz_p, self.nnz_a = qp.P.nnz, qp.A.nnz
        self.settings = B.osqp_set_default_settings(**settings)
        self.handle = B.osqp_setup(qp.P, qp.q, qp.A, qp.l, qp.u, self.settings, stream)

    def solve(self) -> Result:
        B.osqp_solve(self.handle)
        return self.result()

    def result(self) -> Result:
        x, y, z, info = B.osqp_get_solution(self.handle, self.n, self.m)
        return Result(x, y, z, info.status, info.iter, info.pcg_iters, info.rho_updates,
                      info.obj_val, info.prim_res, info.dual_res, info.rho_estimate,
                      info.setup_time, info.solve_time, info.launch, info.polished)

    def certificate(self):
        return B.osqp_get_certificate(self.handle, self.n, self.m)

    def scaling(self):
        """(D, E, c, Jacobi diagonal) as held on the device."""
        return B.osqp_diag_scaling(self.handle, self.n, self.m)

    def update_vectors(self, q=None, l=None, u=None):
        B.osqp_update_vectors(self.handle, _sized("q", q, self.n), _sized("l", l, self.m),
                              _sized("u", u, self.m))

    def update_matrices(self, P_val=None, A_val=None):
        B.osqp_update_matrices(self.handle, _sized("P_val", P_val, self.nnz_p),
                               _sized("A_val", A_val, self.nnz_a))

    def update_rho(self, rho_bar: float):
        B.osqp_update_rho(self.handle, rho_bar)

    def warm_start(self, x=None, y=None):
        B.osqp_warm_start(self.handle, _sized("x", x, self.n), _sized("y", y, self.m))

    def close(self):
        if self.handle:
            B.osqp_cleanup(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """Many independent QPs resident on the GPU, solved by one persistent launch."""

    def __init__(self, qps, stream: int | None = None, **settings):
        self.sizes = [(qp.P.shape[0], qp.A.shape[0]) for qp in qps]
        self.settings = B.osqp_set_default_settings(**settings)
        self.handle = B.osqp_batch_setup(qps, self.settings, stream)

    def solve(self, subset=None):
        if subset is None:
            B.osqp_batch_solve(self.handle)
        else:
            B.osqp_batch_solve_subset(self.handle, subset)

    def reset(self):
        B.osqp_batch_reset(self.handle)

    def update_vectors(self, i, q=None, l=None, u=None):
        n, m = self.sizes[i]
        B.osqp_batch_update_vectors(self.handle, i, _sized("q", q, n), _sized("l", l, m),
                                    _sized("u", u, m))

    def result(self, i) -> Result:
        n, m = self.sizes[i]
        x, y, z, info = B.osqp_batch_get(self.handle, i, n, m)
        return Result(x, y, z, info.status, info.iter, info.pcg_iters, info.rho_updates,
                      info.obj_val, info.prim_res, info.dual_res, info.rho_estimate,
                      info.setup_time, info.solve_time, info.launch, info.polished)

    def close(self):
        if self.handle:
            B.osqp_batch_cleanup(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

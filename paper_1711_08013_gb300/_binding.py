"""Thin ctypes binding of libosqp_gb300.so (names as in include/osqp_gb300.h).

Argument marshalling only: numpy arrays (host) or raw device pointers (ints,
e.g. ``torch.Tensor.data_ptr()``) are passed straight to the C ABI; every
numeric step runs in the library's CUDA kernels.  Loading fails loudly when
the library is missing — there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OSQP_OK = 0
OSQP_ERR_DIMS, OSQP_ERR_CSC, OSQP_ERR_NONFINITE, OSQP_ERR_LGTU = -1, -2, -3, -4
OSQP_ERR_SETTINGS, OSQP_ERR_CUDA, OSQP_ERR_OOM, OSQP_ERR_ARG = -5, -6, -7, -8
OSQP_ERR_DEVICE, OSQP_ERR_LIMIT = -9, -10
UNSOLVED, SOLVED, MAX_ITER, PRIMAL_INFEASIBLE, DUAL_INFEASIBLE = 0, 1, 2, 3, 4
TIME_LIMIT, NUMERICAL_ERROR = 5, 6
FP64, FP32_MIXED = 0, 1

_lib = None


class osqp_csc(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("n_cols", C.c_int32), ("nnz", C.c_int32),
                ("colptr", C.c_void_p), ("rowind", C.c_void_p), ("val", C.c_void_p)]


class osqp_settings(C.Structure):
    _fields_ = [
        ("rho", C.c_double), ("sigma", C.c_double), ("alpha", C.c_double),
        ("eps_abs", C.c_double), ("eps_rel", C.c_double),
        ("eps_pinf", C.c_double), ("eps_dinf", C.c_double),
        ("adaptive_rho_tolerance", C.c_double), ("eps_equil", C.c_double),
        ("pcg_tol_fraction", C.c_double), ("pcg_tol_floor", C.c_double),
        ("time_limit", C.c_double),
        ("max_iter", C.c_int32), ("check_interval", C.c_int32), ("adaptive_rho", C.c_int32),
        ("scaling_iters", C.c_int32), ("max_rho_updates", C.c_int32),
        ("pcg_max_iter", C.c_int32), ("precision", C.c_int32), ("warm_start", C.c_int32),
        ("launch", C.c_int32), ("polish", C.c_int32), ("polish_refine_iter", C.c_int32),
        ("delta", C.c_double), ("autotune", C.c_int32), ("pad2", C.c_int32),
    ]


class osqp_info(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("iter", C.c_int32), ("pcg_iters", C.c_int32),
        ("rho_updates", C.c_int32), ("ruiz_passes", C.c_int32), ("launch", C.c_int32),
        ("obj_val", C.c_double), ("prim_res", C.c_double), ("dual_res", C.c_double),
        ("rho_estimate", C.c_double), ("setup_time", C.c_double), ("solve_time", C.c_double),
        ("polished", C.c_int32), ("pad", C.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_SIGS = {
    "osqp_set_default_settings": (None, [C.POINTER(osqp_settings)]),
    "osqp_error_message": (C.c_char_p, [C.c_int32]),
    "osqp_setup": (C.c_int32, [C.POINTER(_P), C.POINTER(osqp_csc), _P, C.POINTER(osqp_csc), _P, _P,
                               C.POINTER(osqp_settings), _P]),
    "osqp_solve": (C.c_int32, [_P]),
    "osqp_solve_async": (C.c_int32, [_P]),
    "osqp_update_vectors": (C.c_int32, [_P, _P, _P, _P]),
    "osqp_update_matrices": (C.c_int32, [_P, _P, _P]),
    "osqp_load_data": (C.c_int32, [_P, _P, _P, _P, _P, _P]),
    "osqp_load_data_device": (C.c_int32, [_P, _P, _P, _P, _P, _P]),
    "osqp_update_rho": (C.c_int32, [_P, C.c_double]),
    "osqp_warm_start": (C.c_int32, [_P, _P, _P]),
    "osqp_get_solution": (C.c_int32, [_P, _P, _P, _P, C.POINTER(osqp_info)]),
    "osqp_get_solution_device": (C.c_int32, [_P, _P, _P]),
    "osqp_get_certificate": (C.c_int32, [_P, _P, _P]),
    "osqp_cleanup": (C.c_int32, [_P]),
    "osqp_diag_barrier_timeout": (C.c_int32, [C.c_double]),
    "osqp_diag_scaling": (C.c_int32, [_P, _P, _P, _P, _P]),
    "osqp_diag_schedule": (C.c_int32, [_P, _P, _P]),
    "osqp_batch_uses_cluster": (C.c_int32, [_P, C.c_int32]),
    "osqp_batch_setup": (C.c_int32, [C.POINTER(_P), C.c_int32, _P, _P, _P, _P, _P,
                                     C.POINTER(osqp_settings), _P]),
    "osqp_batch_solve": (C.c_int32, [_P]),
    "osqp_batch_solve_async": (C.c_int32, [_P]),
    "osqp_batch_solve_subset": (C.c_int32, [_P, _P, C.c_int32]),
    "osqp_batch_reset": (C.c_int32, [_P]),
    "osqp_batch_update_vectors": (C.c_int32, [_P, C.c_int32, _P, _P, _P]),
    "osqp_batch_get": (C.c_int32, [_P, C.c_int32, _P, _P, _P, C.POINTER(osqp_info)]),
    "osqp_batch_cleanup": (C.c_int32, [_P]),
    "osqp_batch_launch": (C.c_int32, [_P, C.c_int32, _P, C.c_int32, _P, _P, _P]),
    "osqp_batch_slot_query": (C.c_int32, [_P, C.c_int32]),
    "osqp_batch_slot_wait": (C.c_int32, [_P, C.c_int32]),
    "osqp_batch_footprint": (C.c_int64, [_P, C.c_int32]),
    "osqp_batch_schedule": (C.c_int32, [_P, C.c_int32, _P]),
    "osqp_batch_update_all": (C.c_int32, [_P, _P, _P, _P]),
    "osqp_batch_get_all": (C.c_int32, [_P, _P, _P]),
    "osqp_batch_tuning": (C.c_int32, [_P, C.c_int32, _P, _P]),
}
OSQP_BATCH_MAX_SLOTS = 32


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load (building first if needed) the CUDA library."""
    global _lib
    if _lib is None:
        if not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"CUDA library missing: {_build.LIB}")
        L = C.CDLL(_build.LIB)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class OsqpError(RuntimeError):
    def __init__(self, code, where=""):
        msg = lib().osqp_error_message(code).decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


def _check(rc, where):
    if rc != OSQP_OK:
        raise OsqpError(rc, where)


def _ptr(a):
    """Host numpy array → pointer; int (device address) passes through."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    return a.ctypes.data_as(C.c_void_p).value


def osqp_set_default_settings(**overrides) -> osqp_settings:
    s = osqp_settings()
    lib().osqp_set_default_settings(C.byref(s))
    for k, v in overrides.items():
        if not hasattr(s, k):
            raise KeyError(f"unknown setting {k}")
        setattr(s, k, v)
    return s


def _csc(M, keep):
    colptr = np.ascontiguousarray(M.indptr, dtype=np.int32)
    rowind = np.ascontiguousarray(M.indices, dtype=np.int32)
    val = np.ascontiguousarray(M.data, dtype=np.float64)
    keep += [colptr, rowind, val]
    return osqp_csc(M.shape[0], M.shape[1], int(val.size), _ptr(colptr), _ptr(rowind), _ptr(val))


def osqp_setup(P_upper, q, A, l, u, settings: osqp_settings, stream: int | None = None):
    """P_upper, A: scipy CSC (sorted indices); q, l, u: float64 arrays."""
    keep = []
    Pc = _csc(P_upper, keep)
    Ac = _csc(A, keep)
    q = np.ascontiguousarray(q, np.float64)
    l = np.ascontiguousarray(l, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    h = C.c_void_p()
    rc = lib().osqp_setup(C.byref(h), C.byref(Pc), _ptr(q), C.byref(Ac), _ptr(l), _ptr(u),
                          C.byref(settings), stream)
    _check(rc, "osqp_setup")
    return h.value


def osqp_solve(h):
    _check(lib().osqp_solve(h), "osqp_solve")


def osqp_solve_async(h):
    _check(lib().osqp_solve_async(h), "osqp_solve_async")


def osqp_update_vectors(h, q=None, l=None, u=None):
    arrs = [None if v is None else np.ascontiguousarray(v, np.float64) for v in (q, l, u)]
    _check(lib().osqp_update_vectors(h, *[_ptr(a) for a in arrs]), "osqp_update_vectors")


def osqp_update_matrices(h, P_val=None, A_val=None):
    arrs = [None if v is None else np.ascontiguousarray(v, np.float64) for v in (P_val, A_val)]
    _check(lib().osqp_update_matrices(h, *[_ptr(a) for a in arrs]), "osqp_update_matrices")


def osqp_load_data(h, P_val, q, A_val, l, u):
    """Host arrays (numpy) or host addresses (ints, e.g. pinned tensors)."""
    _check(lib().osqp_load_data(h, _ptr(P_val), _ptr(q), _ptr(A_val), _ptr(l), _ptr(u)),
           "osqp_load_data")


def osqp_load_data_device(h, P_val: int, q: int, A_val: int, l: int, u: int):
    _check(lib().osqp_load_data_device(h, P_val, q, A_val, l, u), "osqp_load_data_device")


def osqp_update_rho(h, rho_bar: float):
    _check(lib().osqp_update_rho(h, float(rho_bar)), "osqp_update_rho")


def osqp_warm_start(h, x=None, y=None):
    arrs = [None if v is None else np.ascontiguousarray(v, np.float64) for v in (x, y)]
    _check(lib().osqp_warm_start(h, *[_ptr(a) for a in arrs]), "osqp_warm_start")


def osqp_get_solution(h, n: int, m: int):
    x, y, z = np.empty(n), np.empty(m), np.empty(m)
    info = osqp_info()
    _check(lib().osqp_get_solution(h, _ptr(x), _ptr(y), _ptr(z), C.byref(info)),
           "osqp_get_solution")
    return x, y, z, info


def osqp_get_solution_device(h, x_dev: int | None, y_dev: int | None):
    _check(lib().osqp_get_solution_device(h, x_dev, y_dev), "osqp_get_solution_device")


def osqp_get_certificate(h, n: int, m: int):
    py, dx = np.empty(m), np.empty(n)
    _check(lib().osqp_get_certificate(h, _ptr(py), _ptr(dx)), "osqp_get_certificate")
    return py, dx


def osqp_diag_scaling(h, n: int, m: int):
    """D (n), E (m), c and the Jacobi diagonal (n) as the solver holds them."""
    D, E, dg, c = np.empty(n), np.empty(m), np.empty(n), C.c_double(0.0)
    _check(lib().osqp_diag_scaling(h, _ptr(D), _ptr(E), C.addressof(c), _ptr(dg)),
           "osqp_diag_scaling")
    return D, E, c.value, dg


def osqp_cleanup(h):
    if h:
        _check(lib().osqp_cleanup(h), "osqp_cleanup")


# ---------------------------------------------------------------------------
# batched solves
# ---------------------------------------------------------------------------
def osqp_batch_setup(qps, settings: osqp_settings, stream: int | None = None):
    """qps: sequence of objects with P (upper CSC), q, A (CSC), l, u."""
    count = len(qps)
    keep = []
    Ps = (osqp_csc * count)()
    As = (osqp_csc * count)()
    qv, lv, uv = (C.c_void_p * count)(), (C.c_void_p * count)(), (C.c_void_p * count)()
    for i, qp in enumerate(qps):
        Ps[i] = _csc(qp.P, keep)
        As[i] = _csc(qp.A, keep)
        arrs = [np.ascontiguousarray(v, np.float64) for v in (qp.q, qp.l, qp.u)]
        keep += arrs
        qv[i], lv[i], uv[i] = (_ptr(a) for a in arrs)
    h = C.c_void_p()
    rc = lib().osqp_batch_setup(C.byref(h), count, C.cast(Ps, C.c_void_p), C.cast(qv, C.c_void_p),
                                C.cast(As, C.c_void_p), C.cast(lv, C.c_void_p),
                                C.cast(uv, C.c_void_p), C.byref(settings), stream)
    _check(rc, "osqp_batch_setup")
    return h.value


def osqp_batch_solve(h):
    _check(lib().osqp_batch_solve(h), "osqp_batch_solve")


def osqp_batch_solve_async(h):
    _check(lib().osqp_batch_solve_async(h), "osqp_batch_solve_async")


def osqp_batch_solve_subset(h, idx):
    a = np.ascontiguousarray(idx, np.int32)
    _check(lib().osqp_batch_solve_subset(h, _ptr(a), int(a.size)), "osqp_batch_solve_subset")


def osqp_batch_reset(h):
    _check(lib().osqp_batch_reset(h), "osqp_batch_reset")


def osqp_batch_update_vectors(h, i, q=None, l=None, u=None):
    arrs = [None if v is None else np.ascontiguousarray(v, np.float64) for v in (q, l, u)]
    _check(lib().osqp_batch_update_vectors(h, int(i), *[_ptr(a) for a in arrs]),
           "osqp_batch_update_vectors")


def osqp_batch_get(h, i, n, m):
    x, y, z = np.empty(n), np.empty(m), np.empty(m)
    info = osqp_info()
    _check(lib().osqp_batch_get(h, int(i), _ptr(x), _ptr(y), _ptr(z), C.byref(info)),
           "osqp_batch_get")
    return x, y, z, info


def osqp_batch_cleanup(h):
    if h:
        _check(lib().osqp_batch_cleanup(h), "osqp_batch_cleanup")


def osqp_batch_launch(h, slot, idx, q=None, l=None, u=None):
    """idx: problem indices; q/l/u: None or one host array (or None) per problem."""
    a = np.ascontiguousarray(idx, np.int32)
    keep = [a]

    def ptrs(vs):
        if vs is None:
            return None
        arr = (C.c_void_p * len(vs))()
        for j, v in enumerate(vs):
            if v is None:
                arr[j] = None
            elif isinstance(v, int):
                arr[j] = v
            else:
                vv = np.ascontiguousarray(v, np.float64)
                keep.append(vv)
                arr[j] = _ptr(vv)
        keep.append(arr)
        return C.cast(arr, C.c_void_p)

    rc = lib().osqp_batch_launch(h, int(slot), _ptr(a), int(a.size), ptrs(q), ptrs(l), ptrs(u))
    _check(rc, "osqp_batch_launch")


def osqp_batch_slot_query(h, slot) -> bool:
    rc = lib().osqp_batch_slot_query(h, int(slot))
    if rc < 0:
        _check(rc, "osqp_batch_slot_query")
    return rc == 1


def osqp_batch_slot_wait(h, slot):
    _check(lib().osqp_batch_slot_wait(h, int(slot)), "osqp_batch_slot_wait")


def osqp_batch_uses_cluster(h, i) -> bool:
    v = lib().osqp_batch_uses_cluster(h, int(i))
    if v < 0:
        _check(int(v), "osqp_batch_uses_cluster")
    return bool(v)


def osqp_batch_footprint(h, i) -> int:
    v = lib().osqp_batch_footprint(h, int(i))
    if v < 0:
        _check(int(v), "osqp_batch_footprint")
    return int(v)


def osqp_batch_schedule(h, i):
    g = np.zeros(2, np.int32)
    _check(lib().osqp_batch_schedule(h, int(i), _ptr(g)), "osqp_batch_schedule")
    return int(g[0]), int(g[1])


def osqp_batch_tuning(h):
    """The autotuner's classes: list of (kind, rows bucket, mean bucket,
    longest-row bucket, representative, chosen G, cycles of G = 1…32)."""
    n = lib().osqp_batch_tuning(h, 0, None, None)
    if n < 0:
        _check(n, "osqp_batch_tuning")
    info = np.zeros(6 * max(n, 1), np.int32)
    cyc = np.zeros(6 * max(n, 1))
    lib().osqp_batch_tuning(h, n, _ptr(info), _ptr(cyc))
    return [tuple(int(v) for v in info[6 * k:6 * k + 6]) + (cyc[6 * k:6 * k + 6].copy(),)
            for k in range(n)]


def osqp_batch_update_all(h, q_all=None, l_all=None, u_all=None):
    """Concatenated q (Σn), l and u (Σm) of every problem: numpy arrays or
    host addresses (ints, e.g. pinned tensors)."""
    arrs = [None if v is None or isinstance(v, int) else np.ascontiguousarray(v, np.float64)
            for v in (q_all, l_all, u_all)]
    ptrs = [v if isinstance(v, int) else _ptr(a) for v, a in zip((q_all, l_all, u_all), arrs)]
    _check(lib().osqp_batch_update_all(h, *ptrs), "osqp_batch_update_all")


def osqp_batch_get_all(h, x_all, y_all):
    """Fill host arrays (numpy, or int addresses) with every problem's x, y."""
    _check(lib().osqp_batch_get_all(h, x_all if isinstance(x_all, int) else _ptr(x_all),
                                    y_all if isinstance(y_all, int) else _ptr(y_all)),
           "osqp_batch_get_all")


def osqp_diag_schedule(h):
    """(G of Kn, G of Ā, tuned flag, ms per candidate of Kn (6), of Ā (6))."""
    g = np.zeros(3, np.int32)
    ms = np.zeros(12)
    _check(lib().osqp_diag_schedule(h, _ptr(g), _ptr(ms)), "osqp_diag_schedule")
    return int(g[0]), int(g[1]), int(g[2]), ms[:6].copy(), ms[6:].copy()

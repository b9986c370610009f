"""ctypes wrapper of the FP64 CPU oracle — TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this module.  It shares no code with the CUDA
path (``paper_1711_08013_gb300``) and never imports it.

``build()`` compiles ``osqp_oracle.cpp`` with the host C++ compiler into
``oracle/_build/liboracle.so``; ``solve(qp, **settings)`` runs the oracle on a
``problems.QP``-like object (attributes P (upper CSC), q, A (CSC), l, u).
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "osqp_oracle.cpp")
LIB = os.path.join(HERE, "_build", "liboracle.so")

SOLVED, MAX_ITER, PRIMAL_INFEASIBLE, DUAL_INFEASIBLE, NUMERICAL_ERROR = 1, 2, 3, 4, 6

_lock = threading.Lock()
_lib = None


class Settings(C.Structure):
    _fields_ = [
        ("rho", C.c_double), ("sigma", C.c_double), ("alpha", C.c_double),
        ("eps_abs", C.c_double), ("eps_rel", C.c_double),
        ("eps_pinf", C.c_double), ("eps_dinf", C.c_double),
        ("adaptive_rho_tolerance", C.c_double), ("eps_equil", C.c_double),
        ("max_iter", C.c_int), ("check_interval", C.c_int), ("adaptive_rho", C.c_int),
        ("scaling_iters", C.c_int), ("max_rho_updates", C.c_int), ("warm_start", C.c_int),
        ("polish", C.c_int), ("polish_refine_iter", C.c_int), ("delta", C.c_double),
    ]


class Info(C.Structure):
    _fields_ = [
        ("status", C.c_int), ("iter", C.c_int), ("rho_updates", C.c_int), ("ruiz_passes", C.c_int),
        ("obj_val", C.c_double), ("prim_res", C.c_double), ("dual_res", C.c_double),
        ("rho_bar", C.c_double), ("setup_time", C.c_double), ("solve_time", C.c_double),
        ("nnz_L", C.c_longlong), ("polished", C.c_int), ("pad", C.c_int),
    ]


# Defaults of §5.2 and §7; check_interval 25 and the Ruiz cap are readings.
DEFAULTS = dict(rho=0.1, sigma=1e-6, alpha=1.6, eps_abs=1e-3, eps_rel=1e-3, eps_pinf=1e-4,
                eps_dinf=1e-4, adaptive_rho_tolerance=5.0, eps_equil=1e-3, max_iter=4000,
                check_interval=25, adaptive_rho=1, scaling_iters=10, max_rho_updates=20,
                warm_start=0, polish=0, polish_refine_iter=3, delta=1e-6)


def build(force: bool = False) -> str:
    """Compile the oracle library (host C++ compiler, no CUDA)."""
    with _lock:
        if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
                os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "osqp_oracle.h"))):
            return LIB
        os.makedirs(os.path.dirname(LIB), exist_ok=True)
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [os.environ.get("CXX", "g++"), "-O2", "-std=c++17", "-shared", "-fPIC",
               "-o", tmp, SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
        return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        L.oracle_solve.restype = C.c_int
        L.oracle_solve.argtypes = [C.c_int, C.c_int, ip, ip, dp, dp, ip, ip, dp, dp, dp,
                                   C.POINTER(Settings), dp, dp, dp, dp, dp, C.POINTER(Info)]
        L.oracle_ruiz.restype = C.c_int
        L.oracle_ruiz.argtypes = [C.c_int, C.c_int, ip, ip, dp, dp, ip, ip, dp, dp, dp, C.c_int,
                                  C.c_double, dp, dp, C.POINTER(C.c_double), dp, dp, dp, dp, dp]
        L.oracle_min_degree.restype = C.c_int
        L.oracle_min_degree.argtypes = [C.c_int, ip, ip, ip]
        L.oracle_ldl_solve.restype = C.c_longlong
        L.oracle_ldl_solve.argtypes = [C.c_int, ip, ip, dp, C.c_int, dp, dp, dp]
        _lib = L
    return _lib


@dataclasses.dataclass
class Result:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    prim_cert: np.ndarray
    dual_cert: np.ndarray
    status: int
    iter: int
    rho_updates: int
    obj_val: float
    prim_res: float
    dual_res: float
    rho_bar: float
    setup_time: float
    solve_time: float
    nnz_L: int
    ruiz_passes: int
    polished: int = 0


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def solve(qp, x0=None, y0=None, **overrides) -> Result:
    """Run the oracle; keyword arguments override DEFAULTS."""
    s = dict(DEFAULTS)
    s.update(overrides)
    if x0 is not None or y0 is not None:
        s["warm_start"] = 1
    st = Settings(**s)
    n, m = qp.P.shape[0], qp.A.shape[0]
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    y = np.zeros(m) if y0 is None else _f64(y0).copy()
    z = np.zeros(m)
    pc = np.zeros(m)
    dc = np.zeros(n)
    info = Info()
    rc = lib().oracle_solve(n, m, _i32(qp.P.indptr), _i32(qp.P.indices), _f64(qp.P.data),
                            _f64(qp.q), _i32(qp.A.indptr), _i32(qp.A.indices), _f64(qp.A.data),
                            _f64(qp.l), _f64(qp.u), C.byref(st), x, y, z, pc, dc, C.byref(info))
    if rc != 0:
        raise ValueError(f"oracle_solve rejected the problem (code {rc})")
    return Result(x, y, z, pc, dc, info.status, info.iter, info.rho_updates, info.obj_val,
                  info.prim_res, info.dual_res, info.rho_bar, info.setup_time, info.solve_time,
                  int(info.nnz_L), info.ruiz_passes, info.polished)


def ruiz(Pfull, q, A, l, u, scaling_iters=10, eps_equil=1e-3):
    """Alg. 2 alone on full symmetric P (CSC) and A (CSC)."""
    n, m = Pfull.shape[0], A.shape[0]
    D, E = np.zeros(n), np.zeros(m)
    c = C.c_double(0.0)
    Pb, qb, Ab = np.zeros(Pfull.nnz), np.zeros(n), np.zeros(A.nnz)
    lb, ub = np.zeros(m), np.zeros(m)
    passes = lib().oracle_ruiz(n, m, _i32(Pfull.indptr), _i32(Pfull.indices), _f64(Pfull.data),
                               _f64(q), _i32(A.indptr), _i32(A.indices), _f64(A.data), _f64(l),
                               _f64(u), scaling_iters, eps_equil, D, E, C.byref(c), Pb, qb, Ab,
                               lb, ub)
    return dict(D=D, E=E, c=c.value, P_x=Pb, q=qb, A_x=Ab, l=lb, u=ub, passes=passes)


def min_degree(K) -> np.ndarray:
    """Minimum-degree ordering of the symmetric pattern of K (CSC)."""
    N = K.shape[0]
    perm = np.zeros(N, np.int32)
    lib().oracle_min_degree(N, _i32(K.indptr), _i32(K.indices), perm)
    return perm


def ldl_solve(K_upper, g):
    """Solve K t = g through the oracle's LDLᵀ; g is (N,) or (N, r)."""
    N = K_upper.shape[0]
    G = np.asarray(g, np.float64)
    one = G.ndim == 1
    G2 = G.reshape(N, -1)
    r = G2.shape[1]
    gcols = _f64(G2.T.copy())
    t = np.zeros_like(gcols)
    D = np.zeros(N)
    nnzL = lib().oracle_ldl_solve(N, _i32(K_upper.indptr), _i32(K_upper.indices),
                                  _f64(K_upper.data), r, gcols, t, D)
    if nnzL < 0:
        raise ValueError(f"oracle_ldl_solve failed ({nnzL})")
    T = t.reshape(r, N).T
    return (T[:, 0] if one else T), D, int(nnzL)

"""osqp_solve_noalloc — the entry point for callers that cannot allocate.

Code inside a CUDA-graph capture, plugins whose host framework owns all
device memory, and real-time loops that forbid cudaMalloc/cudaFree after
start-up cannot use osqp_setup, which allocates the solver's device memory.
osqp_solve_noalloc solves one small QP with every work array inside a fixed,
statically allocated device buffer.  These tests call it through the C ABI
and check it against the allocating entry points on two calls in a row, and
replay it from a CUDA graph on inputs rewritten between replays.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1711_08013_gb300 import _binding as B
from paper_1711_08013_gb300 import problems as pb

_P = C.c_void_p


def noalloc_fn():
    f = B.lib().osqp_solve_noalloc
    f.restype = C.c_int32
    f.argtypes = [C.c_int32, C.c_int32, _P, _P, _P, C.c_int32, _P, _P, _P, _P, C.c_int32, _P, _P,
                  C.POINTER(B.osqp_settings), _P, _P, C.POINTER(B.osqp_info), _P]
    return f


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """The size check runs on the host before any device work: a problem
    needing more than the 16 MiB work array is refused with OSQP_ERR_LIMIT."""
    st = B.osqp_set_default_settings()
    info = B.osqp_info()
    fake = 256  # never dereferenced: the call returns before touching memory
    rc = noalloc_fn()(2_000_000, 2_000_000, fake, fake, fake, 4_000_000, fake, fake, fake, fake,
                      8_000_000, fake, fake, C.byref(st), fake, fake, C.byref(info), None)
    assert rc == B.OSQP_ERR_LIMIT


def _device_inputs(torch, qp):
    dev = torch.device("cuda", 0)
    t = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    return dict(Pp=t(qp.P.indptr, torch.int32), Pi=t(qp.P.indices, torch.int32),
                Px=t(qp.P.data, torch.float64), q=t(qp.q, torch.float64),
                Ap=t(qp.A.indptr, torch.int32), Ai=t(qp.A.indices, torch.int32),
                Ax=t(qp.A.data, torch.float64), l=t(qp.l, torch.float64),
                u=t(qp.u, torch.float64))


def _call(torch, f, qp, d, st, x, y):
    info = B.osqp_info()
    x.fill_(float("nan"))
    y.fill_(float("nan"))
    rc = f(qp.n, qp.m, d["Pp"].data_ptr(), d["Pi"].data_ptr(), d["Px"].data_ptr(), qp.P.nnz,
           d["q"].data_ptr(), d["Ap"].data_ptr(), d["Ai"].data_ptr(), d["Ax"].data_ptr(),
           qp.A.nnz, d["l"].data_ptr(), d["u"].data_ptr(), C.byref(st), x.data_ptr(),
           y.data_ptr(), C.byref(info), None)
    torch.cuda.synchronize()
    return rc, info, x.cpu().numpy().copy(), y.cpu().numpy().copy()


# The same exact-solve settings as the iterate-parity tests: fixed ρ, a fixed
# number of iterations and PCG run to 1e-14·‖rhs‖∞.
STEP = dict(adaptive_rho=0, eps_abs=0.0, eps_rel=0.0, eps_pinf=1e-300, eps_dinf=1e-300,
            pcg_tol_fraction=0.0, pcg_tol_floor=1e-14, pcg_max_iter=2000, check_interval=1,
            max_iter=40)


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))


@pytest.mark.gpu
@pytest.mark.parametrize("name,make,kw", [
    ("random_qp_exact", lambda: pb.random_qp(40, 160, seed=21), STEP),
    ("portfolio_exact", lambda: pb.portfolio(3, seed=22), STEP),          # long rows
    ("mpc_default", lambda: pb.mpc(6, 8, seed=23), {}),
    ("lasso_fp32_default", lambda: pb.lasso(4, seed=24), dict(precision=B.FP32_MIXED)),
])
def test_noalloc_matches_allocating_entry_point_twice(name, make, kw):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_08013_gb300.solver import Solver
    torch.cuda.set_device(0)
    qp = make()
    with Solver(qp, launch=1, **kw) as s:
        ref = s.solve()
    d = _device_inputs(torch, qp)
    x = torch.empty(qp.n, dtype=torch.float64, device="cuda")
    y = torch.empty(qp.m, dtype=torch.float64, device="cuda")
    st = B.osqp_set_default_settings(launch=1, **kw)
    f = noalloc_fn()
    for call in range(2):
        rc, info, xg, yg = _call(torch, f, qp, d, st, x, y)
        assert rc == B.OSQP_OK, (name, call, rc)
        assert info.status == ref.status and info.iter == ref.iter, (name, call)
        assert _rel(xg, ref.x) <= 1e-8, (name, call, _rel(xg, ref.x))
        assert _rel(yg, ref.y) <= 1e-8, (name, call, _rel(yg, ref.y))
        assert abs(info.obj_val - ref.obj_val) <= 1e-8 * max(1.0, abs(ref.obj_val))


def get_info_fn():
    f = B.lib().osqp_noalloc_get_info
    f.restype = C.c_int32
    f.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(B.osqp_info), _P]
    return f


def test_noalloc_get_info_rejects_bad_arguments():
    """Argument checks of the status read-back run on the host before any
    device call."""
    f = get_info_fn()
    info = B.osqp_info()
    assert f(10, 5, 3, 4, B.FP64, None, None) == B.OSQP_ERR_ARG
    assert f(0, 5, 3, 4, B.FP64, C.byref(info), None) == B.OSQP_ERR_DIMS
    assert f(10, -1, 3, 4, B.FP64, C.byref(info), None) == B.OSQP_ERR_DIMS
    assert f(10, 5, 3, 4, 7, C.byref(info), None) == B.OSQP_ERR_SETTINGS


@pytest.mark.gpu
def test_noalloc_captured_in_cuda_graph_replays_a_control_loop():
    """Captured once in a CUDA graph, the solve replays on inputs rewritten in
    place between replays (q, l and u perturbed as a receding-horizon loop
    does): each replay equals an uncaptured call on the same buffers, and
    osqp_noalloc_get_info reports the replay's status and iterations."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    qp = pb.mpc(6, 8, seed=23)
    d = _device_inputs(torch, qp)
    x = torch.empty(qp.n, dtype=torch.float64, device="cuda")
    y = torch.empty(qp.m, dtype=torch.float64, device="cuda")
    st = B.osqp_set_default_settings(launch=1)
    f, gi = noalloc_fn(), get_info_fn()
    rc, _, _, _ = _call(torch, f, qp, d, st, x, y)  # first call: before any capture
    assert rc == B.OSQP_OK
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        rc = f(qp.n, qp.m, d["Pp"].data_ptr(), d["Pi"].data_ptr(), d["Px"].data_ptr(), qp.P.nnz,
               d["q"].data_ptr(), d["Ap"].data_ptr(), d["Ai"].data_ptr(), d["Ax"].data_ptr(),
               qp.A.nnz, d["l"].data_ptr(), d["u"].data_ptr(), C.byref(st), x.data_ptr(),
               y.data_ptr(), None, stream.cuda_stream)
    assert rc == B.OSQP_OK
    rng = np.random.default_rng(5)
    for step in range(3):
        q2, l2, u2 = pb.perturb_vectors(rng, qp)
        for key, v in (("q", q2), ("l", l2), ("u", u2)):
            d[key].copy_(torch.from_numpy(np.ascontiguousarray(v)))
        x.fill_(float("nan"))
        y.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        xg, yg = x.cpu().numpy().copy(), y.cpu().numpy().copy()
        info = B.osqp_info()
        assert gi(qp.n, qp.m, qp.P.nnz, qp.A.nnz, B.FP64, C.byref(info), None) == B.OSQP_OK
        rc, ref, xr, yr = _call(torch, f, qp, d, st, x, y)
        assert rc == B.OSQP_OK and ref.status == B.SOLVED
        assert info.status == ref.status and info.iter == ref.iter, (step, info.iter, ref.iter)
        assert _rel(xg, xr) <= 1e-12 and _rel(yg, yr) <= 1e-12, step


def _raw_call(torch, f, n, m, Pp, Pi, Px, q, Ap, Ai, Ax, l, u, st):
    """One call on device copies of raw CSC arrays (buffer sizes always match
    the stated n, m and nonzero counts, so a rejected input is only ever
    malformed in its contents)."""
    dev = torch.device("cuda", 0)
    ti = lambda a: torch.tensor(np.asarray(a, dtype=np.int32), device=dev)
    tf = lambda a: torch.tensor(np.asarray(a, dtype=np.float64), device=dev)
    d = [ti(Pp), ti(Pi), tf(Px), tf(q), ti(Ap), ti(Ai), tf(Ax), tf(l), tf(u)]
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    y = torch.zeros(max(m, 1), dtype=torch.float64, device=dev)
    info = B.osqp_info()
    rc = f(n, m, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), len(Px), d[3].data_ptr(),
           d[4].data_ptr(), d[5].data_ptr(), d[6].data_ptr(), len(Ax), d[7].data_ptr(),
           d[8].data_ptr(), C.byref(st), x.data_ptr(), y.data_ptr(), C.byref(info), None)
    torch.cuda.synchronize()
    return rc


def _bad_inputs():
    eye4 = dict(Pp=[0, 1, 2, 3, 4], Pi=[0, 1, 2, 3], Px=[1.0, 1.0, 1.0, 1.0])
    a4 = dict(Ap=[0, 1, 2, 3, 4], Ai=[0, 0, 1, 1], Ax=[1.0, 1.0, 1.0, 1.0])
    base = dict(n=4, m=2, q=[1.0, -1.0, 0.5, 0.0], l=[-1.0, -1.0], u=[1.0, 1.0], **eye4, **a4)
    cases = []
    cases.append(("colptr_decreasing", dict(base, Pp=[0, 2, 1, 3, 4]), B.OSQP_ERR_CSC))
    cases.append(("lower_triangle_in_P", dict(base, Pp=[0, 2, 3, 4, 4], Pi=[0, 1, 1, 2]),
                  B.OSQP_ERR_CSC))
    cases.append(("unsorted_A_column", dict(base, Ap=[0, 2, 2, 3, 4], Ai=[1, 0, 1, 1]),
                  B.OSQP_ERR_CSC))
    cases.append(("nan_in_q", dict(base, q=[1.0, float("nan"), 0.0, 0.0]), B.OSQP_ERR_NONFINITE))
    cases.append(("inf_in_A", dict(base, Ax=[1.0, float("inf"), 1.0, 1.0]), B.OSQP_ERR_NONFINITE))
    cases.append(("nan_bound", dict(base, u=[1.0, float("nan")]), B.OSQP_ERR_NONFINITE))
    cases.append(("l_above_u", dict(base, l=[-1.0, 2.0]), B.OSQP_ERR_LGTU))
    # one A row of 8193 entries (above the 8192-entry row limit)
    n = 8193
    cases.append(("long_A_row", dict(n=n, m=1, Pp=list(range(n + 1)), Pi=list(range(n)),
                                     Px=[1.0] * n, q=[0.0] * n, Ap=list(range(n + 1)),
                                     Ai=[0] * n, Ax=[1.0] * n, l=[-1.0], u=[1.0]),
                  B.OSQP_ERR_LIMIT))
    # a P row of 8193 entries in the full symmetric matrix (row 0 dense)
    Pp, Pi = [0, 1], [0]
    for j in range(1, n):
        Pi += [0, j]
        Pp.append(len(Pi))
    cases.append(("long_P_row", dict(n=n, m=0, Pp=Pp, Pi=Pi, Px=[1e-3] * len(Pi), q=[0.0] * n,
                                     Ap=[0] * (n + 1), Ai=[], Ax=[], l=[], u=[]),
                  B.OSQP_ERR_LIMIT))
    return cases


BAD = _bad_inputs()


@pytest.mark.gpu
def test_noalloc_rejects_bad_inputs_on_the_device_then_recovers():
    """The input checks of osqp_setup run inside the kernel here: malformed
    CSC, non-finite values, l > u and rows beyond the 8192-entry limit each
    give their error code from the call and again from
    osqp_noalloc_get_info, and a valid solve in the same array afterwards
    still equals the allocating entry point's."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    f, gi = noalloc_fn(), get_info_fn()
    st = B.osqp_set_default_settings(launch=1)
    for name, c, want in BAD:
        rc = _raw_call(torch, f, c["n"], c["m"], c["Pp"], c["Pi"], c["Px"], c["q"], c["Ap"],
                       c["Ai"], c["Ax"], c["l"], c["u"], st)
        assert rc == want, (name, rc)
        info = B.osqp_info()
        rc2 = gi(c["n"], c["m"], len(c["Px"]), len(c["Ax"]), B.FP64, C.byref(info), None)
        assert rc2 == want, (name, rc2)
    from paper_1711_08013_gb300.solver import Solver
    qp = pb.random_qp(30, 90, seed=31)
    with Solver(qp, launch=1) as s:
        ref = s.solve()
    d = _device_inputs(torch, qp)
    x = torch.empty(qp.n, dtype=torch.float64, device="cuda")
    y = torch.empty(qp.m, dtype=torch.float64, device="cuda")
    rc, info, xg, yg = _call(torch, f, qp, d, st, x, y)
    assert rc == B.OSQP_OK and info.status == ref.status and info.iter == ref.iter
    assert _rel(xg, ref.x) <= 1e-8 and _rel(yg, ref.y) <= 1e-8

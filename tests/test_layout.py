"""The sliced sparse layout built on the host for every matrix (no GPU),
checked through osqp_diag_sliced_layout against its stated contract: every
CSR entry gets its own position; a short row's nonzeros sit at
first + 32·step + lane on its G lanes in CSR order; slices hold rows sorted
by decreasing length, stable in the row index; long rows follow in CSR
order, cut into chunks of at most 256 positions that cover them exactly."""
import ctypes as C

import numpy as np
import pytest

from paper_1711_08013_gb300 import _binding as B
from paper_1711_08013_gb300 import build as BLD

_P = C.c_void_p


@pytest.fixture(scope="module")
def layout():
    BLD.build()
    f = B.lib().osqp_diag_sliced_layout
    f.restype = C.c_int32
    f.argtypes = [C.c_int32, _P, C.c_int64, _P, _P, _P]

    def run(lengths, nwarps):
        rp = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int32)
        nnz = int(rp[-1])
        stats = np.zeros(6, dtype=np.int32)
        assert f(len(lengths), rp.ctypes.data, nwarps, None, None, stats.ctypes.data) == 0
        pos = np.full(max(nnz, 1), -7, dtype=np.int32)
        chunks = np.zeros(4 * max(int(stats[5]), 1), dtype=np.int32)
        assert f(len(lengths), rp.ctypes.data, nwarps, pos.ctypes.data, chunks.ctypes.data,
                 stats.ctypes.data) == 0
        return rp, pos[:nnz], chunks[:4 * int(stats[5])].reshape(-1, 4), stats
    return run


def _lengths(rng, kind, nrows):
    if kind == "uniform":
        return rng.integers(0, 12, nrows)
    if kind == "skewed":          # a few very long rows among short ones
        v = rng.integers(1, 6, nrows)
        v[rng.choice(nrows, 3, replace=False)] = [700, 300, 1500]
        return v
    if kind == "empty_rows":
        v = rng.integers(0, 40, nrows)
        v[::3] = 0
        return v
    return np.full(nrows, 64)      # "dense": equal rows


@pytest.mark.parametrize("kind", ["uniform", "skewed", "empty_rows", "dense"])
@pytest.mark.parametrize("nwarps", [16, 152 * 16])
def test_layout_contract(layout, kind, nwarps):
    rng = np.random.default_rng(abs(hash((kind, nwarps))) % 2**32)
    nrows = 700
    lengths = _lengths(rng, kind, nrows)
    rp, pos, chunks, stats = layout(lengths, nwarps)
    G, thresh, nslices, npos, nlong, nchunks = (int(v) for v in stats)
    nnz = int(rp[-1])
    assert G in (1, 2, 4, 8, 16, 32)
    assert thresh == max(256, 8 * int(np.ceil(nnz / nrows)))
    # every entry has its own position
    assert np.all((pos >= 0) & (pos < npos)) and len(np.unique(pos)) == nnz
    long_rows = [r for r in range(nrows) if lengths[r] > thresh]
    short_rows = [r for r in range(nrows) if lengths[r] <= thresh]
    assert nlong == len(long_rows)
    # short rows: sorted by decreasing length, stable in the row index
    order = sorted(short_rows, key=lambda r: (-lengths[r], r))
    spw = 32 // G
    assert nslices == (len(order) + spw - 1) // spw
    firsts = []
    for sl in range(nslices):
        rows = order[sl * spw:(sl + 1) * spw]
        first = None
        for loc, r in enumerate(rows):
            for j in range(lengths[r]):
                p = int(pos[rp[r] + j])
                if first is None:
                    first = p - (loc * G + j % G) - 32 * (j // G)
                assert p == first + 32 * (j // G) + loc * G + j % G, (sl, r, j)
        if first is not None:
            assert first % 32 == 0
            firsts.append(first)
    assert firsts == sorted(firsts)
    # long rows: after the slices, in CSR order, contiguous, chunked exactly
    end_short = max((int(pos[rp[r] + j]) for r in short_rows for j in range(lengths[r])), default=-1)
    expect = []
    nxt = None
    for r in long_rows:
        p0 = int(pos[rp[r]])
        assert p0 > end_short and (nxt is None or p0 == nxt)
        assert np.array_equal(pos[rp[r]:rp[r + 1]], np.arange(p0, p0 + lengths[r]))
        nxt = p0 + int(lengths[r])
        for b in range(0, int(lengths[r]), 256):
            expect.append((r, p0 + b, p0 + min(b + 256, int(lengths[r])), 1 if b == 0 else 0))
    assert nchunks == len(expect)
    assert [tuple(int(v) for v in c) for c in chunks] == expect
    # padding stays small for the length-sorted slices
    assert npos - nnz <= 0.5 * nnz + 32 * 32


def test_group_width_follows_row_statistics(layout):
    """Short rows share a warp on G lanes (a power of two): one lane per row
    when rows are short and many, a whole warp per row when they are long
    and few.  Otherwise as many lanes as the warps can give every row, but
    at least enough to cap a lane at 16 nonzeros of a mean row (40 rows of
    200 on 16 warps: occupancy allows 8, the cap needs 16), and never more
    than the next power of two of the mean row length."""
    _, _, _, s_short = layout(np.full(5000, 3), 16)
    _, _, _, s_long = layout(np.full(10, 200), 16)
    _, _, _, s_occ = layout(np.full(40, 200), 16)
    assert s_short[0] == 1
    assert s_long[0] == 32
    assert s_occ[0] == 16
    for n_nz in (5, 17, 33):
        _, _, _, s = layout(np.full(30, n_nz), 152 * 16)
        assert s[0] <= 1 << int(np.ceil(np.log2(n_nz)))


def test_rejects_bad_row_pointers(layout):
    f = B.lib().osqp_diag_sliced_layout
    stats = np.zeros(6, dtype=np.int32)
    bad = np.array([0, 3, 2], dtype=np.int32)
    assert f(2, bad.ctypes.data, 16, None, None, stats.ctypes.data) == B.OSQP_ERR_CSC
    off = np.array([1, 3], dtype=np.int32)
    assert f(1, off.ctypes.data, 16, None, None, stats.ctypes.data) == B.OSQP_ERR_CSC
    ok = np.array([0, 1], dtype=np.int32)
    assert f(1, ok.ctypes.data, 0, None, None, stats.ctypes.data) == B.OSQP_ERR_ARG
    assert f(1, ok.ctypes.data, 16, None, None, None) == B.OSQP_ERR_ARG


def test_degenerate_matrices(layout):
    """No rows, and rows without nonzeros: no positions, no long rows; empty
    rows still take their place in a slice (their product writes a zero)."""
    _, pos, chunks, st = layout(np.zeros(0, dtype=np.int64), 16)
    assert list(st[2:]) == [0, 0, 0, 0] and pos.size == 0 and chunks.size == 0
    _, pos, chunks, st = layout(np.zeros(40, dtype=np.int64), 16)
    assert st[0] == 1 and st[2] == (40 + 31) // 32 and st[3] == 0 and st[4] == 0

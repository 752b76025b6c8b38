"""The library's host-side preparation (csrc/host_prep.cpp), checked on the CPU
through a test-only shim: the balanced split of rows over a group's CTAs, the
lifting of variable bounds into rows (reading D1's CG_LIFTED), and the
SELL-C-sigma packing, against the CSR it packs.  The kernels rely on this layout:

* rows whose longest matrix row exceeds 64 entries are "long" (warp per row),
  those with 2048 or more are "huge" (CTA per row); the rest are "regular";
* the permutation lists every regular row once, then -1 padding to whole slices
  of 32, and inside each window of 1024 positions orders rows by their summed
  length over both matrices, longest first, ties in row order;
* slice s of matrix k is 32 x w_k(s) column-major, w_k(s) the longest row of
  the slice in that matrix, ptr_k[s] its first element; lane l holds the row in
  slot l, its column indices first, then zeros.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2602_23967_b300", "csrc")
OUT = os.path.join(ROOT, "tests", "_build")
SIGMA, LONG, HUGE = 1024, 64, 2048


@pytest.fixture(scope="module")
def shim():
    os.makedirs(OUT, exist_ok=True)
    lib = os.path.join(OUT, "libhostprep_shim.so")
    srcs = [os.path.join(ROOT, "tests", "host_prep_shim.cpp"), os.path.join(CSRC, "host_prep.cpp")]
    cmd = ["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           "-I", "/usr/local/cuda/include", *srcs, "-o", lib]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = C.CDLL(lib)
    L.shim_build_sell.restype = C.c_int
    return L


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def pack(L, mats, layout=None):
    """Run build_sell on one or two CSR matrices with the same row count
    (layout: (sigma, long_row, huge_row), or None for the defaults)."""
    rps = [np.ascontiguousarray(M.indptr, dtype=np.int32) for M in mats]
    cis = [np.ascontiguousarray(M.indices, dtype=np.int32) for M in mats]
    nrows = mats[0].shape[0]
    two = len(mats) == 2
    args = (C.c_int32(nrows), _p(rps[0], C.c_int32), _p(cis[0], C.c_int32),
            _p(rps[1], C.c_int32) if two else None, _p(cis[1], C.c_int32) if two else None)
    if layout is None:
        L.shim_build_sell(*args)
    else:
        L.shim_build_sell_layout(*args, C.c_int32(layout[0]), C.c_int64(layout[1]), C.c_int64(layout[2]))
    sz = np.zeros(6, dtype=np.int64)
    L.shim_sizes(_p(sz, C.c_int64))
    ns, nl, nh, c0, c1, p1 = (int(v) for v in sz)
    perm = np.zeros(ns * 32, np.int32)
    longs, huges = np.zeros(max(nl, 1), np.int32), np.zeros(max(nh, 1), np.int32)
    ptr0, ptr1 = np.zeros(ns + 1, np.int64), np.zeros(max(p1, 1), np.int64)
    col0, col1 = np.zeros(max(c0, 1), np.int32), np.zeros(max(c1, 1), np.int32)
    L.shim_copy(_p(perm, C.c_int32), _p(longs, C.c_int32), _p(huges, C.c_int32), _p(ptr0, C.c_int64),
                _p(ptr1, C.c_int64), _p(col0, C.c_int32), _p(col1, C.c_int32))
    return dict(nslices=ns, perm=perm, longs=longs[:nl], huges=huges[:nh], ptr=[ptr0, ptr1[: ns + 1]],
                col=[col0[:c0], col1[:c1]])


def random_rows(rng, nrows, ncols, lengths):
    rows = []
    for r, ln in enumerate(lengths):
        cols = np.sort(rng.choice(ncols, size=ln, replace=False))
        rows.append(cols)
    indptr = np.concatenate([[0], np.cumsum([len(c) for c in rows])])
    indices = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    return sp.csr_matrix((np.ones(len(indices)), indices, indptr), shape=(nrows, ncols))


def check_layout(mats, out, SIGMA=SIGMA, LONG=LONG, HUGE=HUGE):
    nrows = mats[0].shape[0]
    lens = np.array([np.diff(M.indptr) for M in mats])        # nmat x nrows
    mx, tot = lens.max(axis=0), lens.sum(axis=0)
    huge = np.flatnonzero(mx >= HUGE)
    long = np.flatnonzero((mx > LONG) & (mx < HUGE))
    regular = np.flatnonzero(mx <= LONG)
    assert sorted(out["huges"].tolist()) == huge.tolist()
    assert sorted(out["longs"].tolist()) == long.tolist()
    perm = out["perm"]
    assert out["nslices"] == (len(regular) + 31) // 32
    live = perm[: len(regular)]
    assert np.all(perm[len(regular):] == -1)
    assert sorted(live.tolist()) == regular.tolist()
    # windows of sigma positions: non-increasing total length, ties in row order
    for w0 in range(0, len(regular), SIGMA):
        win = live[w0: w0 + SIGMA]
        keys = list(zip(-tot[win], win))
        assert keys == sorted(keys)
    for k, M in enumerate(mats):
        ptr, col = out["ptr"][k], out["col"][k]
        assert ptr[0] == 0 and len(col) == ptr[-1]
        for s in range(out["nslices"]):
            slot = perm[32 * s: 32 * s + 32]
            w = max((lens[k][r] for r in slot if r >= 0), default=0)
            assert ptr[s + 1] - ptr[s] == 32 * w
            block = col[ptr[s]: ptr[s + 1]].reshape(w, 32)    # column-major: entry j of lane l at 32 j + l
            for l, r in enumerate(slot):
                got = block[:, l]
                if r < 0:
                    assert np.all(got == 0)
                    continue
                ln = lens[k][r]
                want = M.indices[M.indptr[r]: M.indptr[r + 1]]
                assert np.array_equal(got[:ln], want)
                assert np.all(got[ln:] == 0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sell_packing_one_matrix(shim, seed):
    rng = np.random.default_rng(seed)
    nrows, ncols = 2500, 4000
    lengths = rng.integers(0, 20, nrows)
    lengths[rng.integers(0, nrows)] = 100      # one long row
    lengths[rng.integers(0, nrows)] = 3000     # one huge row
    M = random_rows(rng, nrows, ncols, lengths)
    check_layout([M], pack(shim, [M]))


def test_sell_packing_two_matrices(shim):
    # the variable space packs A^T and Q together: classification by the longer
    # row, ordering by the summed length, one slice geometry per matrix
    rng = np.random.default_rng(7)
    nrows, ncols = 1500, 1500
    l1 = rng.integers(0, 12, nrows)
    l2 = rng.integers(0, 12, nrows)
    l2[5] = 70                                  # long through the second matrix only
    A = random_rows(rng, nrows, ncols, l1)
    Q = random_rows(rng, nrows, ncols, l2)
    check_layout([A, Q], pack(shim, [A, Q]))


def test_sell_packing_tiny_and_empty_rows(shim):
    rng = np.random.default_rng(3)
    for nrows in (1, 31, 32, 33):
        lengths = rng.integers(0, 3, nrows)
        M = random_rows(rng, nrows, 10, lengths)
        check_layout([M], pack(shim, [M]))


@pytest.mark.parametrize("nblk", [1, 3, 7, 64])
def test_split_balanced_ranges(shim, nblk):
    # contiguous ranges, each within one largest item of total / nblk (an item
    # goes to the range that holds the midpoint of its prefix-sum interval)
    rng = np.random.default_rng(nblk)
    w = np.ascontiguousarray((rng.pareto(1.5, 5000) * 10 + 1).astype(np.int64))
    b = np.zeros(nblk + 1, np.int32)
    shim.shim_split_balanced(_p(w, C.c_int64), C.c_int32(len(w)), C.c_int32(nblk), _p(b, C.c_int32))
    assert b[0] == 0 and b[-1] == len(w) and np.all(np.diff(b) >= 0)
    share, wmax = w.sum() / nblk, w.max()
    for k in range(nblk):
        assert abs(w[b[k]: b[k + 1]].sum() - share) <= wmax


def test_lift_box_rows(shim):
    # the CG_LIFTED reading: one row e_j^T per variable with a finite bound, in
    # variable order, carrying that variable's bounds; every variable then free
    from paper_2602_23967_b300 import pdhcg
    rng = np.random.default_rng(4)
    n, m = 12, 5
    A = sp.random(m, n, density=0.4, random_state=rng, format="csr")
    lv = np.where(rng.random(n) < 0.5, -rng.random(n), -np.inf)
    uv = np.where(rng.random(n) < 0.5, rng.random(n) + 1, np.inf)
    lc, uc = -np.ones(m), np.ones(m)
    c = rng.normal(size=n)
    indptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
    indices = np.ascontiguousarray(A.indices, dtype=np.int32)
    data = np.ascontiguousarray(A.data, dtype=np.float64)
    As = pdhcg.Csr(m, n, A.nnz, indptr.ctypes.data, indices.ctypes.data, data.ctypes.data)
    rc = shim.shim_lift(None, C.byref(As), _p(c, C.c_double), _p(lc, C.c_double), _p(uc, C.c_double),
                        _p(lv, C.c_double), _p(uv, C.c_double))
    assert rc == 0
    sz = np.zeros(3, np.int64)
    shim.shim_lift_sizes(_p(sz, C.c_int64))
    m2, nnz2, m_user = (int(v) for v in sz)
    boxed = np.flatnonzero(np.isfinite(lv) | np.isfinite(uv))
    assert m2 == m + len(boxed) and m_user == m and nnz2 == A.nnz + len(boxed)
    Ap, Ac, Av = np.zeros(m2 + 1, np.int32), np.zeros(nnz2, np.int32), np.zeros(nnz2)
    ATp, ATc, ATv = np.zeros(n + 1, np.int32), np.zeros(nnz2, np.int32), np.zeros(nnz2)
    lc2, uc2, lv2, uv2 = np.zeros(m2), np.zeros(m2), np.zeros(n), np.zeros(n)
    vt = np.zeros(n, np.int8)
    shim.shim_lift_copy(_p(Ap, C.c_int32), _p(Ac, C.c_int32), _p(Av, C.c_double), _p(ATp, C.c_int32),
                        _p(ATc, C.c_int32), _p(ATv, C.c_double), _p(lc2, C.c_double), _p(uc2, C.c_double),
                        _p(lv2, C.c_double), _p(uv2, C.c_double), _p(vt, C.c_int8))
    lifted = sp.csr_matrix((Av, Ac, Ap), shape=(m2, n)).toarray()
    expect = np.vstack([A.toarray(), np.eye(n)[boxed]])
    np.testing.assert_array_equal(lifted, expect)
    np.testing.assert_array_equal(sp.csr_matrix((ATv, ATc, ATp), shape=(n, m2)).toarray(), expect.T)
    np.testing.assert_array_equal(lc2, np.concatenate([lc, lv[boxed]]))
    np.testing.assert_array_equal(uc2, np.concatenate([uc, uv[boxed]]))
    assert np.all(np.isneginf(lv2)) and np.all(np.isposinf(uv2)) and np.all(vt == 0)


@pytest.mark.parametrize("layout", [(128, 64, 2048), (8192, 32, 2048), (1024, 16, 200), (32, 128, 8192)])
def test_sell_packing_other_layouts(shim, layout):
    # the layouts the autotuner tries: other sort windows and long / huge thresholds
    rng = np.random.default_rng(11)
    nrows, ncols = 3000, 5000
    lengths = rng.integers(0, 40, nrows)
    lengths[rng.integers(0, nrows, 5)] = rng.integers(100, 400, 5)
    lengths[rng.integers(0, nrows)] = 2500
    M = random_rows(rng, nrows, ncols, lengths)
    sg, lo, hu = layout
    check_layout([M], pack(shim, [M], layout), SIGMA=sg, LONG=lo, HUGE=hu)


def test_autotune_selection_rule(shim):
    shim.shim_pick_fastest.restype = C.c_int

    def pick(ts, margin=0.03):
        a = np.array(ts, dtype=np.float64)
        return shim.shim_pick_fastest(_p(a, C.c_double), C.c_int32(len(a)), C.c_double(margin))

    assert pick([1.0, 0.5, 0.9]) == 1               # a clear winner
    assert pick([1.0, 0.98, 0.99]) == 0             # within the margin: keep the defaults
    assert pick([1.0, 0.96]) == 1                   # 4 % faster beats a 3 % margin
    assert pick([1.0, -1.0, float("nan"), 0.2]) == 3  # failed runs never win
    assert pick([-1.0, 2.0, 1.5]) == 2              # the defaults failed: the fastest that ran
    assert pick([-1.0, float("inf")]) == -1         # nothing ran
    assert pick([0.7]) == 0


@pytest.mark.parametrize("nrows", [1, 31, 32, 33, 1000, 4097])
def test_slice_count_within_the_shared_memory_bound(shim, nrows):
    """A pool CTA keeps each row space's nslices + 1 slice offsets in shared
    memory, budgeted as n/32 + 2 entries (smem_vector_bytes): the packing never
    makes more slices than that, whatever the layout or the share of long rows."""
    rng = np.random.default_rng(nrows)
    lengths = rng.integers(0, 12, size=nrows)
    lengths[rng.random(nrows) < 0.05] = 100  # some long rows (warp-per-row, not in slices)
    M = random_rows(rng, nrows, 200, lengths)
    for layout in (None, (1, 64, 2048), (8192, 16, 64)):
        lay = pack(shim, [M], layout)
        assert lay["nslices"] + 1 <= nrows // 32 + 2, (layout, lay["nslices"])
        assert len(lay["ptr"][0]) == lay["nslices"] + 1

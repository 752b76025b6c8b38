"""C-ABI checks that need no GPU: the library loads, exports every function that
include/pdhcg.h declares, and rejects malformed problems before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2602_23967_b300 import pdhcg
from paper_2602_23967_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(pdhcg_\w+)\s*\(", txt, re.M):
                names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = pdhcg.lib()
    names = declared_functions()
    assert "pdhcg_create" in names and "pdhcg_solve_batch" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_default_params_and_strerror():
    p = pdhcg.default_params()
    assert p.struct_size == C.sizeof(pdhcg.Params)
    assert p.eps_tol == 1e-6 and p.k_eval == 64 and p.theta == 1.0
    assert p.gamma_inner == 5e-4 and p.eps_inner_min == 1e-9
    assert pdhcg.strerror(pdhcg.E_INVALID).startswith("invalid")


def _bad(qp, **kw):
    with pytest.raises(pdhcg.PdhcgError) as ei:
        pdhcg.Problem(qp, pdhcg.default_params(**kw))
    assert ei.value.code == pdhcg.E_INVALID
    return str(ei.value)


def test_rejects_malformed_problems():
    base = W.random_qp(n=20, m=8, n_eq=4, m_rows=5, density=0.3, seed=0)
    qp = W.random_qp(n=20, m=8, n_eq=4, m_rows=5, density=0.3, seed=0)
    qp.lc = qp.lc.copy(); qp.lc[5] = qp.uc[5] + 1.0
    assert "bound" in _bad(qp)
    qp = W.random_qp(n=20, m=8, n_eq=4, m_rows=5, density=0.3, seed=0)
    qp.c = qp.c.copy(); qp.c[0] = np.nan
    assert "c" in _bad(qp)
    qp = W.random_qp(n=20, m=8, n_eq=4, m_rows=5, density=0.3, seed=0)
    Qd = qp.Q.toarray(); Qd[0, 1] += 1.0
    qp.Q = sp.csr_matrix(Qd)
    assert "symmetric" in _bad(qp)
    qp = W.random_qp(n=20, m=8, n_eq=4, m_rows=5, density=0.3, seed=0)
    qp.lv = qp.lv.copy(); qp.lv[3] = np.inf
    assert "bound" in _bad(qp)
    # CG is only valid when every variable is free; DIAG needs a diagonal Q
    assert "CG" in _bad(base, inner="cg")
    assert "DIAG" in _bad(base, inner="diag")


def test_rejects_bad_csr_structure():
    qp = W.random_qp(n=20, m=8, n_eq=4, m_rows=5, density=0.3, seed=1)
    A = qp.A.copy()
    A.indices = A.indices.copy(); A.indices[0] = 25    # column out of range
    qp.A = A
    assert "range" in _bad(qp)


def test_rejects_bad_params():
    qp = W.random_qp(n=20, m=8, n_eq=4, m_rows=5, density=0.3, seed=1)
    p = pdhcg.default_params()
    p.struct_size = 12
    with pytest.raises(pdhcg.PdhcgError):
        pdhcg.Problem(qp, p)
    with pytest.raises(pdhcg.PdhcgError):
        pdhcg.Problem(qp, pdhcg.default_params(k_eval=0))


def test_rejects_malformed_structured_objective():
    # pdhcg_create_qr (Q = P + R^T R, Sec. 2.2) validates R before any device work
    def factored():
        return W.random_qp(n=20, m=8, n_eq=4, m_rows=5, density=0.3, seed=2, factored=True)
    qp = factored()
    R = qp.R.tocsr().copy()
    R.indices = R.indices.copy(); R.indices[0] = qp.n + 3   # column beyond n
    qp.R = R
    assert "range" in _bad(qp)
    qp = factored()
    R = qp.R.tocsr().copy()
    R.data = R.data.copy(); R.data[0] = np.inf
    qp.R = R
    assert "finite" in _bad(qp)
    qp = factored()
    qp.R = sp.csr_matrix((0, qp.n))
    assert "k >= 1" in _bad(qp)
    # R^T R makes Q non-diagonal: the closed-form inner solve does not apply
    assert "DIAG" in _bad(factored(), inner="diag")
    # the batched creation takes plain Q only
    with pytest.raises(ValueError):
        pdhcg.create_batch([factored()], pdhcg.default_params())


def test_empty_batches_and_negative_counts():
    # a batch of zero problems is a no-op for every batched entry point, and a
    # negative count is rejected; neither touches the device
    assert pdhcg.create_batch([], pdhcg.default_params()) == []
    assert pdhcg.solve_batch([]) == []
    assert pdhcg.solve_batch([], want_solutions=False) == []
    assert pdhcg.solve_batch_noalloc([]) == []
    L = pdhcg.lib()
    res = (pdhcg.Result * 1)()
    handles = (C.c_void_p * 1)()
    assert L.pdhcg_solve_batch(handles, -1, res, None, None) == pdhcg.E_INVALID
    assert L.pdhcg_solve_batch_noalloc(handles, -1, res, None, None) == pdhcg.E_INVALID


def test_noalloc_output_checks_reject_bad_buffers():
    # pdhcg_solve_batch_noalloc writes through the raw pointers of the caller's
    # tensors, so the binding rejects every buffer it could overrun before the call
    import collections

    import torch
    from paper_2602_23967_b300 import pdhcg

    P = collections.namedtuple("P", "n m")
    probs = [P(5, 3), P(4, 2)]
    ok_x = [None, None]
    pdhcg.check_noalloc_outputs(probs, ok_x, None)            # None entries are allowed
    bad = [
        ([torch.zeros(5, dtype=torch.float32), None], None, "dtype"),
        ([torch.zeros(10, dtype=torch.float64)[::2], None], None, "contiguous"),
        ([torch.zeros(4, dtype=torch.float64), None], None, "elements"),
        (None, [None, torch.zeros(1, dtype=torch.float64)], "elements"),
        ([torch.zeros(5, dtype=torch.float64), None], None, "CUDA"),
        ([None], None, "entries"),
    ]
    for xo, yo, word in bad:
        with pytest.raises(ValueError, match=word):
            pdhcg.check_noalloc_outputs(probs, xo, yo)

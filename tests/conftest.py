import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: larger CPU cases")


def _have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _have_gpu():
        return
    skip = pytest.mark.skip(reason="no CUDA GPU in this environment")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def golden_closed_form_qps():
    """The hand-derived QPs of tests/golden/closed_form_qps.json as (QP, x*, f*)."""
    import json

    import numpy as np
    import scipy.sparse as sp

    from paper_2602_23967_b300 import workloads as W

    def vec(v, absent):
        return np.array([absent if a is None else a for a in v], dtype=np.float64)

    with open(os.path.join(ROOT, "tests", "golden", "closed_form_qps.json")) as f:
        data = json.load(f)
    out = []
    for p in data["problems"]:
        n = len(p["c"])
        m = len(p["A"])
        Q = sp.csr_matrix(np.array(p["Q"], dtype=np.float64))
        A = sp.csr_matrix(np.array(p["A"], dtype=np.float64).reshape(m, n))
        lc, uc = vec(p["lc"], -np.inf), vec(p["uc"], np.inf)  # null = absent bound
        lv, uv = vec(p["lv"], -np.inf), vec(p["uv"], np.inf)
        qp = W.QP(n, m, Q, A, np.array(p["c"], dtype=np.float64), lc, uc, lv, uv, name=p["name"])
        out.append((qp, np.array(p["x"], dtype=np.float64), float(p["objective"])))
    return out

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


def _frac(v):
    """A fixture number: a float or an exact fraction written as 'p/q'."""
    from fractions import Fraction
    return float(Fraction(v)) if isinstance(v, str) else float(v)


def golden_step_trace():
    """tests/golden/step_trace_1d.json: the one-variable QP, its settings and the
    hand-derived step trace (eps_k and T(z) per step) for each theta."""
    import json

    import numpy as np
    import scipy.sparse as sp

    from paper_2602_23967_b300 import workloads as W

    with open(os.path.join(ROOT, "tests", "golden", "step_trace_1d.json")) as f:
        data = json.load(f)

    def qp_of(p):
        vec = (lambda v, absent: np.array([absent if a is None else _frac(a) for a in v], dtype=np.float64))
        Q = sp.csr_matrix(np.array(p["Q"], dtype=np.float64))
        A = sp.csr_matrix(np.array(p["A"], dtype=np.float64))
        return W.QP(1, 1, Q, A, vec(p["c"], 0.0), vec(p["lc"], -np.inf), vec(p["uc"], np.inf),
                    vec(p["lv"], -np.inf), vec(p["uv"], np.inf), name="step_trace_1d")

    s = data["settings"]
    settings = {k: s[k] for k in ("ruiz_iters", "eta_override", "omega0_override", "gamma_inner",
                                  "eps_inner_min", "eps_inner_first")}
    cases = []
    for c in data["cases"]:
        outs = {int(K): (np.array([_frac(v) for v in o["x"]]), np.array([_frac(v) for v in o["y"]]))
                for K, o in c["outputs_by_max_iter"].items() if K != "note"}
        cases.append({"theta": float(c["theta"]), "eps_trace": np.array([_frac(v) for v in c["eps_trace"]]),
                      "outputs": outs})
    g = data["gap"]
    gap = {"qp": qp_of(g["problem"]), "x": np.array([_frac(v) for v in g["point"]["x"]]),
           "y": np.array([_frac(v) for v in g["point"]["y"]]),
           "expect": {k: _frac(g[k]) for k in ("r_primal", "r_dual", "r_gap", "primal_obj", "dual_obj")}}
    return {"qp": qp_of(data["problem"]), "settings": settings, "x0": np.array(s["x0"], dtype=np.float64),
            "y0": np.array(s["y0"], dtype=np.float64), "cases": cases, "gap": gap}

"""The autotuner (pdhcg_autotune): its choice of row layout and launch shape
changes how the work is laid out, never what is computed.

* A single multi-CTA solve tuned on a mid-size sparse QP: FP64 iterates after
  100 PDHG steps with the chosen settings equal the oracle's to 1e-10, the
  same bar as the defaults; a double-float solve reaches KKT 1e-6 on the
  oracle's evaluator.  A second problem of the same shape class takes the
  cached choice without timing.
* A batch of MPC QPs tuned as a batch: every instance OPTIMAL at KKT 1e-6 on
  the oracle's evaluator, and FP64 iterates of a sample equal the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_2602_23967_b300 import pdhcg
from paper_2602_23967_b300 import workloads as W

pytestmark = pytest.mark.gpu


def kkt_of(qp, x, y):
    Qx = qp.Q @ x if qp.Q is not None else np.zeros(qp.n)
    return oracle.kkt(qp.n, qp.m, x, y, qp.A @ x, qp.A.T @ y, Qx, qp.c, qp.lc, qp.uc, qp.lv, qp.uv)


def test_autotuned_single_solve_matches_oracle():
    qp = W.large_sparse_qp(n=20000, m=10000, seed=0)
    base = pdhcg.default_params()
    tuned, rep = pdhcg.autotune([qp], base)
    assert rep["from_cache"] == 0 and rep["candidates"] >= 5
    assert rep["seconds_per_step"] > 0 and rep["seconds_per_step"] <= rep["default_seconds_per_step"] * 1.10
    for f in ("sell_sigma", "long_row", "huge_row", "group_blocks", "pipeline"):
        assert getattr(tuned, f) == rep[f]
    # same shape class: taken from the cache
    _, rep2 = pdhcg.autotune([W.large_sparse_qp(n=20000, m=10000, seed=1)], base)
    assert rep2["from_cache"] == 1 and rep2["candidates"] == 0
    assert all(rep2[f] == rep[f] for f in ("sell_sigma", "long_row", "huge_row", "group_blocks", "pipeline"))
    N = 100
    tuned.max_iter = N
    p = pdhcg.Problem(qp, tuned)
    try:
        x, y, r = p.solve()
        eta, _ = p.eta()
    finally:
        p.close()
    xo, yo, ro = oracle.solve(qp, oracle.default_params(max_iter=N, eta_override=eta))
    assert r["inner_iterations"] == ro["inner_iterations"]
    assert np.max(np.abs(x - xo)) <= 1e-10 * (1 + np.max(np.abs(xo)))
    assert np.max(np.abs(y - yo)) <= 1e-10 * (1 + np.max(np.abs(yo)))
    tuned.max_iter = 400000
    tuned.precision = pdhcg.PRECISION["dfloat"]
    p = pdhcg.Problem(qp, tuned)
    try:
        x, y, r = p.solve()
    finally:
        p.close()
    assert r["status_name"] == "OPTIMAL", r
    assert max(kkt_of(qp, x, y)[:3]) <= 1e-6


def test_autotuned_batch_matches_oracle():
    qps = W.mpc_batch(count=64, seed=3)
    base = pdhcg.default_params(precision="dfloat", eps_tol=1e-6)
    tuned, rep = pdhcg.autotune(qps, base)
    assert rep["candidates"] >= 2 and rep["seconds_per_step"] > 0
    probs = pdhcg.create_batch(qps, tuned)
    try:
        out = pdhcg.solve_batch(probs)
    finally:
        for p in probs:
            p.close()
    for q, (x, y, r) in zip(qps, out):
        assert r["status_name"] == "OPTIMAL"
        assert max(kkt_of(q, x, y)[:3]) <= 1e-6
    fp64 = pdhcg.default_params(max_iter=100)
    for f in ("sell_sigma", "long_row", "huge_row", "pool_ctas_per_sm"):
        setattr(fp64, f, getattr(tuned, f))
    sample = qps[:4]
    probs = pdhcg.create_batch(sample, fp64)
    try:
        out = pdhcg.solve_batch(probs)
        etas = [p.eta()[0] for p in probs]
    finally:
        for p in probs:
            p.close()
    for q, (x, y, r), eta in zip(sample, out, etas):
        xo, yo, ro = oracle.solve(q, oracle.default_params(max_iter=100, eta_override=eta))
        assert np.max(np.abs(x - xo)) <= 1e-10 * (1 + np.max(np.abs(xo)))
        assert np.max(np.abs(y - yo)) <= 1e-10 * (1 + np.max(np.abs(yo)))

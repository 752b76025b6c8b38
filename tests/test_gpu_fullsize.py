"""Parity at the full sizes of the benchmark workloads, in the launch
configurations the benchmark uses.

* 4,096 MPC QPs in one persistent launch (double-float, as bench.py): every
  instance OPTIMAL; the oracle's independent KKT evaluator (Sec. 4.2) on every
  GPU solution <= 1e-6; objective against the oracle's own solve <= 1e-6 on a
  sample of 16 instances (the oracle takes ~40 ms per instance).
* The large sparse QP (n = 2e6, m = 1e6, power-law column degrees): FP64
  iterates after 3 PDHG steps (BB inner solver, auto multi-CTA group) equal the
  oracle's to 1e-10 relative, with the same number of inner steps; after 64
  steps the double-float and mixed modes (the same FP32 matrix values) agree
  to 1e-8; in the benchmark's configuration (double-float, pipeline form, 64
  steps) the device's residuals equal the oracle's evaluation of its point,
  and the trajectory follows the oracle's.
* The factor-model portfolio QP (n = 1e5 + 1e3 variables, the 1e5-entry budget
  row): FP64 iterates after 20 steps equal the oracle's to 1e-10, and the
  double-float solve at 1e-6 matches the oracle's objective to 1e-6.
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


def rel(a, b):
    return abs(a - b) / (1.0 + abs(b))


def test_mpc_batch_4096_double_float():
    qps = W.mpc_batch(count=4096, seed=0)
    probs = pdhcg.create_batch(qps, pdhcg.default_params(precision="dfloat", eps_tol=1e-6))
    try:
        out = pdhcg.solve_batch(probs, want_solutions=True)
    finally:
        for p in probs:
            p.close()
    worst = 0.0
    for qp, (x, y, r) in zip(qps, out):
        assert r["status_name"] == "OPTIMAL"
        rp, rd, rg, _, _ = kkt_of(qp, x, y)
        worst = max(worst, rp, rd, rg)
    assert worst <= 1e-6, worst
    for i in range(0, 4096, 256):
        x, y, r = out[i]
        _, _, _, pobj, _ = kkt_of(qps[i], x, y)
        _, _, ro = oracle.solve(qps[i], oracle.default_params(eps_tol=1e-6))
        assert rel(pobj, ro["primal_obj"]) <= 1e-6, (i, pobj, ro["primal_obj"])


@pytest.fixture(scope="module")
def large_sparse():
    return W.large_sparse_qp(seed=0)


def solve_n(qp, N, **kw):
    p = pdhcg.Problem(qp, pdhcg.default_params(max_iter=N, **kw))
    try:
        x, y, r = p.solve()
        eta, _ = p.eta()
    finally:
        p.close()
    return x, y, r, eta


def test_large_sparse_fp64_iterates_full_size(large_sparse):
    qp = large_sparse
    N = 3
    x, y, r, eta = solve_n(qp, N)
    xo, yo, ro = oracle.solve(qp, oracle.default_params(max_iter=N, eta_override=eta))
    assert r["iterations"] == ro["iterations"] == N
    assert r["inner_iterations"] == ro["inner_iterations"]
    assert np.max(np.abs(x - xo)) <= 1e-10 * (1 + np.max(np.abs(xo)))
    assert np.max(np.abs(y - yo)) <= 1e-10 * (1 + np.max(np.abs(yo)))


def test_large_sparse_double_float_matches_mixed_full_size(large_sparse):
    qp = large_sparse
    N = 64
    xm, ym, rm, _ = solve_n(qp, N, precision="mixed")
    xd, yd, rd, _ = solve_n(qp, N, precision="dfloat")
    assert rd["inner_iterations"] == rm["inner_iterations"]
    assert np.max(np.abs(xd - xm)) <= 1e-8 * (1 + np.max(np.abs(xm)))
    assert np.max(np.abs(yd - ym)) <= 1e-8 * (1 + np.max(np.abs(ym)))


def test_large_sparse_bench_configuration_full_size(large_sparse):
    # The large-instance leg of bench.py: double-float, the automatic form (the
    # pipeline graph at this size), 64 PDHG steps ending at a check.
    # (a) The residuals and objective the device reports (FP64-accurate checks,
    #     Sec. 4.2) equal the oracle's independent FP64 evaluation of the
    #     returned point.
    # (b) The trajectory is the oracle's: after the same 64 steps (same step
    #     size), objective and residuals agree to 1e-4 (FP32 matrix values,
    #     double-float vectors against FP64 throughout).
    qp = large_sparse
    N = 64
    x, y, r, eta = solve_n(qp, N, precision="dfloat", eps_tol=1e-12)
    assert r["status_name"] == "ITERATION_LIMIT" and r["iterations"] == N, r
    assert r["form"] == 2, r["form"]  # the pipeline graph
    rp, rd, rg, pobj, _ = kkt_of(qp, x, y)
    for dev, host in ((r["r_primal"], rp), (r["r_dual"], rd), (r["r_gap"], rg), (r["primal_obj"], pobj)):
        assert abs(dev - host) <= 1e-9 * (1 + abs(host)), (dev, host)
    _, _, ro = oracle.solve(qp, oracle.default_params(max_iter=N, eta_override=eta))
    assert ro["iterations"] == N
    for key in ("r_primal", "r_dual", "r_gap", "primal_obj"):
        assert abs(r[key] - ro[key]) <= 1e-4 * (1 + abs(ro[key])), (key, r[key], ro[key])


def test_factor_portfolio_full_size():
    qp = W.factor_portfolio(seed=0)
    N = 20
    x, y, r, eta = solve_n(qp, N)
    xo, yo, ro = oracle.solve(qp, oracle.default_params(max_iter=N, eta_override=eta))
    assert np.max(np.abs(x - xo)) <= 1e-10 * (1 + np.max(np.abs(xo)))
    assert np.max(np.abs(y - yo)) <= 1e-10 * (1 + np.max(np.abs(yo)))
    p = pdhcg.Problem(qp, pdhcg.default_params(precision="dfloat", eps_tol=1e-6, time_limit_s=300.0))
    try:
        x, y, r = p.solve()
    finally:
        p.close()
    assert r["status_name"] == "OPTIMAL", r
    rp, rd, rg, pobj, _ = kkt_of(qp, x, y)
    assert max(rp, rd, rg) <= 1e-6
    _, _, ro = oracle.solve(qp, oracle.default_params(eps_tol=1e-6))
    assert ro["status_name"] == "OPTIMAL"
    assert rel(pobj, ro["primal_obj"]) <= 1e-6

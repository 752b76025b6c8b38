"""The pipeline form of pdhcg_solve: one kernel per phase in a CUDA graph with
device-driven conditional nodes (params.pipeline = 1 forces it; large problems
use it by default).

* FP64 iterates after N = 1 .. 100 PDHG steps equal the oracle's to 1e-10,
  with equal inner-step counts, for the BB, CG and closed-form inner solvers;
* double-float solves reach KKT 1e-6 on the oracle's evaluator and the
  oracle's objective;
* the statuses of Sec. 5 (primal and dual infeasibility, with their rays), the
  limits, and a warm start behave as in the persistent kernel.
"""
import numpy as np
import pytest

import oracle
from paper_2602_23967_b300 import pdhcg
from paper_2602_23967_b300 import workloads as W
from certificates import check_dual_ray, check_primal_ray

pytestmark = pytest.mark.gpu


def kkt_of(qp, x, y):
    Qx = qp.Q @ x if qp.Q is not None else np.zeros(qp.n)
    return oracle.kkt(qp.n, qp.m, x, y, qp.A @ x, qp.A.T @ y, Qx, qp.c, qp.lc, qp.uc, qp.lv, qp.uv)


def solve(qp, x0=None, y0=None, **kw):
    p = pdhcg.Problem(qp, pdhcg.default_params(pipeline=1, **kw))
    try:
        x, y, r = p.solve(x0=x0, y0=y0)
        eta, _ = p.eta()
    finally:
        p.close()
    return x, y, r, eta


CASES = {
    "bb_large_sparse": lambda: W.large_sparse_qp(n=6000, m=3000, seed=1),
    "bb_tiny_random": lambda: W.random_qp(seed=4),
    "cg_equality": lambda: W.equality_qp(n=120, m=40, seed=2),
    "diag_portfolio": lambda: W.factor_portfolio(n=20000, k=50, seed=0),
}


@pytest.mark.parametrize("N", [1, 17, 64, 100])
@pytest.mark.parametrize("name", list(CASES))
def test_pipeline_fp64_iterates(name, N):
    qp = CASES[name]()
    x, y, r, eta = solve(qp, max_iter=N)
    xo, yo, ro = oracle.solve(qp, oracle.default_params(max_iter=N, eta_override=eta))
    assert r["iterations"] == ro["iterations"] == N
    assert r["form"] == 2                                   # the pipeline graph ran
    assert r["inner_method"] == ro["inner_method"]
    assert r["inner_iterations"] == ro["inner_iterations"]
    assert np.max(np.abs(x - xo)) <= 1e-10 * (1 + np.max(np.abs(xo)))
    assert np.max(np.abs(y - yo)) <= 1e-10 * (1 + np.max(np.abs(yo)))


@pytest.mark.parametrize("name", ["bb_large_sparse", "diag_portfolio", "cg_equality"])
def test_pipeline_double_float_solves(name):
    qp = CASES[name]()
    x, y, r, _ = solve(qp, precision="dfloat", eps_tol=1e-6, max_iter=400000)
    assert r["status_name"] == "OPTIMAL", r
    rp, rd, rg, pobj, _ = kkt_of(qp, x, y)
    assert max(rp, rd, rg) <= 1e-6
    _, _, ro = oracle.solve(qp, oracle.default_params(eps_tol=1e-6))
    assert abs(pobj - ro["primal_obj"]) <= 1e-6 * (1 + abs(ro["primal_obj"]))


@pytest.mark.parametrize("seed", [0, 1])
def test_pipeline_infeasibility(seed):
    qp = W.infeasible_qp(n=8, m=4, seed=seed)
    x, y, r, _ = solve(qp)
    assert r["status_name"] == "PRIMAL_INFEASIBLE"
    assert np.max(np.abs(y)) == pytest.approx(1.0)
    check_primal_ray(qp, y)   # the whole certificate of Sec. 5.1
    qp = W.unbounded_qp(n=6, seed=seed)
    x, y, r, _ = solve(qp)
    assert r["status_name"] == "DUAL_INFEASIBLE"
    check_dual_ray(qp, x)     # the whole certificate of Sec. 5.2


def test_pipeline_limits_and_warm_start():
    qp = W.large_sparse_qp(n=20000, m=10000, seed=0)
    x, y, r, _ = solve(qp, precision="dfloat", eps_tol=1e-12, time_limit_s=1e-3)
    assert r["status_name"] == "TIME_LIMIT" and r["iterations"] % 64 == 0
    qp = W.random_qp(seed=9)
    x, y, r, _ = solve(qp, eps_tol=1e-7)
    assert r["status_name"] == "OPTIMAL"
    x2, y2, r2, _ = solve(qp, x0=x, y0=y, eps_tol=1e-7)
    assert r2["status_name"] == "OPTIMAL" and r2["iterations"] <= r["iterations"]


def test_pipeline_and_persistent_kernel_agree():
    # the same problem through both forms: same decisions, iterates equal to rounding
    qp = W.large_sparse_qp(n=6000, m=3000, seed=2)
    xp, yp, rp, _ = solve(qp, max_iter=200)
    p = pdhcg.Problem(qp, pdhcg.default_params(pipeline=-1, max_iter=200, group_blocks=16))
    try:
        xg, yg, rg = p.solve()
    finally:
        p.close()
    assert rp["form"] == 2 and rg["form"] == 1
    assert rp["inner_iterations"] == rg["inner_iterations"]
    assert np.max(np.abs(xp - xg)) <= 1e-10 * (1 + np.max(np.abs(xg)))

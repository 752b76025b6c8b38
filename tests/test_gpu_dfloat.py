"""The double-float precision mode (FP32 matrix values, vectors as hi + lo FP32
pairs on the FP32 pipe) against the FP64 oracle and against the FP64-vector
(mixed) mode on the same FP32 matrix values.

Bars: relative KKT (oracle's evaluator on the GPU solution) <= eps and
relative objective difference to the oracle <= 1e-6, as for the mixed mode;
after 100 PDHG steps the double-float iterates equal the mixed-mode iterates to
1e-9 relative (both round the matrix to FP32 identically, so the difference is
the vector arithmetic alone: ~2^-48 per operation).
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


def rel(a, b):
    return abs(a - b) / (1.0 + abs(b))


def solve(qp, **kw):
    kw.setdefault("time_limit_s", 120.0)
    prob = pdhcg.Problem(qp, pdhcg.default_params(**kw))
    try:
        return prob.solve()
    finally:
        prob.close()


CASES = {
    "tiny_random_bb": lambda: W.random_qp(seed=0),
    "tiny_random_bb_seed1": lambda: W.random_qp(seed=1),
    "equality_cg": lambda: W.equality_qp(n=30, m=10, seed=2),
    "mpc_diag": lambda: W.mpc_qp(seed=11),
    "large_sparse_multi_cta": lambda: W.large_sparse_qp(n=20000, m=10000, seed=0),
}


@pytest.mark.parametrize("name", list(CASES))
def test_dfloat_optimal_parity(name):
    qp = CASES[name]()
    eps = 1e-6
    x, y, r = solve(qp, precision="dfloat", eps_tol=eps, max_iter=200000)
    assert r["status_name"] == "OPTIMAL", r
    rp, rd, rg, pobj, _ = kkt_of(qp, x, y)
    assert max(rp, rd, rg) <= eps, (rp, rd, rg)
    xo, yo, ro = oracle.solve(qp, oracle.default_params(eps_tol=eps))
    assert ro["status_name"] == "OPTIMAL"
    assert rel(pobj, ro["primal_obj"]) <= 1e-6, (pobj, ro["primal_obj"])


def test_dfloat_long_row_multi_cta():
    # the budget row has 20000 nonzeros and is summed by a whole CTA
    qp = W.factor_portfolio(n=20000, k=50, seed=0)
    x, y, r = solve(qp, precision="dfloat", eps_tol=1e-6, group_blocks=16, max_iter=200000)
    assert r["status_name"] == "OPTIMAL", r
    rp, rd, rg, pobj, _ = kkt_of(qp, x, y)
    assert max(rp, rd, rg) <= 1e-6
    xo, yo, ro = oracle.solve(qp, oracle.default_params(eps_tol=1e-6))
    assert rel(pobj, ro["primal_obj"]) <= 1e-6


@pytest.mark.parametrize("name", ["tiny_random_bb", "equality_cg", "mpc_diag", "large_sparse_multi_cta"])
@pytest.mark.parametrize("N", [1, 17, 100])
def test_dfloat_iterates_match_fp64_vectors(name, N):
    qp = CASES[name]()
    xm, ym, rm = solve(qp, precision="mixed", max_iter=N)
    xd, yd, rd = solve(qp, precision="dfloat", max_iter=N)
    assert rd["iterations"] == rm["iterations"] == N
    assert rd["inner_iterations"] == rm["inner_iterations"]
    assert np.max(np.abs(xd - xm)) <= 1e-9 * (1 + np.max(np.abs(xm)))
    assert np.max(np.abs(yd - ym), initial=0.0) <= 1e-9 * (1 + np.max(np.abs(ym), initial=0.0))


@pytest.mark.parametrize("seed", [0, 1])
def test_dfloat_infeasibility(seed):
    qp = W.infeasible_qp(n=8, m=4, seed=seed)
    x, y, r = solve(qp, precision="dfloat", max_iter=200000)
    assert r["status_name"] == "PRIMAL_INFEASIBLE"
    check_primal_ray(qp, y)
    # Q d = 0 holds bit for bit in FP32 storage too (mirrored columns)
    qp = W.unbounded_qp(n=6, seed=seed)
    x, y, r = solve(qp, precision="dfloat", max_iter=200000)
    assert r["status_name"] == "DUAL_INFEASIBLE"
    check_dual_ray(qp, x)


def test_dfloat_batch_equals_single():
    qps = W.mpc_batch(count=24, seed=3) + [W.random_qp(seed=5)]
    prm = pdhcg.default_params(precision="dfloat", eps_tol=1e-6)
    probs = pdhcg.create_batch(qps, prm)
    try:
        out = pdhcg.solve_batch(probs, want_solutions=True)
    finally:
        for p in probs:
            p.close()
    for qp, (xb, yb, rb) in zip(qps, out):
        xs, ys, rs = solve(qp, precision="dfloat", eps_tol=1e-6)
        assert rb["status_name"] == rs["status_name"] == "OPTIMAL"
        assert rb["iterations"] == rs["iterations"]
        assert np.max(np.abs(xb - xs)) <= 1e-12 * (1 + np.max(np.abs(xs)))

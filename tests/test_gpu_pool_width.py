"""Pool CTA width and shared-memory placement (one-CTA solves of small problems).

* pdhcg_params.pool_threads picks 256-thread pool CTAs (default) or 128-thread
  ones; either way a problem gives the same bits alone and in a batch, and
  both widths reach relative KKT <= 1e-6 on the oracle's FP64 evaluator
  (Sec. 4.2).
* Narrow CTAs run four to an SM; an instance whose vectors exceed a quarter of
  the SM's shared memory keeps only part of them on chip.  Placement changes
  no arithmetic: such an instance, batched with small ones (partial
  placement), equals its solve alone (every vector on chip) bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2602_23967_b300 import pdhcg
from paper_2602_23967_b300 import workloads as W

pytestmark = pytest.mark.gpu


def kkt_of(qp, x, y):
    Qx = qp.Q @ x if qp.Q is not None else np.zeros(qp.n)
    r = oracle.kkt(qp.n, qp.m, x, y, qp.A @ x, qp.A.T @ y, Qx, qp.c, qp.lc, qp.uc, qp.lv, qp.uv)
    return max(r[:3])


def solve_alone(qp, prm):
    p = pdhcg.Problem(qp, prm)
    try:
        return p.solve()
    finally:
        p.close()


@pytest.mark.parametrize("width", [0, 128])
def test_width_same_bits_alone_and_batched(width):
    qps = [W.mpc_qp(T=t, seed=300 + t) for t in (10, 24, 37, 50)]
    prm = pdhcg.default_params(precision="dfloat", eps_tol=1e-6, pool_threads=width)
    probs = [pdhcg.Problem(q, prm) for q in qps]
    try:
        batch = pdhcg.solve_batch(probs)
    finally:
        for p in probs:
            p.close()
    for q, (xb, yb, rb) in zip(qps, batch):
        xs, ys, rs = solve_alone(q, prm)
        assert rb["status_name"] == rs["status_name"] == "OPTIMAL"
        assert rb["iterations"] == rs["iterations"]
        assert np.array_equal(xb, xs) and np.array_equal(yb, ys)
        assert kkt_of(q, xs, ys) <= 1e-6


def test_widths_agree_to_tolerance():
    qps = [W.mpc_qp(seed=400 + i) for i in range(6)]
    out = {}
    for width in (0, 128):
        probs = pdhcg.create_batch(qps, pdhcg.default_params(precision="dfloat", eps_tol=1e-6,
                                                             pool_threads=width))
        try:
            out[width] = pdhcg.solve_batch(probs)
        finally:
            for p in probs:
                p.close()
    for q, (xw, yw, rw), (xn, yn, rn) in zip(qps, out[0], out[128]):
        assert rw["status_name"] == rn["status_name"] == "OPTIMAL"
        assert kkt_of(q, xw, yw) <= 1e-6 and kkt_of(q, xn, yn) <= 1e-6
        assert abs(rw["primal_obj"] - rn["primal_obj"]) <= 1e-6 * (1 + abs(rn["primal_obj"]))


def test_partial_placement_same_bits():
    # T = 50: 88 KB of vectors, more than a narrow CTA's quarter of an SM
    big = W.mpc_qp(T=50, seed=7)
    small = [W.mpc_qp(T=12, seed=500 + i) for i in range(300)]
    prm = pdhcg.default_params(precision="dfloat", eps_tol=1e-6, pool_threads=128)
    probs = pdhcg.create_batch([big] + small, prm)
    try:
        xb, yb, rb = pdhcg.solve_batch(probs)[0]
    finally:
        for p in probs:
            p.close()
    xs, ys, rs = solve_alone(big, prm)
    assert rb["status_name"] == rs["status_name"] == "OPTIMAL"
    assert rb["iterations"] == rs["iterations"]
    assert np.array_equal(xb, xs) and np.array_equal(yb, ys)
    assert kkt_of(big, xs, ys) <= 1e-6

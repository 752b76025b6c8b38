"""Serving loop (pdhcg_server_*): continuous batching at iteration granularity.

Each request's result is the same alone (pdhcg_solve) and in the mix: pausing a
solve at a slice boundary and resuming it in a later launch changes nothing in
its arithmetic, so the comparison is to 1e-12 (in practice bit-identical).
"""
import time

import numpy as np
import pytest

from paper_2602_23967_b300 import pdhcg
from paper_2602_23967_b300 import workloads as W

pytestmark = pytest.mark.gpu


def wait_all(srv, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            r = srv.poll(t)
            if r is not None:
                out[t] = r
        if time.time() - t0 > timeout:
            raise TimeoutError(f"{len(out)}/{len(tickets)} finished")
        time.sleep(0.002)
    return out


def test_mix_results_equal_alone():
    prm = pdhcg.default_params(precision="mixed", eps_tol=1e-6)
    qps = ([W.mpc_qp(seed=300 + i) for i in range(10)] +
           [W.random_qp(n=400, m=200, n_eq=100, m_rows=100, per_row=10, seed=50 + i) for i in range(3)] +
           [W.infeasible_qp(n=8, m=4, seed=1)])
    srv = pdhcg.Server(hbm_budget_bytes=2 << 30, max_slots=8, params=prm)
    try:
        tickets = []
        for q in qps:
            tickets.append(srv.submit(q))
            time.sleep(0.001)          # arrivals while others run
        got = wait_all(srv, tickets)
        st = srv.stats()
        assert st["completed"] == len(qps) and st["launches"] > 1
        assert st["hbm_in_use"] == 0 and st["live"] == 0
    finally:
        srv.close()
    for q, t in zip(qps, tickets):
        p = pdhcg.Problem(q, prm)
        xs, ys, rs = p.solve()
        p.close()
        xm, ym, rm = got[t]
        # wall-clock submit-to-ready latency covers at least the device solve
        assert rm["latency_seconds"] >= rm["solve_seconds"] > 0
        assert rs["latency_seconds"] == 0.0
        assert rm["status_name"] == rs["status_name"]
        assert rm["iterations"] == rs["iterations"]
        assert np.max(np.abs(xm - xs)) <= 1e-12 * (1 + np.max(np.abs(xs)))
        if q.m:
            assert np.max(np.abs(ym - ys)) <= 1e-12 * (1 + np.max(np.abs(ys)))
    assert got[tickets[-1]][2]["status_name"] == "PRIMAL_INFEASIBLE"


def test_budget_and_slots_limit_admission():
    prm = pdhcg.default_params(precision="mixed")
    qps = [W.mpc_qp(T=40, seed=400 + i) for i in range(6)]
    pair = pdhcg.create_batch(qps[:2], prm)       # pooled handles, as the server creates them
    per = max(p.device_bytes() for p in pair) + 4096
    for p in pair:
        p.close()
    budget = int(2.5 * per)
    srv = pdhcg.Server(hbm_budget_bytes=budget, max_slots=4, params=prm)
    try:
        tickets = [srv.submit(q) for q in qps]
        seen_live = 0
        t0 = time.time()
        while srv.stats()["completed"] < len(qps) and time.time() - t0 < 60:
            st = srv.stats()
            seen_live = max(seen_live, st["live"])
            assert st["hbm_in_use"] <= budget
            time.sleep(0.001)
        assert 1 <= seen_live <= 2
        got = wait_all(srv, tickets)
        assert all(r[2]["status_name"] == "OPTIMAL" for r in got.values())
    finally:
        srv.close()


def test_invalid_request_rejected_alone():
    prm = pdhcg.default_params(precision="mixed")
    srv = pdhcg.Server(hbm_budget_bytes=1 << 30, max_slots=4, params=prm)
    try:
        good = srv.submit(W.mpc_qp(seed=7))
        bad = W.mpc_qp(seed=8)
        bad.c = bad.c.copy()
        bad.c[0] = np.nan
        with pytest.raises(pdhcg.PdhcgError):
            srv.submit(bad)
        got = wait_all(srv, [good])
        assert got[good][2]["status_name"] == "OPTIMAL"
    finally:
        srv.close()


def _served(prm, qps, slots=16, gap=0.001):
    srv = pdhcg.Server(hbm_budget_bytes=8 << 30, max_slots=slots, params=prm)
    try:
        tickets = []
        for q in qps:
            tickets.append(srv.submit(q))
            time.sleep(gap)
        got = wait_all(srv, tickets, timeout=600.0)
        st = srv.stats()
    finally:
        srv.close()
    return [got[t] for t in tickets], st


def test_mix_with_large_requests_equal_alone():
    # The request mix of the serving workload at test size: MPC QPs on pool
    # CTAs, and random QPs (one made infeasible by a contradictory equality
    # row, Sec. 5.1) and a factor-model QP large enough to run on multi-CTA
    # groups, in a cooperative launch of their own beside the pool launch of
    # each slice.  Every request's result is the same served alone and in the
    # mix: pool solves keep their 128-thread kernel and groups their size, so
    # the arithmetic does not depend on what else is live.
    prm = pdhcg.default_params(precision="dfloat", eps_tol=1e-6, max_iter=400000)
    qps = ([W.mpc_qp(seed=500 + i) for i in range(6)] +
           [W.build_request("random", 61, 8000), W.build_request("random_infeasible", 62, 6000),
            W.factor_portfolio(n=30000, k=300, seed=63), W.build_request("random", 64, 1500)])
    mixed, st = _served(prm, qps)
    assert st["completed"] == len(qps) and st["launches"] > 1
    for q, (xm, ym, rm) in zip(qps, mixed):
        alone, _ = _served(prm, [q])
        xs, ys, rs = alone[0]
        assert rm["status_name"] == rs["status_name"], (q.name, rm, rs)
        assert rm["iterations"] == rs["iterations"], q.name
        assert np.max(np.abs(xm - xs)) <= 1e-12 * (1 + np.max(np.abs(xs))), q.name
        if q.m:
            assert np.max(np.abs(ym - ys)) <= 1e-12 * (1 + np.max(np.abs(ys))), q.name
    names = [r[2]["status_name"] for r in mixed]
    assert names[7] == "PRIMAL_INFEASIBLE", names
    assert all(n == "OPTIMAL" for i, n in enumerate(names) if i != 7), names

"""Failure detection without a GPU fault (limits of Sec. 6.1 and the bounded waits).

* The paper's limits: a wall-clock budget ends a solve with TIME_LIMIT and an
  outer-step budget with ITERATION_LIMIT, at the first check past the limit,
  for single and batched solves.
* Every spin-wait of the kernel gives up after its limit and reports
  PDHCG_E_DEVICE_TIMEOUT; pdhcg_selftest_bounded_wait makes a group barrier
  and a flag wait run out on purpose (nothing sets what they wait for), and a
  solve afterwards shows the context is still usable.
* Serving admission: a request larger than the whole HBM budget is refused
  with E_OOM at submit, a full queue with E_BUSY, and the requests that were
  accepted still finish.
"""
import ctypes as C
import time

import numpy as np
import pytest

from paper_2602_23967_b300 import pdhcg
from paper_2602_23967_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_time_limit_ends_the_solve():
    qp = W.large_sparse_qp(n=20000, m=10000, seed=0)
    p = pdhcg.Problem(qp, pdhcg.default_params(precision="dfloat", eps_tol=1e-9, time_limit_s=1e-3))
    try:
        _, _, r = p.solve()
    finally:
        p.close()
    assert r["status_name"] == "TIME_LIMIT", r
    assert r["iterations"] % 64 == 0 and r["iterations"] >= 64       # stopped at a check
    assert r["solve_seconds"] >= 1e-3


def test_iteration_limit_single_and_batched():
    qps = [W.random_qp(seed=s) for s in range(3)]
    prm = pdhcg.default_params(max_iter=100, eps_tol=1e-12)
    p = pdhcg.Problem(qps[0], prm)
    try:
        _, _, r = p.solve()
    finally:
        p.close()
    assert r["status_name"] == "ITERATION_LIMIT" and r["iterations"] == 100
    probs = [pdhcg.Problem(q, prm) for q in qps]
    try:
        out = pdhcg.solve_batch(probs)
    finally:
        for q in probs:
            q.close()
    assert all(rr["status_name"] == "ITERATION_LIMIT" and rr["iterations"] == 100 for _, _, rr in out)


def test_time_limit_in_a_batch():
    qps = [W.large_sparse_qp(n=4000, m=2000, seed=s) for s in range(4)]
    probs = [pdhcg.Problem(q, pdhcg.default_params(precision="dfloat", eps_tol=1e-12, time_limit_s=2e-3))
             for q in qps]
    try:
        out = pdhcg.solve_batch(probs, want_solutions=False)
    finally:
        for q in probs:
            q.close()
    assert all(r["status_name"] == "TIME_LIMIT" for r in out), [r["status_name"] for r in out]


def test_bounded_waits_give_up_and_report():
    L = pdhcg.lib()
    L.pdhcg_selftest_bounded_wait.argtypes = [C.c_int32, C.POINTER(C.c_double)]
    waited = C.c_double()
    rc = L.pdhcg_selftest_bounded_wait(2000, C.byref(waited))
    assert rc == pdhcg.E_DEVICE_TIMEOUT, (rc, L.pdhcg_last_error())
    assert 2 * 2e-3 <= waited.value < 2.0            # both waits ran to their 2 ms limit and stopped
    assert L.pdhcg_selftest_bounded_wait(0, None) == pdhcg.E_INVALID
    # the context is still usable: a solve right after succeeds
    p = pdhcg.Problem(W.random_qp(seed=0), pdhcg.default_params())
    try:
        _, _, r = p.solve()
    finally:
        p.close()
    assert r["status_name"] == "OPTIMAL"


def test_serving_refuses_oversized_and_overflowing_requests():
    prm = pdhcg.default_params(precision="dfloat", eps_tol=1e-6)
    small = W.mpc_qp(seed=3)
    probe = pdhcg.create_batch([small, small], prm)
    per = max(q.device_bytes() for q in probe) + 4096
    for q in probe:
        q.close()
    # budget below one problem: refused at submit, nothing queued
    srv = pdhcg.Server(hbm_budget_bytes=per // 4, max_slots=2, params=prm)
    try:
        with pytest.raises(pdhcg.PdhcgError) as ei:
            srv.submit(small)
        assert ei.value.code == pdhcg.E_OOM
        assert srv.stats()["submitted"] == 0
    finally:
        srv.close()
    # one slot held by a long solve and a bounded queue (64 per slot): the
    # submit after the queue is full is refused with E_BUSY
    long_qp = W.large_sparse_qp(n=20000, m=10000, seed=1)
    slow = pdhcg.default_params(precision="dfloat", eps_tol=1e-12, time_limit_s=5.0)
    srv = pdhcg.Server(hbm_budget_bytes=1 << 30, max_slots=1, params=slow)
    try:
        first = srv.submit(long_qp)
        t0 = time.time()
        while srv.stats()["live"] == 0 and time.time() - t0 < 30:
            time.sleep(0.001)
        accepted, busy = [first], None
        for _ in range(200):
            try:
                accepted.append(srv.submit(small))
            except pdhcg.PdhcgError as e:
                busy = e
                break
        assert busy is not None and busy.code == pdhcg.E_BUSY
        assert len(accepted) == 1 + 64
        st = srv.stats()
        assert st["queued"] <= 64 and st["submitted"] == len(accepted)
    finally:
        srv.close()

"""pdhcg_solve_batch_noalloc (static device scratch) against pdhcg_solve_batch.

Collected last on purpose: the static scratch is process-wide, so this file also
shows that the entry point works after every other test of the session has run
(and alone: ``pytest tests/test_zz_no_alloc.py``).
"""
import ctypes as C

import numpy as np
import pytest

from paper_2602_23967_b300 import pdhcg
from paper_2602_23967_b300 import workloads as W

pytestmark = pytest.mark.gpu

# The batched kernel is deterministic per instance (one CTA solves it start to
# finish), so both entry points should give the same bits; the bar allows for
# nothing more than rounding.
RTOL = 1e-12


def _close(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.max(np.abs(a - b), initial=0.0) <= RTOL * (1.0 + np.max(np.abs(b), initial=0.0))


def _instances():
    qps = W.mpc_batch(count=40, seed=11)
    qps += [W.random_qp(seed=s) for s in (21, 22)]    # BB inner solver on a non-diagonal Q
    qps += [W.equality_qp(n=30, m=10, seed=23)]       # CG inner solver
    return qps


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_solve_batch_twice(precision):
    import torch
    qps = _instances()
    probs = pdhcg.create_batch(qps, pdhcg.default_params(precision=precision, eps_tol=1e-6))
    try:
        ref = pdhcg.solve_batch(probs, want_solutions=True)
        assert all(rr["status_name"] == "OPTIMAL" for _, _, rr in ref[:40])   # the MPC instances
        for call in range(2):  # two calls in a row reuse the same static scratch
            xs = [torch.full((p.n,), np.nan, dtype=torch.float64, device="cuda") for p in probs]
            ys = [torch.full((max(p.m, 1),), np.nan, dtype=torch.float64, device="cuda") for p in probs]
            out = pdhcg.solve_batch_noalloc(probs, xs, ys)
            torch.cuda.synchronize()
            for i, (xr, yr, rr) in enumerate(ref):
                r = out[i]
                assert r["status_name"] == rr["status_name"], (call, i, r, rr)
                assert r["iterations"] == rr["iterations"], (call, i)
                assert r["inner_iterations"] == rr["inner_iterations"], (call, i)
                for key in ("r_primal", "r_dual", "r_gap", "primal_obj", "dual_obj", "omega"):
                    assert _close(r[key], rr[key]), (call, i, key, r[key], rr[key])
                assert _close(xs[i].cpu().numpy(), xr), (call, i)
                assert _close(ys[i][: probs[i].m].cpu().numpy(), yr), (call, i)
    finally:
        for p in probs:
            p.close()


def test_noalloc_results_only_and_limits():
    qps = W.mpc_batch(count=6, seed=5)
    probs = pdhcg.create_batch(qps, pdhcg.default_params(precision="mixed", eps_tol=1e-6))
    try:
        ref = pdhcg.solve_batch(probs, want_solutions=False)
        out = pdhcg.solve_batch_noalloc(probs)           # no solution buffers at all
        assert [r["iterations"] for r in out] == [r["iterations"] for r in ref]
        assert pdhcg.solve_batch_noalloc([]) == []      # count 0 is a no-op
        # more instances than the static scratch holds: rejected before any launch
        L = pdhcg.lib()
        count = pdhcg.NOALLOC_MAX_INSTANCES + 1
        handles = (C.c_void_p * count)(*([probs[0].handle] * count))
        rc = L.pdhcg_solve_batch_noalloc(handles, count, None, None, None)
        assert rc == -1
        assert b"1024" in L.pdhcg_last_error()
    finally:
        for p in probs:
            p.close()

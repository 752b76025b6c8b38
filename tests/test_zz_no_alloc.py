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


@pytest.mark.parametrize("precision", ["fp64", "mixed", "dfloat"])
def test_noalloc_matches_solve_batch_twice(precision):
    import torch
    qps = _instances()
    probs = pdhcg.create_batch(qps, pdhcg.default_params(precision=precision, eps_tol=1e-6))
    # a lifted-bound handle (PDHCG_INNER_CG_LIFTED): its kernel writes the
    # handle's own dual staging, and only the original rows' duals reach y_out
    probs.append(pdhcg.Problem(W.random_qp(seed=24), pdhcg.default_params(precision=precision, eps_tol=1e-6,
                                                                         inner="cg_lifted", max_iter=200000)))
    try:
        ref = pdhcg.solve_batch(probs, want_solutions=True)
        assert all(rr["status_name"] == "OPTIMAL" for _, _, rr in ref[:40])   # the MPC instances
        assert ref[-1][2]["status_name"] == "OPTIMAL" and ref[-1][2]["inner_method"] == 2
        # every output buffer exists before the first call, so nothing in the
        # measured region below allocates on the caller's side either
        xs = [torch.empty((p.n,), dtype=torch.float64, device="cuda") for p in probs]
        ys = [torch.empty((max(p.m, 1),), dtype=torch.float64, device="cuda") for p in probs]
        torch.cuda.synchronize()
        mem = []
        for call in range(2):  # two calls in a row reuse the same static scratch
            for t in xs + ys:
                t.fill_(np.nan)
            out = pdhcg.solve_batch_noalloc(probs, xs, ys)
            torch.cuda.synchronize()
            # device memory after the call: free bytes (driver) and torch's reserve
            mem.append((torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()))
            for i, (xr, yr, rr) in enumerate(ref):
                r = out[i]
                assert r["status_name"] == rr["status_name"], (call, i, r, rr)
                assert r["iterations"] == rr["iterations"], (call, i)
                assert r["inner_iterations"] == rr["inner_iterations"], (call, i)
                for key in ("r_primal", "r_dual", "r_gap", "primal_obj", "dual_obj", "omega"):
                    assert _close(r[key], rr[key]), (call, i, key, r[key], rr[key])
                assert _close(xs[i].cpu().numpy(), xr), (call, i)
                assert _close(ys[i][: probs[i].m].cpu().numpy(), yr), (call, i)
        # the second call (after the first set up the scratch address) took no device memory
        assert mem[1] == mem[0], mem
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

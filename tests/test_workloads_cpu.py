"""The synthetic generators match the recipes the design notes state for them
(shapes, structure, value ranges, determinism).  No arithmetic of the method is
involved: these are properties of the inputs."""
import numpy as np
import scipy.sparse as sp

from paper_2602_23967_b300 import workloads as W


def test_mpc_qp_recipe():
    for seed in range(6):
        qp = W.mpc_qp(seed=seed)
        T = qp.meta["T"]
        assert 10 <= T <= 50 and qp.n == 16 * T and qp.m == 12 * T
        d = qp.Q.diagonal()
        assert qp.Q.nnz == qp.n and np.allclose(qp.Q.toarray(), np.diag(d))
        u = d.reshape(T, 16)[:, :4]
        x = d.reshape(T, 16)[:, 4:]
        assert np.all((u >= 0.1) & (u <= 1.0)) and np.all((x >= 1.0) & (x <= 10.0))
        assert np.all(qp.c == 0) and np.array_equal(qp.lc, qp.uc)
        lv, uv = qp.lv.reshape(T, 16), qp.uv.reshape(T, 16)
        assert np.all(lv[:, :4] == -1) and np.all(uv[:, :4] == 1)
        assert np.all(np.isneginf(lv[:, 4:])) and np.all(np.isposinf(uv[:, 4:]))
        per_row = np.diff(qp.A.indptr)
        assert np.all(per_row[:12] == 5) and np.all(per_row[12:] == 17)
        # rows of step 1 hold -A_d on x_1: its spectral radius is at most 1.05
        Ad = -qp.A[12:24, 4:16].toarray()
        assert np.max(np.abs(np.linalg.eigvals(Ad))) <= 1.05 + 1e-12


def test_mpc_batch_is_seeded_and_distinct():
    a = W.mpc_batch(count=6, seed=0)
    b = W.mpc_batch(count=6, seed=0)
    for p, q in zip(a, b):
        assert p.n == q.n and (p.A != q.A).nnz == 0 and np.array_equal(p.lc, q.lc)
    assert len({(q.n, float(q.lc[0])) for q in a}) == len(a)


def test_large_sparse_qp_recipe_at_reduced_size():
    n, m = 20_000, 10_000
    qp = W.large_sparse_qp(n=n, m=m, seed=1)
    Q = qp.Q
    assert abs(Q - Q.T).max() == 0
    off = Q - sp.diags(Q.diagonal())
    margin = Q.diagonal() - np.asarray(abs(off).sum(axis=1)).ravel()
    assert np.all((margin >= 0.1 - 1e-12) & (margin <= 1.0 + 1e-12))      # diagonally dominant
    assert 9.0 <= Q.nnz / n <= 11.0                                           # ~10 per row
    assert 6.0 <= qp.A.nnz / m <= 10.0                                        # ~8 per row
    deg = np.diff(qp.A.tocsc().indptr)
    assert deg.max() >= 10 * deg.mean()                                       # heavy-tailed columns
    assert np.sum(qp.lc == qp.uc) == round(0.3 * m)                           # 30 % equality rows
    boxed = np.isfinite(qp.lv)
    assert 0.45 <= boxed.mean() <= 0.55
    assert np.all(qp.lv[boxed] == -100) and np.all(qp.uv[boxed] == 100)


def test_factor_portfolio_recipe_at_reduced_size():
    n, k = 2_000, 20
    qp = W.factor_portfolio(n=n, k=k, seed=0)
    assert qp.n == n + k and qp.m == k + 1
    d = qp.Q.diagonal()
    assert np.all((d[:n] >= 0.02) & (d[:n] <= 0.2)) and np.all(d[n:] == 2.0)
    assert np.array_equal(qp.A[k].toarray().ravel(), np.r_[np.ones(n), np.zeros(k)])   # budget row
    assert np.array_equal(qp.A[:k, n:].toarray(), -np.eye(k))                             # F^T x - y = 0
    assert np.all(qp.lv[:n] == 0) and np.all(qp.uv[:n] == 0.01)


def test_serving_trace_rate_and_mix():
    rate, dur = 2000.0, 4.0
    tr = W.serving_trace(rate_per_s=rate, duration_s=dur, seed=3)
    t = np.array([e[0] for e in tr])
    assert np.all(np.diff(t) > 0) and t[-1] <= dur
    expect = rate * dur
    assert abs(len(tr) - expect) <= 5 * np.sqrt(expect)                       # Poisson count
    kinds = [e[1] for e in tr]
    frac_mpc = kinds.count("mpc") / len(tr)
    frac_factor = kinds.count("factor") / len(tr)
    assert abs(frac_mpc - 0.70) < 0.03 and abs(frac_factor - 0.05) < 0.015
    only_mpc = W.serving_trace(rate_per_s=rate, duration_s=1.0, seed=3, mix=(1.0, 0.0, 0.0))
    assert all(e[1] == "mpc" for e in only_mpc)

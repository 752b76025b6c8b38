"""Checks of returned infeasibility certificates against the conditions of
Sec. 5.1 (primal: a dual ray) and Sec. 5.2 (dual: a primal ray), with the
componentwise recession cones of reading D11.  Shared by the GPU tests."""
import numpy as np


def support(z, lo, hi):
    """p(z; l, u) = u^T z+ - l^T z- with 0 * inf = 0 (Sec. 4.2)."""
    return sum(hi[i] * z[i] if z[i] > 0 else (lo[i] * z[i] if z[i] < 0 else 0.0) for i in range(len(z)))


def check_primal_ray(qp, y, tol=1e-6):
    """y certifies Ax in S, x in X empty: y in the sign cone of the rows,
    A^T y in the cone R that makes p(-A^T y; l, u) finite, and
    p(-A^T y; lv, uv) + p(y; lc, uc) < 0."""
    y = np.asarray(y, dtype=np.float64)
    scale = max(np.max(np.abs(y)), 1e-300)
    for i in range(qp.m):
        lf, uf = np.isfinite(qp.lc[i]), np.isfinite(qp.uc[i])
        if lf and not uf:
            assert y[i] <= tol * scale, (i, y[i])
        if uf and not lf:
            assert y[i] >= -tol * scale, (i, y[i])
        if not lf and not uf:
            assert abs(y[i]) <= tol * scale, (i, y[i])
    g = qp.A.T @ y
    val = support(-g, qp.lv, qp.uv) + support(y, qp.lc, qp.uc)
    assert val < 0, val
    viol = 0.0
    for j in range(qp.n):
        lf, uf = np.isfinite(qp.lv[j]), np.isfinite(qp.uv[j])
        if not lf and not uf:
            viol = max(viol, abs(g[j]))
        elif lf and not uf:
            viol = max(viol, -g[j])
        elif uf and not lf:
            viol = max(viol, g[j])
    assert viol <= tol * abs(val), (viol, val)
    return val


def check_dual_ray(qp, d, tol=1e-5):
    """d certifies an unbounded objective: c^T d < 0, Q d = 0, d in Recc(X)
    and A d in Recc(S) (componentwise: {0} for two finite bounds, R+ for a
    lower one only, R- for an upper one only, R for none)."""
    d = np.asarray(d, dtype=np.float64)
    scale = np.max(np.abs(d))
    assert scale > 0
    d = d / scale
    assert qp.c @ d < 0, qp.c @ d
    if qp.Q is not None:
        assert np.max(np.abs(qp.Q @ d)) <= tol

    def in_recc(v, lo, hi):
        for i in range(len(v)):
            lf, uf = np.isfinite(lo[i]), np.isfinite(hi[i])
            if lf and uf:
                assert abs(v[i]) <= tol, (i, v[i])
            elif lf:
                assert v[i] >= -tol, (i, v[i])
            elif uf:
                assert v[i] <= tol, (i, v[i])

    in_recc(d, qp.lv, qp.uv)
    in_recc(qp.A @ d, qp.lc, qp.uc)

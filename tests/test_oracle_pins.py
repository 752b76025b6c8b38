"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these checks re-types the oracle's formulas: each compares the oracle
with an independent route to the same answer.

* equality-only QP with free x: the KKT system of Sec. 4.1 is linear, solved
  here by dense LU (numpy.linalg.solve);
* boxed / inequality QPs with n <= 8: active-set brute force over the sign
  conditions of Sec. 2 (y in Y, r in R) and Sec. 4.1;
* LP special case (Q = 0): scipy's HiGHS linprog;
* constructed infeasible / unbounded instances: the certificate systems of
  Sec. 5.1 and the theorem of Sec. 5.2;
* ||A||_2 against the SVD; the CG subproblem against a dense solve; the BB
  subproblem against box brute force (Sec. 2.2);
* invariants: Halpern keeps a fixed point fixed (Sec. 3.1), the PID law keeps
  a balanced weight and moves it in the right direction (Eq. pid), the
  adaptive inner tolerance is monotone and floored (Sec. 3.3).
"""
import itertools

import numpy as np
import pytest
import scipy.optimize
import scipy.sparse as sp

import oracle
from paper_2602_23967_b300 import workloads as W

TIGHT = dict(eps_tol=1e-10, max_iter=400000)


def dense(M):
    return M.toarray() if M is not None else None


def kkt_dense_solve(qp):
    Q, A = dense(qp.Q), dense(qp.A)
    n, m = qp.n, qp.m
    K = np.block([[Q, A.T], [A, np.zeros((m, m))]])
    rhs = np.concatenate([-qp.c, qp.lc])
    sol = np.linalg.solve(K, rhs)
    return sol[:n], sol[n:]


def brute_force_qp(qp):
    """Enumerate active sets of a small QP; return the KKT point satisfying every sign rule.

    Variable states: at lower, at upper, free.  Row states: equality rows always
    active; one-sided rows active or inactive.  Sign rules (Sec. 2 cones): reduced
    cost r = Qx + c + A^T y is >= 0 at a lower bound, <= 0 at an upper bound,
    0 when free; y_i >= 0 for an active upper row, <= 0 for an active lower row,
    0 when inactive."""
    Q, A = dense(qp.Q), dense(qp.A)
    n, m = qp.n, qp.m
    var_states = []
    for j in range(n):
        s = ["free"]
        if np.isfinite(qp.lv[j]):
            s.append("lo")
        if np.isfinite(qp.uv[j]):
            s.append("up")
        var_states.append(s)
    row_states = []
    for i in range(m):
        if qp.lc[i] == qp.uc[i]:
            row_states.append(["eq"])
        else:
            s = ["off"]
            if np.isfinite(qp.lc[i]):
                s.append("lo")
            if np.isfinite(qp.uc[i]):
                s.append("up")
            row_states.append(s)
    best = None
    tol = 1e-9
    for vs in itertools.product(*var_states):
        fixed = [j for j in range(n) if vs[j] != "free"]
        free = [j for j in range(n) if vs[j] == "free"]
        xf = np.zeros(n)
        for j in fixed:
            xf[j] = qp.lv[j] if vs[j] == "lo" else qp.uv[j]
        for rs in itertools.product(*row_states):
            act = [i for i in range(m) if rs[i] != "off"]
            bvals = np.array([qp.lc[i] if rs[i] in ("eq", "lo") else qp.uc[i] for i in act])
            # unknowns: x_free, y_act ; equations: (Qx + c + A^T y)_free = 0, A_act x = b
            nf, na = len(free), len(act)
            Kf = np.zeros((nf + na, nf + na))
            rhs = np.zeros(nf + na)
            Kf[:nf, :nf] = Q[np.ix_(free, free)]
            Kf[:nf, nf:] = A[np.ix_(act, free)].T
            Kf[nf:, :nf] = A[np.ix_(act, free)]
            rhs[:nf] = -(qp.c[free] + Q[np.ix_(free, fixed)] @ xf[fixed])
            rhs[nf:] = bvals - A[np.ix_(act, fixed)] @ xf[fixed]
            try:
                sol, *_ = np.linalg.lstsq(Kf, rhs, rcond=None)
            except np.linalg.LinAlgError:
                continue
            if np.linalg.norm(Kf @ sol - rhs) > 1e-8 * (1 + np.linalg.norm(rhs)):
                continue
            x = xf.copy()
            x[free] = sol[:nf]
            y = np.zeros(m)
            y[act] = sol[nf:]
            if np.any(x < qp.lv - tol) or np.any(x > qp.uv + tol):
                continue
            Ax = A @ x
            if np.any(Ax < qp.lc - tol) or np.any(Ax > qp.uc + tol):
                continue
            r = Q @ x + qp.c + A.T @ y
            ok = True
            for j in range(n):
                if vs[j] == "lo" and r[j] < -tol:
                    ok = False
                if vs[j] == "up" and r[j] > tol:
                    ok = False
            for i in range(m):
                if rs[i] == "up" and y[i] < -tol:
                    ok = False
                if rs[i] == "lo" and y[i] > tol:
                    ok = False
            if not ok:
                continue
            f = 0.5 * x @ Q @ x + qp.c @ x
            if best is None or f < best[0] - 1e-12:
                best = (f, x, y)
    return best


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equality_qp_matches_dense_kkt(seed):
    qp = W.equality_qp(n=30, m=10, seed=seed)
    xs, ys = kkt_dense_solve(qp)
    x, y, r = oracle.solve(qp, oracle.default_params(**TIGHT))
    assert r["status_name"] == "OPTIMAL"
    assert np.linalg.norm(x - xs) <= 1e-7 * (1 + np.linalg.norm(xs))
    assert np.linalg.norm(y - ys) <= 1e-6 * (1 + np.linalg.norm(ys))
    fs = 0.5 * xs @ dense(qp.Q) @ xs + qp.c @ xs
    assert abs(r["primal_obj"] - fs) <= 1e-8 * (1 + abs(fs))


@pytest.mark.parametrize("inner", ["auto", "bb"])
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_small_box_qp_matches_brute_force(seed, inner):
    qp = W.small_box_qp(n=6, m=3, seed=seed)
    best = brute_force_qp(qp)
    assert best is not None
    f_star, x_star, y_star = best
    x, y, r = oracle.solve(qp, oracle.default_params(inner=inner, **TIGHT))
    assert r["status_name"] == "OPTIMAL"
    assert abs(r["primal_obj"] - f_star) <= 1e-8 * (1 + abs(f_star))
    assert np.linalg.norm(x - x_star) <= 1e-6 * (1 + np.linalg.norm(x_star))


def test_kkt_residuals_vanish_at_brute_force_optimum():
    # At an exact KKT point every residual of Sec. 4.2 must be ~0; a dropped
    # term or wrong sign in any of them would leave a visible residual.
    for seed in range(3):
        qp = W.small_box_qp(n=6, m=3, seed=seed)
        f_star, x, y = brute_force_qp(qp)
        Q, A = dense(qp.Q), dense(qp.A)
        rp, rd, rg, pobj, dobj = oracle.kkt(qp.n, qp.m, x, y, A @ x, A.T @ y, Q @ x, qp.c, qp.lc,
                                            qp.uc, qp.lv, qp.uv)
        assert rp <= 1e-9 and rd <= 1e-9 and rg <= 1e-9
        assert abs(pobj - f_star) <= 1e-9 * (1 + abs(f_star))
        assert abs(dobj - f_star) <= 1e-8 * (1 + abs(f_star))   # strong duality


def test_kkt_residuals_detect_perturbation():
    qp = W.equality_qp(n=20, m=6, seed=4)
    xs, ys = kkt_dense_solve(qp)
    Q, A = dense(qp.Q), dense(qp.A)
    base = oracle.kkt(qp.n, qp.m, xs, ys, A @ xs, A.T @ ys, Q @ xs, qp.c, qp.lc, qp.uc, qp.lv, qp.uv)
    assert max(base[:3]) <= 1e-10
    x2 = xs + 1e-3 * np.random.default_rng(0).standard_normal(qp.n)
    pert = oracle.kkt(qp.n, qp.m, x2, ys, A @ x2, A.T @ ys, Q @ x2, qp.c, qp.lc, qp.uc, qp.lv, qp.uv)
    assert pert[0] > 1e-5 and pert[1] > 1e-5


def test_lp_special_case_matches_highs():
    rng = np.random.default_rng(3)
    n, m = 12, 6
    A = rng.standard_normal((m, n))
    x0 = rng.uniform(0, 1, n)
    b = A @ x0
    c = rng.uniform(0.1, 1.0, n) + np.abs(A.T @ rng.standard_normal(m)) * 0.0
    qp = W.QP(n, m, None, W._csr(A), c, b.copy(), b.copy(), np.zeros(n), np.full(n, 2.0))
    ref = scipy.optimize.linprog(c, A_eq=A, b_eq=b, bounds=[(0, 2)] * n, method="highs")
    assert ref.status == 0
    x, y, r = oracle.solve(qp, oracle.default_params(eps_tol=1e-9, max_iter=2000000))
    assert r["status_name"] == "OPTIMAL"
    assert abs(r["primal_obj"] - ref.fun) <= 1e-6 * (1 + abs(ref.fun))


def test_random_qp_matches_scipy_trust_constr():
    qp = W.random_qp(n=40, m=20, n_eq=10, m_rows=10, density=0.2, seed=5)
    Q, A = dense(qp.Q), dense(qp.A)
    cons = [scipy.optimize.LinearConstraint(A, qp.lc, qp.uc)]
    ref = scipy.optimize.minimize(lambda v: 0.5 * v @ Q @ v + qp.c @ v, np.zeros(qp.n),
                                  jac=lambda v: Q @ v + qp.c, hess=lambda v: Q,
                                  constraints=cons, bounds=scipy.optimize.Bounds(qp.lv, qp.uv),
                                  method="trust-constr", options={"gtol": 1e-10, "xtol": 1e-12,
                                                                  "maxiter": 20000})
    x, y, r = oracle.solve(qp, oracle.default_params(eps_tol=1e-9, max_iter=400000))
    assert r["status_name"] == "OPTIMAL"
    assert r["primal_obj"] <= ref.fun + 1e-5 * (1 + abs(ref.fun))
    assert abs(r["primal_obj"] - ref.fun) <= 1e-4 * (1 + abs(ref.fun))


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_primal_infeasible_certificate(seed):
    qp = W.infeasible_qp(n=8, m=4, seed=seed)
    x, y, r = oracle.solve(qp, oracle.default_params(max_iter=200000))
    assert r["status_name"] == "PRIMAL_INFEASIBLE"
    # returned ray: y in Y, A^T y in R (approx), and p(-A^T y; lv, uv) + p(y; lc, uc) < 0
    A = dense(qp.A)
    g = A.T @ y
    for i in range(qp.m):
        lf, uf = np.isfinite(qp.lc[i]), np.isfinite(qp.uc[i])
        if lf and not uf:
            assert y[i] <= 1e-12
        if uf and not lf:
            assert y[i] >= -1e-12
    def p(z, lo, hi):
        return sum(hi[i] * z[i] if z[i] > 0 else (lo[i] * z[i] if z[i] < 0 else 0.0)
                   for i in range(len(z)))
    val = p(-g, qp.lv, qp.uv) + p(y, qp.lc, qp.uc)
    assert val < 0
    viol = 0.0
    for j in range(qp.n):
        lf, uf = np.isfinite(qp.lv[j]), np.isfinite(qp.uv[j])
        if not lf and not uf:
            viol = max(viol, abs(g[j]))
        elif lf and not uf:
            viol = max(viol, -g[j])
        elif uf and not lf:
            viol = max(viol, g[j])
    assert viol <= 1e-6 * abs(val)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_dual_infeasible_certificate(seed):
    qp = W.unbounded_qp(n=6, seed=seed)
    x, y, r = oracle.solve(qp, oracle.default_params(max_iter=200000))
    assert r["status_name"] == "DUAL_INFEASIBLE"
    d = x
    Q, A = dense(qp.Q), dense(qp.A)
    assert np.max(np.abs(d)) == pytest.approx(1.0)
    assert qp.c @ d < 0
    assert np.max(np.abs(Q @ d)) <= 1e-5
    Ad = A @ d
    assert abs(Ad[0]) <= 1e-5           # equality row: Recc = {0}
    assert Ad[1] <= 1e-5                # <= row: Recc = R-
    assert np.all(np.abs(d[2:]) <= 1e-5)  # boxed variables: Recc = {0}


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_feasible_instances_are_not_flagged(seed):
    for qp in (W.random_qp(n=60, m=30, n_eq=15, m_rows=20, density=0.1, seed=seed),
               W.mpc_qp(T=10, seed=seed)):
        x, y, r = oracle.solve(qp, oracle.default_params(max_iter=200000))
        assert r["status_name"] == "OPTIMAL"


def test_norm_estimate_matches_svd():
    rng = np.random.default_rng(7)
    for shape in [(30, 50), (80, 20), (1, 10)]:
        A = sp.random(*shape, density=0.3, random_state=rng, format="csr")
        A = W._csr(A)
        est, it = oracle.norm_estimate(A, max_iter=100000, tol=1e-14)
        assert est == pytest.approx(np.linalg.norm(A.toarray(), 2), rel=1e-6)


@pytest.mark.parametrize("seed", [0, 1])
def test_inner_cg_matches_dense_solve(seed):
    rng = np.random.default_rng(seed)
    n = 40
    M = rng.standard_normal((n, n))
    Q = M.T @ M / n
    tau = 0.7
    b = rng.standard_normal(n)
    x, steps = oracle.inner_solve(W._csr(Q), np.full(n, -np.inf), np.full(n, np.inf), tau, b,
                                  np.zeros(n), 1e-13, 10000, "cg")
    ref = np.linalg.solve(Q + np.eye(n) / tau, b)
    assert np.linalg.norm(x - ref) <= 1e-11 * (1 + np.linalg.norm(ref))
    assert steps <= 200


def test_inner_bb_matches_box_brute_force():
    rng = np.random.default_rng(11)
    n = 6
    for trial in range(5):
        M = rng.standard_normal((n, n))
        Q = M.T @ M / n
        tau = 0.5
        H = Q + np.eye(n) / tau
        b = 4.0 * rng.standard_normal(n)
        lo, hi = -np.ones(n), np.ones(n)
        best = None
        for st in itertools.product(["lo", "up", "free"], repeat=n):
            fr = [j for j in range(n) if st[j] == "free"]
            fx = [j for j in range(n) if st[j] != "free"]
            x = np.zeros(n)
            for j in fx:
                x[j] = lo[j] if st[j] == "lo" else hi[j]
            if fr:
                x[fr] = np.linalg.solve(H[np.ix_(fr, fr)], b[fr] - H[np.ix_(fr, fx)] @ x[fx])
            if np.any(x < lo - 1e-12) or np.any(x > hi + 1e-12):
                continue
            f = 0.5 * x @ H @ x - b @ x
            if best is None or f < best[0]:
                best = (f, x)
        x, steps = oracle.inner_solve(W._csr(Q), lo, hi, tau, b, np.zeros(n), 1e-12, 100000, "bb")
        assert np.linalg.norm(x - best[1]) <= 1e-9


def test_halpern_keeps_fixed_point():
    qp = W.equality_qp(n=25, m=8, seed=9)
    xs, ys = kkt_dense_solve(qp)
    x, y, r = oracle.solve(qp, oracle.default_params(max_iter=50, k_eval=10, eps_inner_min=1e-14,
                                                     eps_inner_first=1e-14), x0=xs, y0=ys)
    assert np.linalg.norm(x - xs) <= 1e-9 * (1 + np.linalg.norm(xs))
    assert np.linalg.norm(y - ys) <= 1e-9 * (1 + np.linalg.norm(ys))


def test_pid_law():
    # balanced movement (omega * dx / dy = 1): no change, no accumulated error
    lw, es, ep = oracle.pid_update(np.log(2.0), 0.0, 0.0, 1.0, 2.0)
    assert lw == pytest.approx(np.log(2.0)) and es == 0.0
    # primal moves more than balanced: omega must decrease (Eq. pid with e_n > 0)
    lw2, es2, _ = oracle.pid_update(0.0, 0.0, 0.0, 3.0, 1.0)
    assert lw2 < 0.0 and es2 == pytest.approx(np.log(3.0))
    assert lw2 == pytest.approx(-(0.99 + 0.01) * np.log(3.0))
    # degenerate movement: skipped
    lw3, es3, _ = oracle.pid_update(0.5, 0.1, 0.0, 0.0, 1.0)
    assert lw3 == 0.5 and es3 == 0.1


def test_adaptive_inner_tolerance_monotone():
    qp = W.random_qp(n=80, m=40, n_eq=20, m_rows=20, density=0.1, seed=2)
    x, y, r, tr = oracle.solve(qp, oracle.default_params(max_iter=3000), eps_trace_len=3000)
    assert len(tr) > 10
    assert np.all(np.diff(tr) <= 0.0)
    assert np.all(tr >= 1e-9)


def test_ruiz_equilibrates():
    qp = W.random_qp(n=60, m=30, n_eq=10, m_rows=20, density=0.2, seed=1)
    qp.A = W._csr(qp.A.multiply(np.exp(np.random.default_rng(0).normal(0, 2, qp.A.shape[1]))))
    D, E = oracle.ruiz(qp, passes=30)
    Q = dense(qp.Q) * D[:, None] * D[None, :]
    A = dense(qp.A) * E[:, None] * D[None, :]
    K = np.block([[Q, A.T], [A, np.zeros((qp.m, qp.m))]])
    cn = np.max(np.abs(K), axis=0)
    assert np.all(np.abs(cn - 1.0) <= 1e-3)


@pytest.mark.parametrize("seed", [3, 4])
def test_lasso_matches_sklearn(seed):
    # LASSO as the QP of Sec. 6.4 (y = A x - b, -t <= x <= t): the oracle's x
    # attains scikit-learn's coordinate-descent optimum of ||Ax - b||^2 + lam ||x||_1
    from sklearn.linear_model import Lasso
    rows, cols = 300, 40
    qp = W.lasso_qp(rows=rows, cols=cols, density=0.1, seed=seed)
    lam = qp.meta["lam"]
    x, y, r = oracle.solve(qp, oracle.default_params(eps_tol=1e-9, max_iter=2_000_000))
    assert r["status_name"] == "OPTIMAL"
    A = qp.A[:rows, :cols].toarray()
    b = qp.lc[:rows]

    def f(w):
        return np.sum((A @ w - b) ** 2) + lam * np.sum(np.abs(w))

    ref = Lasso(alpha=lam / (2 * rows), fit_intercept=False, tol=1e-14, max_iter=10**6).fit(A, b).coef_
    assert f(x[:cols]) == pytest.approx(f(ref), rel=1e-8)
    assert r["primal_obj"] == pytest.approx(f(ref), rel=1e-8)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_factored_q_reaches_the_formed_q_optimum(seed):
    # Sec. 2.2's structured objective: Q = P + R^T R applied matrix-free must
    # reach the optimum of the same QP with Q formed explicitly (scipy product)
    qf = W.random_qp(seed=seed, factored=True)
    formed = W.QP(qf.n, qf.m, W._csr(qf.Q + qf.R.T @ qf.R), qf.A, qf.c, qf.lc, qf.uc, qf.lv, qf.uv)
    xf, yf, rf = oracle.solve(qf, oracle.default_params(eps_tol=1e-9, max_iter=2_000_000))
    x, y, r = oracle.solve(formed, oracle.default_params(eps_tol=1e-9, max_iter=2_000_000))
    assert rf["status_name"] == r["status_name"] == "OPTIMAL"
    assert rf["primal_obj"] == pytest.approx(r["primal_obj"], rel=1e-8)
    # the factored solution satisfies the formed problem's KKT conditions
    Qx = formed.Q @ xf
    rp, rd, rg, _, _ = oracle.kkt(formed.n, formed.m, xf, yf, formed.A @ xf, formed.A.T @ yf, Qx,
                                  formed.c, formed.lc, formed.uc, formed.lv, formed.uv)
    assert max(rp, rd, rg) <= 2e-9


@pytest.mark.parametrize("seed", [0, 1])
def test_factored_ruiz_equals_formed_when_RtR_is_diagonal(seed):
    # Scaling of a structured Q = P + R^T R (Sec. 2.2; the scaling itself is a
    # reading): the column maxima take the scaled diagonal of R^T R.  With one
    # nonzero per row of R, R^T R is exactly diagonal, so with P = 0 the factored
    # scaling must equal Ruiz on the explicitly formed Q = R^T R (scipy product).
    rng = np.random.default_rng(seed)
    n, m, k = 30, 12, 45
    cols = rng.integers(0, n, k)
    vals = rng.normal(size=k) * rng.uniform(0.1, 10.0, k)
    R = sp.csr_matrix((vals, (np.arange(k), cols)), shape=(k, n))
    A = sp.random(m, n, density=0.3, random_state=rng, format="csr")
    A.data = rng.normal(size=A.nnz) * 5.0
    c = rng.normal(size=n)
    lv, uv = -np.ones(n), np.ones(n)
    lc, uc = -np.ones(m), np.ones(m)
    formed = W.QP(n, m, W._csr(R.T @ R), A, c, lc, uc, lv, uv)
    factored = W.QP(n, m, None, A, c, lc, uc, lv, uv, R=R)
    Df, Ef = oracle.ruiz(factored, 10)
    D, E = oracle.ruiz(formed, 10)
    np.testing.assert_allclose(Df, D, rtol=1e-14)
    np.testing.assert_allclose(Ef, E, rtol=1e-14)
    # and the reading is not vacuous: without R the scaling differs
    Dn, _ = oracle.ruiz(W.QP(n, m, None, A, c, lc, uc, lv, uv), 10)
    assert np.max(np.abs(Dn - D) / D) > 1e-3


def _ulp_sensitivity(qp, steps=100):
    _, _, r0 = oracle.solve(qp, oracle.default_params(max_iter=1))
    eta = r0["eta"]
    x1, y1, _ = oracle.solve(qp, oracle.default_params(max_iter=steps, eta_override=eta))
    x2, y2, _ = oracle.solve(qp, oracle.default_params(max_iter=steps, eta_override=eta * (1 + 2e-16)))
    return max(np.max(np.abs(x1 - x2)) / (1 + np.max(np.abs(x1))),
               np.max(np.abs(y1 - y2)) / (1 + np.max(np.abs(y1))))


def test_iterate_test_instances_amplify_rounding_little():
    # The GPU iterate tests compare 100 steps at 1e-10.  That is meaningful only
    # where the method itself does not amplify rounding that far: on each
    # instance they use, a one-ulp change of eta moves the oracle's own iterates
    # by less than 1e-11 (the factored seed 6 moves by ~1e-9 and is not used).
    for qp in (W.random_qp(seed=3), W.random_qp(seed=5), W.random_qp(seed=1, factored=True),
               W.random_qp(seed=4, factored=True)):
        assert _ulp_sensitivity(qp) < 1e-11
    assert _ulp_sensitivity(W.random_qp(seed=6, factored=True)) > 1e-10


def test_golden_closed_forms():
    # tests/golden/closed_form_qps.json: QPs solved by hand from the optimality
    # conditions (equality-constrained, separable box, one active row)
    from conftest import golden_closed_form_qps
    for qp, xs, fs in golden_closed_form_qps():
        x, y, r = oracle.solve(qp, oracle.default_params(eps_tol=1e-10, max_iter=1_000_000))
        assert r["status_name"] == "OPTIMAL", (qp.name, r)
        np.testing.assert_allclose(x, xs, atol=1e-8, err_msg=qp.name)
        assert r["primal_obj"] == pytest.approx(fs, rel=1e-9, abs=1e-9), qp.name


def test_golden_step_trace_inner_tolerance_and_halpern():
    # tests/golden/step_trace_1d.json: the first four steps on a one-variable QP,
    # derived by hand in exact fractions.  eps_k pins the adaptive inner
    # tolerance of Sec. 3.3 (the gamma * omega * movement / tau term, the
    # running min and the first tolerance); T(z_k) after K = 2..4 steps depends
    # on the reflected Halpern weights (k+1)/(k+2), 1/(k+2) and theta of
    # Sec. 3.1 through the iterate z_k it is taken at.
    from conftest import golden_step_trace
    g = golden_step_trace()
    for case in g["cases"]:
        prm = dict(g["settings"], theta=case["theta"])
        _, _, r, tr = oracle.solve(g["qp"], oracle.default_params(max_iter=len(case["eps_trace"]), **prm),
                                   x0=g["x0"], y0=g["y0"], eps_trace_len=len(case["eps_trace"]))
        np.testing.assert_allclose(tr, case["eps_trace"], rtol=1e-14, atol=0)
        for K, (xs, ys) in case["outputs"].items():
            x, y, r = oracle.solve(g["qp"], oracle.default_params(max_iter=K, **prm), x0=g["x0"], y0=g["y0"])
            assert r["status_name"] == "ITERATION_LIMIT" and r["iterations"] == K
            np.testing.assert_allclose(x, xs, rtol=1e-14, err_msg=f"theta={case['theta']} K={K}")
            np.testing.assert_allclose(y, ys, rtol=1e-14, err_msg=f"theta={case['theta']} K={K}")


def test_golden_gap_term():
    # Sec. 4.2 at a primal- and dual-feasible point that is not optimal: only
    # the gap term is nonzero, so its numerator (x^T Q x + c^T x + p(-r) + p(y))
    # and denominator are pinned separately from the other residuals
    from conftest import golden_step_trace
    gp = golden_step_trace()["gap"]
    qp, x, y, e = gp["qp"], gp["x"], gp["y"], gp["expect"]
    Q, A = dense(qp.Q), dense(qp.A)
    rp, rd, rg, pobj, dobj = oracle.kkt(qp.n, qp.m, x, y, A @ x, A.T @ y, Q @ x, qp.c, qp.lc, qp.uc,
                                        qp.lv, qp.uv)
    assert rp == e["r_primal"] and rd == e["r_dual"]
    assert rg == pytest.approx(e["r_gap"], rel=1e-15)
    assert pobj == pytest.approx(e["primal_obj"], abs=1e-15)
    assert dobj == pytest.approx(e["dual_obj"], rel=1e-15)


@pytest.mark.parametrize("seed", [0, 1])
def test_certificate_checks_accept_oracle_rays_and_reject_flipped_ones(seed):
    """The certificate checks the GPU tests apply (tests/certificates.py) accept
    the oracle's rays, whose conditions the two tests above verify one by one,
    and reject the same rays with the sign flipped."""
    from certificates import check_dual_ray, check_primal_ray
    qp = W.infeasible_qp(n=8, m=4, seed=seed)
    _, y, r = oracle.solve(qp, oracle.default_params(max_iter=200000))
    assert r["status_name"] == "PRIMAL_INFEASIBLE"
    check_primal_ray(qp, y)
    with pytest.raises(AssertionError):
        check_primal_ray(qp, -y)
    qp = W.unbounded_qp(n=6, seed=seed)
    d, _, r = oracle.solve(qp, oracle.default_params(max_iter=200000))
    assert r["status_name"] == "DUAL_INFEASIBLE"
    check_dual_ray(qp, d)
    with pytest.raises(AssertionError):
        check_dual_ray(qp, -d)

"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bars (written in each test):
* final results: the oracle's independent KKT evaluator (Sec. 4.2) applied to
  the GPU solution is <= eps_tol, and the relative objective difference to the
  oracle's solve is <= 1e-6;
* FP64 iterates: after N = 1 .. 100 PDHG steps the GPU iterate equals the
  oracle's to 1e-10 relative (same eta, passed to the oracle);
* setup: Ruiz vectors to 1e-13, ||A|| to 1e-6.
"""
import numpy as np
import pytest

import oracle
from paper_2602_23967_b300 import pdhcg
from paper_2602_23967_b300 import workloads as W
from certificates import check_dual_ray, check_primal_ray

pytestmark = pytest.mark.gpu


def kkt_of(qp, x, y):
    Q = qp.Q
    Qx = Q @ x if Q is not None else np.zeros(qp.n)
    return oracle.kkt(qp.n, qp.m, x, y, qp.A @ x, qp.A.T @ y, Qx, qp.c, qp.lc, qp.uc, qp.lv, qp.uv)


def rel(a, b):
    return abs(a - b) / (1.0 + abs(b))


def gpu_solve(qp, **kw):
    prob = pdhcg.Problem(qp, pdhcg.default_params(**kw))
    try:
        x, y, r = prob.solve()
        eta, _ = prob.eta()
    finally:
        prob.close()
    return x, y, r, eta


def check_optimal_parity(qp, eps=1e-6, precision="fp64", obj_tol=1e-6, **kw):
    x, y, r, _ = gpu_solve(qp, eps_tol=eps, precision=precision, **kw)
    assert r["status_name"] == "OPTIMAL", r
    rp, rd, rg, pobj, _ = kkt_of(qp, x, y)
    # the device's stopping test evaluates the residuals with FP64-accurate
    # products in every precision mode, so the independent FP64 evaluation of
    # the returned point meets the requested tolerance itself
    assert max(rp, rd, rg) <= eps, (rp, rd, rg)
    xo, yo, ro = oracle.solve(qp, oracle.default_params(eps_tol=eps, **{k: v for k, v in kw.items()
                                                                       if k in ("inner",)}))
    assert ro["status_name"] == "OPTIMAL"
    assert rel(pobj, ro["primal_obj"]) <= obj_tol, (pobj, ro["primal_obj"])
    return r, ro


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_random_qp_fp64(seed):
    r, ro = check_optimal_parity(W.random_qp(seed=seed))
    # same algorithm, same decisions: iteration counts agree closely
    assert abs(r["iterations"] - ro["iterations"]) <= 64


def test_setup_matches_oracle():
    qp = W.random_qp(seed=3)
    prob = pdhcg.Problem(qp, pdhcg.default_params())
    D, E = prob.scaling()
    eta, normA = prob.eta()
    prob.close()
    Do, Eo = oracle.ruiz(qp, passes=10)
    assert np.max(np.abs(D - Do) / Do) <= 1e-13
    assert np.max(np.abs(E - Eo) / Eo) <= 1e-13
    import scipy.sparse as sp
    As = sp.diags(Eo) @ qp.A @ sp.diags(Do)
    ref = np.linalg.norm(As.toarray(), 2)
    assert normA == pytest.approx(ref, rel=1e-6)


@pytest.mark.parametrize("group_blocks", [1, 7])
@pytest.mark.parametrize("N", [1, 2, 5, 17, 64, 100])
def test_fp64_iterates_first_100(N, group_blocks):
    qp = W.random_qp(seed=4)
    x, y, r, eta = gpu_solve(qp, max_iter=N, group_blocks=group_blocks)
    xo, yo, ro = oracle.solve(qp, oracle.default_params(max_iter=N, eta_override=eta))
    assert r["iterations"] == ro["iterations"] == N
    assert r["inner_iterations"] == ro["inner_iterations"]
    assert np.max(np.abs(x - xo)) <= 1e-10 * (1 + np.max(np.abs(xo)))
    assert np.max(np.abs(y - yo)) <= 1e-10 * (1 + np.max(np.abs(yo)))


@pytest.mark.parametrize("group_blocks", [3, 16, 0])
def test_multi_cta_iterates_mid_size(group_blocks):
    # several partitions, ragged tails, BB inner solver on a non-diagonal Q
    qp = W.large_sparse_qp(n=6000, m=3000, seed=1)
    N = 100
    x, y, r, eta = gpu_solve(qp, max_iter=N, group_blocks=group_blocks)
    xo, yo, ro = oracle.solve(qp, oracle.default_params(max_iter=N, eta_override=eta))
    assert r["inner_iterations"] == ro["inner_iterations"]
    assert np.max(np.abs(x - xo)) <= 1e-10 * (1 + np.max(np.abs(xo)))
    assert np.max(np.abs(y - yo)) <= 1e-10 * (1 + np.max(np.abs(yo)))


def test_cg_inner_solver_iterates():
    # every variable free -> CG (Sec. 2.2 / Sec. 3.3)
    qp = W.equality_qp(n=120, m=40, seed=2)
    for N in (3, 64, 100):
        x, y, r, eta = gpu_solve(qp, max_iter=N)
        xo, yo, ro = oracle.solve(qp, oracle.default_params(max_iter=N, eta_override=eta))
        assert r["inner_method"] == 2 and ro["inner_method"] == 2
        assert r["inner_iterations"] == ro["inner_iterations"]
        assert np.max(np.abs(x - xo)) <= 1e-10 * (1 + np.max(np.abs(xo)))


def test_equality_qp_matches_dense_kkt():
    qp = W.equality_qp(n=30, m=10, seed=0)
    Q, A = qp.Q.toarray(), qp.A.toarray()
    K = np.block([[Q, A.T], [A, np.zeros((qp.m, qp.m))]])
    sol = np.linalg.solve(K, np.concatenate([-qp.c, qp.lc]))
    x, y, r, _ = gpu_solve(qp, eps_tol=1e-10)
    assert r["status_name"] == "OPTIMAL"
    assert np.linalg.norm(x - sol[:qp.n]) <= 1e-7 * (1 + np.linalg.norm(sol[:qp.n]))


def test_mpc_fp64_and_fp32():
    qp = W.mpc_qp(seed=11)
    check_optimal_parity(qp)
    # FP32 iterates stall near 1e-6 relative KKT on this class; 1e-5 is the FP32 bar,
    # FP32 matrix values with FP64 vectors (mixed) reach 1e-6.
    check_optimal_parity(qp, precision="fp32", eps=1e-5, obj_tol=1e-5, max_iter=200000)
    check_optimal_parity(qp, precision="mixed", max_iter=200000)


def test_factor_portfolio_with_long_row_multi_cta():
    # the budget row 1^T x has 20000 nonzeros and runs on a whole CTA
    qp = W.factor_portfolio(n=20000, k=50, seed=0)
    check_optimal_parity(qp, group_blocks=16)
    x, y, r, eta = gpu_solve(qp, max_iter=100, group_blocks=16)
    xo, yo, ro = oracle.solve(qp, oracle.default_params(max_iter=100, eta_override=eta))
    assert np.max(np.abs(x - xo)) <= 1e-10 * (1 + np.max(np.abs(xo)))
    assert np.max(np.abs(y - yo)) <= 1e-10 * (1 + np.max(np.abs(yo)))


def test_large_sparse_mid_size_fp64_mixed():
    # FP32 iterates stall above 1e-5 on this class; FP32 matrix values with FP64
    # vectors (mixed) reach the 1e-6 bar
    qp = W.large_sparse_qp(n=20000, m=10000, seed=0)
    check_optimal_parity(qp)
    check_optimal_parity(qp, precision="mixed", max_iter=200000)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_primal_infeasible_detected(seed):
    qp = W.infeasible_qp(n=8, m=4, seed=seed)
    x, y, r, _ = gpu_solve(qp)
    assert r["status_name"] == "PRIMAL_INFEASIBLE"
    # the whole Farkas certificate of Sec. 5.1: y in the rows' sign cone,
    # A^T y in R, p(-A^T y) + p(y) < 0
    check_primal_ray(qp, y)


@pytest.mark.parametrize("seed", [0, 1])
def test_dual_infeasible_detected(seed):
    qp = W.unbounded_qp(n=6, seed=seed)
    x, y, r, _ = gpu_solve(qp)
    assert r["status_name"] == "DUAL_INFEASIBLE"
    # the whole certificate of Sec. 5.2: c^T d < 0, Q d = 0, d in Recc(X), A d in Recc(S)
    check_dual_ray(qp, x)


def test_edge_no_constraints_and_lp():
    rng = np.random.default_rng(0)
    n = 37
    base = W.random_qp(n=n, m=10, n_eq=5, m_rows=10, density=0.3, seed=7)
    import scipy.sparse as sp
    qp = W.QP(n, 0, base.Q, W._csr(sp.csr_matrix((0, n))), base.c, np.zeros(0), np.zeros(0),
              base.lv, base.uv, name="no_rows")
    x, y, r, _ = gpu_solve(qp, eps_tol=1e-8)
    xo, yo, ro = oracle.solve(qp, oracle.default_params(eps_tol=1e-8))
    assert r["status_name"] == ro["status_name"] == "OPTIMAL"
    assert rel(r["primal_obj"], ro["primal_obj"]) <= 1e-7
    lp = W.QP(base.n, base.m, None, base.A, base.c, base.lc, base.uc, base.lv, base.uv, name="lp")
    x, y, r, _ = gpu_solve(lp, eps_tol=1e-7)
    xo, yo, ro = oracle.solve(lp, oracle.default_params(eps_tol=1e-7))
    assert r["status_name"] == ro["status_name"] == "OPTIMAL"
    assert rel(r["primal_obj"], ro["primal_obj"]) <= 1e-6


def test_single_variable():
    import scipy.sparse as sp
    qp = W.QP(1, 1, W._csr(sp.csr_matrix(np.array([[2.0]]))), W._csr(sp.csr_matrix(np.array([[1.0]]))),
              np.array([-3.0]), np.array([-np.inf]), np.array([1.0]), np.array([-5.0]), np.array([5.0]))
    x, y, r, _ = gpu_solve(qp, eps_tol=1e-9)
    assert r["status_name"] == "OPTIMAL"
    assert x[0] == pytest.approx(1.0, abs=1e-8)     # min x^2 - 3x s.t. x <= 1


def test_batch_equals_single_solves():
    qps = [W.mpc_qp(seed=100 + i) for i in range(12)] + [W.random_qp(seed=20 + i) for i in range(4)]
    probs = [pdhcg.Problem(q, pdhcg.default_params()) for q in qps]
    try:
        batch = pdhcg.solve_batch(probs)
        for p, (xb, yb, rb) in zip(probs, batch):
            xs, ys, rs = p.solve()
            assert rb["status_name"] == rs["status_name"] == "OPTIMAL"
            assert rb["iterations"] == rs["iterations"]
            assert np.max(np.abs(xb - xs)) <= 1e-12 * (1 + np.max(np.abs(xs)))
    finally:
        for p in probs:
            p.close()


def test_create_batch_matches_single_create():
    qps = [W.mpc_qp(seed=200 + i) for i in range(6)] + [W.random_qp(seed=40 + i) for i in range(3)]
    probs = pdhcg.create_batch(qps, pdhcg.default_params())
    try:
        for q, p in zip(qps, probs):
            single = pdhcg.Problem(q, pdhcg.default_params())
            xs, ys, rs = single.solve()
            eta_s = single.eta()
            single.close()
            xb, yb, rb = p.solve()
            assert p.eta() == pytest.approx(eta_s, rel=1e-12)
            assert rb["status_name"] == rs["status_name"] == "OPTIMAL"
            assert np.max(np.abs(xb - xs)) <= 1e-12 * (1 + np.max(np.abs(xs)))
        out = pdhcg.solve_batch(probs)
        assert all(r["status_name"] == "OPTIMAL" for _, _, r in out)
    finally:
        for p in probs:
            p.close()


def test_warm_start_from_solution_is_immediate():
    qp = W.random_qp(seed=9)
    prob = pdhcg.Problem(qp, pdhcg.default_params(eps_tol=1e-7))
    try:
        x, y, r = prob.solve()
        x2, y2, r2 = prob.solve(x0=x, y0=y)
        assert r2["status_name"] == "OPTIMAL"
        assert r2["iterations"] <= r["iterations"]
    finally:
        prob.close()


@pytest.mark.parametrize("precision", ["fp64", "dfloat"])
def test_lasso_matches_oracle(precision):
    # LASSO in the QP form of Sec. 6.4 (diagonal Q, free variables, one-sided rows)
    qp = W.lasso_qp(rows=4000, cols=400, density=0.01, seed=2)
    check_optimal_parity(qp, precision=precision, max_iter=500000)


def lifted(qp):
    """The same QP with every finite variable bound as a row e_j^T x of A (reading
    D1's CG_LIFTED variant), built here independently of the library."""
    import scipy.sparse as sp
    B = [j for j in range(qp.n) if np.isfinite(qp.lv[j]) or np.isfinite(qp.uv[j])]
    E = sp.csr_matrix((np.ones(len(B)), (np.arange(len(B)), B)), shape=(len(B), qp.n))
    A = W._csr(sp.vstack([qp.A, E]))
    lc = np.concatenate([qp.lc, qp.lv[B]])
    uc = np.concatenate([qp.uc, qp.uv[B]])
    free = np.full(qp.n, np.inf)
    return W.QP(qp.n, qp.m + len(B), qp.Q, A, qp.c, lc, uc, -free, free, name=qp.name + "_lifted")


@pytest.mark.parametrize("N", [1, 17, 100])
def test_cg_lifted_iterates_match_oracle_on_lifted_qp(N):
    qp = W.random_qp(seed=4)
    x, y, r, eta = gpu_solve(qp, max_iter=N, inner="cg_lifted")
    assert r["inner_method"] == 2 and len(y) == qp.m          # CG; only the original rows' duals
    lq = lifted(qp)
    xo, yo, ro = oracle.solve(lq, oracle.default_params(max_iter=N, eta_override=eta, inner="cg"))
    assert r["inner_iterations"] == ro["inner_iterations"]
    assert np.max(np.abs(x - xo)) <= 1e-10 * (1 + np.max(np.abs(xo)))
    assert np.max(np.abs(y - yo[: qp.m])) <= 1e-10 * (1 + np.max(np.abs(yo)))


@pytest.mark.parametrize("precision", ["fp64", "dfloat"])
@pytest.mark.parametrize("seed", [0, 1])
def test_cg_lifted_solves_the_original_qp(precision, seed):
    qp = W.random_qp(seed=seed)
    # the stopping test is on the lifted problem, whose relative residuals are
    # normalised by its own (larger) bound vector; 1e-7 there meets 1e-6 on the original
    x, y, r, _ = gpu_solve(qp, eps_tol=1e-7, precision=precision, inner="cg_lifted", max_iter=500000)
    assert r["status_name"] == "OPTIMAL", r
    # the bounds are rows now: satisfied to the relative primal tolerance of Sec. 4.2
    lq = lifted(qp)
    scale = 1 + max(np.max(np.abs(lq.lc[np.isfinite(lq.lc)])), np.max(np.abs(lq.uc[np.isfinite(lq.uc)])))
    assert np.max(np.maximum(qp.lv - x, x - qp.uv)) <= 1e-6 * scale
    # the original rows' duals plus the implicit bound multipliers satisfy the
    # original KKT conditions (the bound multipliers are the reduced costs)
    rp, rd, rg, pobj, _ = kkt_of(qp, x, y)
    assert max(rp, rd, rg) <= 1e-6, (rp, rd, rg)
    _, _, ro = oracle.solve(qp, oracle.default_params(eps_tol=1e-6))
    assert rel(pobj, ro["primal_obj"]) <= 1e-6, (pobj, ro["primal_obj"])


@pytest.mark.parametrize("group_blocks", [1, 7])
@pytest.mark.parametrize("N", [1, 17, 100])
def test_structured_q_iterates_match_oracle(N, group_blocks):
    # Q = P + R^T R applied as P v + R^T (R v) on both sides (Sec. 2.2)
    qp = W.random_qp(seed=4, factored=True)
    x, y, r, eta = gpu_solve(qp, max_iter=N, group_blocks=group_blocks)
    xo, yo, ro = oracle.solve(qp, oracle.default_params(max_iter=N, eta_override=eta))
    assert r["iterations"] == ro["iterations"] == N
    assert r["inner_iterations"] == ro["inner_iterations"]
    assert np.max(np.abs(x - xo)) <= 1e-10 * (1 + np.max(np.abs(xo)))
    assert np.max(np.abs(y - yo)) <= 1e-10 * (1 + np.max(np.abs(yo)))


@pytest.mark.parametrize("inner", ["auto", "cg_lifted"])
@pytest.mark.parametrize("precision", ["fp64", "dfloat"])
def test_structured_q_solves_to_the_formed_optimum(precision, inner):
    qf = W.random_qp(seed=1, factored=True)
    formed = W.QP(qf.n, qf.m, W._csr(qf.Q + qf.R.T @ qf.R), qf.A, qf.c, qf.lc, qf.uc, qf.lv, qf.uv)
    # CG_LIFTED stops on the lifted problem's residuals (see above): 1e-7 there
    x, y, r, _ = gpu_solve(qf, eps_tol=1e-6 if inner == "auto" else 1e-7, precision=precision, inner=inner,
                           max_iter=500000)
    assert r["status_name"] == "OPTIMAL", r
    rp, rd, rg, pobj, _ = kkt_of(formed, x, y)
    assert max(rp, rd, rg) <= 1e-6, (rp, rd, rg)
    _, _, ro = oracle.solve(formed, oracle.default_params(eps_tol=1e-6))
    assert rel(pobj, ro["primal_obj"]) <= 1e-6, (pobj, ro["primal_obj"])


def test_structured_q_large_factor_multi_cta():
    # a large factor (k = 2000 rows of ~50 entries) on several CTAs: iterates vs oracle
    import scipy.sparse as sp
    rng = np.random.default_rng(8)
    base = W.large_sparse_qp(n=20000, m=10000, seed=2)
    R = W._csr(sp.random(2000, base.n, density=50 / base.n, random_state=rng, format="csr"))
    qp = W.QP(base.n, base.m, base.Q, base.A, base.c, base.lc, base.uc, base.lv, base.uv, R=R)
    x, y, r, eta = gpu_solve(qp, max_iter=64, group_blocks=0)
    xo, yo, ro = oracle.solve(qp, oracle.default_params(max_iter=64, eta_override=eta))
    assert r["inner_iterations"] == ro["inner_iterations"]
    assert np.max(np.abs(x - xo)) <= 1e-10 * (1 + np.max(np.abs(xo)))
    assert np.max(np.abs(y - yo)) <= 1e-10 * (1 + np.max(np.abs(yo)))


def test_mixed_batch_of_plain_and_structured_problems():
    # one pooled launch holding plain problems and structured ones (Q = P + R^T R,
    # Sec. 2.2) runs the structured kernel variant for all of them: FP64 iterates
    # after 100 steps equal the oracle's for both kinds, and a double-float solve
    # of the same batch reaches the oracle's optimum.  (The factored seed 6 is not
    # used: there the oracle's own 100-step iterates move by 1e-9 when eta changes
    # by one ulp, so no second implementation can agree with it to 1e-10.)
    qps = [W.random_qp(seed=3), W.random_qp(seed=1, factored=True), W.random_qp(seed=5),
           W.random_qp(seed=4, factored=True)]
    N = 100
    probs = [pdhcg.Problem(q, pdhcg.default_params(max_iter=N)) for q in qps]
    try:
        out = pdhcg.solve_batch(probs)
        etas = [p.eta()[0] for p in probs]
    finally:
        for p in probs:
            p.close()
    for q, (x, y, r), eta in zip(qps, out, etas):
        xo, yo, ro = oracle.solve(q, oracle.default_params(max_iter=N, eta_override=eta))
        assert r["iterations"] == ro["iterations"] == N
        assert r["inner_iterations"] == ro["inner_iterations"]
        assert np.max(np.abs(x - xo)) <= 1e-10 * (1 + np.max(np.abs(xo)))
        assert np.max(np.abs(y - yo)) <= 1e-10 * (1 + np.max(np.abs(yo)))
    probs = [pdhcg.Problem(q, pdhcg.default_params(precision="dfloat", eps_tol=1e-6, max_iter=500000))
             for q in qps]
    try:
        out = pdhcg.solve_batch(probs)
    finally:
        for p in probs:
            p.close()
    for q, (x, y, r) in zip(qps, out):
        assert r["status_name"] == "OPTIMAL", r
        formed = q if q.R is None else W.QP(q.n, q.m, W._csr(q.Q + q.R.T @ q.R), q.A, q.c, q.lc, q.uc,
                                             q.lv, q.uv)
        rp, rd, rg, pobj, _ = kkt_of(formed, x, y)
        assert max(rp, rd, rg) <= 1e-6, (rp, rd, rg)
        _, _, ro = oracle.solve(formed, oracle.default_params(eps_tol=1e-6))
        assert rel(pobj, ro["primal_obj"]) <= 1e-6, (pobj, ro["primal_obj"])


@pytest.mark.parametrize("precision", ["fp64", "dfloat"])
def test_golden_closed_forms_on_gpu(precision):
    # the hand-derived QPs of tests/golden/closed_form_qps.json on the CUDA path
    from conftest import golden_closed_form_qps
    for qp, xs, fs in golden_closed_form_qps():
        x, y, r, _ = gpu_solve(qp, eps_tol=1e-9, precision=precision, max_iter=1_000_000)
        assert r["status_name"] == "OPTIMAL", (qp.name, r)
        np.testing.assert_allclose(x, xs, atol=1e-7, err_msg=qp.name)
        assert rel(r["primal_obj"], fs) <= 1e-8, (qp.name, r["primal_obj"], fs)


@pytest.mark.parametrize("precision", ["fp64", "dfloat"])
def test_golden_step_trace_on_gpu(precision):
    # tests/golden/step_trace_1d.json on the CUDA path: T(z) after K = 1..4
    # steps, derived by hand, depends on the reflected Halpern weights and theta
    # (Sec. 3.1), the step sizes tau = eta/omega and sigma = eta*omega (Sec. 3.2)
    # and the dual update; FP64 to 1e-14, double-float vectors to 1e-12
    from conftest import golden_step_trace
    g = golden_step_trace()
    tol = 1e-14 if precision == "fp64" else 1e-12
    for case in g["cases"]:
        for K, (xs, ys) in case["outputs"].items():
            prob = pdhcg.Problem(g["qp"], pdhcg.default_params(precision=precision, max_iter=K,
                                                               theta=case["theta"], **g["settings"]))
            try:
                x, y, r = prob.solve(x0=g["x0"], y0=g["y0"])
            finally:
                prob.close()
            assert r["status_name"] == "ITERATION_LIMIT" and r["iterations"] == K, r
            np.testing.assert_allclose(x, xs, rtol=tol, err_msg=f"theta={case['theta']} K={K}")
            np.testing.assert_allclose(y, ys, rtol=tol, err_msg=f"theta={case['theta']} K={K}")


def test_batch_runs_large_instances_on_groups():
    # a batch mixing small instances (pool CTAs) with large ones, which
    # pdhcg_solve_batch runs on multi-CTA groups in the same cooperative
    # launch: FP64 iterates after 100 steps equal the oracle's for every
    # instance, and a double-float solve of the batch reaches the oracle's
    # KKT bar and objective
    qps = [W.mpc_qp(seed=600 + i) for i in range(4)] + [W.random_qp(seed=3)]
    qps += [W.large_sparse_qp(n=20000, m=10000, seed=3), W.factor_portfolio(n=30000, k=300, seed=4)]
    N = 100
    probs = [pdhcg.Problem(q, pdhcg.default_params(max_iter=N)) for q in qps]
    try:
        out = pdhcg.solve_batch(probs)
        etas = [p.eta()[0] for p in probs]
    finally:
        for p in probs:
            p.close()
    for q, (x, y, r), eta in zip(qps, out, etas):
        xo, yo, ro = oracle.solve(q, oracle.default_params(max_iter=N, eta_override=eta))
        assert r["iterations"] == ro["iterations"] == N
        assert r["inner_iterations"] == ro["inner_iterations"], q.name
        assert np.max(np.abs(x - xo)) <= 1e-10 * (1 + np.max(np.abs(xo))), q.name
        assert np.max(np.abs(y - yo)) <= 1e-10 * (1 + np.max(np.abs(yo))), q.name
    probs = pdhcg.create_batch(qps, pdhcg.default_params(precision="dfloat", eps_tol=1e-6, max_iter=400000))
    try:
        out = pdhcg.solve_batch(probs)
    finally:
        for p in probs:
            p.close()
    for q, (x, y, r) in zip(qps, out):
        assert r["status_name"] == "OPTIMAL", (q.name, r)
        rp, rd, rg, pobj, _ = kkt_of(q, x, y)
        assert max(rp, rd, rg) <= 1e-6, (q.name, rp, rd, rg)
        _, _, ro = oracle.solve(q, oracle.default_params(eps_tol=1e-6))
        assert rel(pobj, ro["primal_obj"]) <= 1e-6, (q.name, pobj, ro["primal_obj"])

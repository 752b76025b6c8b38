"""Seeded synthetic QP generators shared by the tests, the benchmark and the oracle side.

This module only draws random problem data and assembles it into CSR; it holds
none of the solver's arithmetic.  Every generator is deterministic in its seed
(``numpy.random.default_rng``).

Problem form (Sec. 2, Eq. QP):  min 1/2 x^T Q x + c^T x  s.t.  lc <= A x <= uc,
lv <= x <= uv, with +-inf marking an absent bound and Q stored as a full
symmetric CSR matrix (or None for Q = 0).

Workloads, with the shapes, value distributions and structure of the paper's
problem classes (random sparse QPs, factor-model portfolios (Sec. 2.2), large
sparse instances with skewed column degrees, MPC batches, LASSO (Sec. 6.3)):

* ``random_qp``          tiny random convex QP (n=200, m=100, 50 equalities)
* ``factor_portfolio``   factor-model portfolio QP, y = F^T x, diagonal Q
* ``large_sparse_qp``    diagonally dominant sparse Q, power-law column degrees in A
* ``mpc_qp`` / ``mpc_batch``  linear MPC with 12 states and 4 inputs, horizon T
* ``serving_trace``      Poisson arrival trace over a mix of the above
* ``lasso_qp``           LASSO reformulated as a QP (Sec. 6.3)
* small hand-made instances for pins: equality-only, infeasible, unbounded
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

INF = np.inf


@dataclass
class QP:
    n: int
    m: int
    Q: sp.csr_matrix | None
    A: sp.csr_matrix
    c: np.ndarray
    lc: np.ndarray
    uc: np.ndarray
    lv: np.ndarray
    uv: np.ndarray
    name: str = "qp"
    meta: dict = field(default_factory=dict)
    # structured objective (Sec. 2.2): when set, the quadratic term is Q + R^T R
    # with Q holding the sparse part P and R (k x n) the low-rank factor
    R: sp.csr_matrix | None = None

    def nnz(self) -> int:
        return int(self.A.nnz + (self.Q.nnz if self.Q is not None else 0))


def _csr(M, shape=None) -> sp.csr_matrix:
    M = sp.csr_matrix(M, shape=shape) if shape is not None else sp.csr_matrix(M)
    M.sum_duplicates()
    M.sort_indices()
    M.data = M.data.astype(np.float64)
    return M


def _sprandn(rng, rows, cols, density, scale=1.0):
    """Random sparse matrix with uniformly placed nonzeros, entries N(0, scale^2)."""
    nnz = int(round(rows * cols * density))
    if nnz == 0:
        return _csr(sp.csr_matrix((rows, cols)))
    flat = rng.choice(rows * cols, size=nnz, replace=False) if rows * cols < 50_000_000 else \
        np.unique(rng.integers(0, rows * cols, size=nnz, dtype=np.int64))
    r = flat // cols
    c = flat % cols
    v = rng.standard_normal(len(flat)) * scale
    return _csr(sp.coo_matrix((v, (r, c)), shape=(rows, cols)))


def _sprandn_rowdeg(rng, rows, cols, per_row, scale=1.0):
    """Sparse matrix with ~per_row nonzeros per row, uniform columns (duplicates merged away)."""
    nnz = int(rows * per_row)
    r = np.repeat(np.arange(rows, dtype=np.int64), per_row) if float(per_row).is_integer() else \
        rng.integers(0, rows, size=nnz)
    c = rng.integers(0, cols, size=len(r))
    key = np.unique(r * cols + c)
    r, c = key // cols, key % cols
    v = rng.standard_normal(len(key)) * scale
    return _csr(sp.coo_matrix((v, (r, c)), shape=(rows, cols)))


def random_qp(n=200, m=100, n_eq=50, density=0.05, m_rows=50, seed=0, box=10.0,
              per_row=None, infeasible=False, factored=False) -> QP:
    """Tiny random convex QP: Q = M^T M + 0.01 I, M m_rows x n, A m x n, both at ``density``
    (or ~``per_row`` nonzeros per row when given), entries N(0,1); c ~ N(0,1); box [-box, box].
    Feasible by construction: x0 ~ U(-5,5), b_eq = A_eq x0, b_ineq = A_ineq x0 + U(0,1).
    ``infeasible`` duplicates one equality row with right-hand side + 1.
    ``factored`` returns the same objective as P = 0.01 I plus the factor R = M
    (Sec. 2.2's structured Q = P + R^T R) instead of the formed M^T M + 0.01 I."""
    rng = np.random.default_rng(seed)
    if per_row is None:
        M = _sprandn(rng, m_rows, n, density)
        A = _sprandn(rng, m, n, density)
    else:
        M = _sprandn_rowdeg(rng, m_rows, n, per_row)
        A = _sprandn_rowdeg(rng, m, n, per_row)
    Q = _csr((M.T @ M) + 0.01 * sp.identity(n, format="csr"))
    c = rng.standard_normal(n)
    x0 = rng.uniform(-5.0, 5.0, n)
    Ax0 = A @ x0
    lc = np.empty(m)
    uc = np.empty(m)
    lc[:n_eq] = Ax0[:n_eq]
    uc[:n_eq] = Ax0[:n_eq]
    lc[n_eq:] = -INF
    uc[n_eq:] = Ax0[n_eq:] + rng.uniform(0.0, 1.0, m - n_eq)
    lv = np.full(n, -box)
    uv = np.full(n, box)
    name = f"random_qp_n{n}_s{seed}"
    if infeasible and n_eq > 0:
        row = A[0:1]
        A = _csr(sp.vstack([A, row]))
        lc = np.append(lc, lc[0] + 1.0)
        uc = np.append(uc, uc[0] + 1.0)
        m += 1
        name += "_infeasible"
    if factored:
        return QP(n, m, _csr(0.01 * sp.identity(n, format="csr")), A, c, lc, uc, lv, uv,
                  name=name + "_factored", meta={"x_feasible": x0}, R=_csr(M))
    return QP(n, m, Q, A, c, lc, uc, lv, uv, name=name, meta={"x_feasible": x0})


def factor_portfolio(n=100_000, k=1_000, density=0.01, seed=0) -> QP:
    """Factor-model portfolio: variables (x in R^n, y in R^k), objective
    x^T D x + y^T y - mu^T x = 1/2 z^T diag(2D, 2I) z + (-mu, 0)^T z,
    constraints F^T x - y = 0 and 1^T x = 1, bounds 0 <= x <= 0.01, y free.
    F is n x k at ``density``, entries N(0, 0.1^2); D ~ U(0.01, 0.1); mu ~ N(0.05, 0.02^2)."""
    rng = np.random.default_rng(seed)
    F = _sprandn(rng, n, k, density, scale=0.1)
    D = rng.uniform(0.01, 0.1, n)
    mu = rng.normal(0.05, 0.02, n)
    N = n + k
    Q = _csr(sp.diags(np.concatenate([2.0 * D, 2.0 * np.ones(k)])).tocsr())
    top = sp.hstack([F.T, -sp.identity(k)])
    bottom = sp.hstack([sp.csr_matrix(np.ones((1, n))), sp.csr_matrix((1, k))])
    A = _csr(sp.vstack([top, bottom]))
    lc = np.concatenate([np.zeros(k), [1.0]])
    uc = lc.copy()
    c = np.concatenate([-mu, np.zeros(k)])
    cap = 0.01 if n >= 200 else 2.0 / n
    lv = np.concatenate([np.zeros(n), np.full(k, -INF)])
    uv = np.concatenate([np.full(n, cap), np.full(k, INF)])
    return QP(N, k + 1, Q, A, c, lc, uc, lv, uv, name=f"factor_portfolio_n{n}_k{k}_s{seed}")


def large_sparse_qp(n=2_000_000, m=1_000_000, eq_frac=0.3, seed=0, q_upper_per_row=4.5,
                    pareto_shape=1.5, deg_min=4.0 / 3.0, box=100.0) -> QP:
    """Large sparse QP.  Q symmetric with ~``q_upper_per_row`` random upper off-diagonals per
    row (mirrored), N(0,1), and Q_ii = sum_j |Q_ij| + U(0.1, 1) (diagonally dominant, ~10/row).
    A has column degrees from a Pareto tail (pdf exponent 2.5, minimum 4/3, mean ~4, so ~8
    nonzeros per row at m = n/2), capped at m, row positions uniform, entries N(0,1).
    Feasible as ``random_qp``; half the variables (random) boxed to [-box, box], the rest free."""
    rng = np.random.default_rng(seed)
    nu = int(round(n * q_upper_per_row))
    i = rng.integers(0, n, size=nu)
    j = rng.integers(0, n, size=nu)
    keep = i != j
    i, j = i[keep], j[keep]
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    key = np.unique(lo.astype(np.int64) * n + hi)
    lo, hi = key // n, key % n
    v = rng.standard_normal(len(key))
    U = sp.coo_matrix((v, (lo, hi)), shape=(n, n)).tocsr()
    Off = U + U.T
    diag = np.asarray(abs(Off).sum(axis=1)).ravel() + rng.uniform(0.1, 1.0, n)
    Q = _csr(Off + sp.diags(diag))
    deg = np.minimum(np.maximum(np.round(deg_min * (1.0 + rng.pareto(pareto_shape, n))), 1), m)
    deg = deg.astype(np.int64)
    cols = np.repeat(np.arange(n, dtype=np.int64), deg)
    rows = rng.integers(0, m, size=len(cols))
    key = np.unique(rows * n + cols)
    rows, cols = key // n, key % n
    A = _csr(sp.coo_matrix((rng.standard_normal(len(key)), (rows, cols)), shape=(m, n)))
    c = rng.standard_normal(n)
    x0 = rng.uniform(-5.0, 5.0, n)
    Ax0 = A @ x0
    n_eq = int(round(eq_frac * m))
    lc = np.empty(m)
    uc = np.empty(m)
    lc[:n_eq] = Ax0[:n_eq]
    uc[:n_eq] = Ax0[:n_eq]
    lc[n_eq:] = -INF
    uc[n_eq:] = Ax0[n_eq:] + rng.uniform(0.0, 1.0, m - n_eq)
    boxed = rng.random(n) < 0.5
    lv = np.where(boxed, -box, -INF)
    uv = np.where(boxed, box, INF)
    return QP(n, m, Q, A, c, lc, uc, lv, uv, name=f"large_sparse_qp_n{n}_s{seed}")


def mpc_qp(T=None, seed=0, nx=12, nu=4) -> QP:
    """Linear MPC over horizon T (T ~ U{10..50} when None).  Variables per step t:
    (u_t in R^4, x_{t+1} in R^12), so n = 16 T; rows x_{t+1} - A_d x_t - B_d u_t = 0
    (x_1 - B_d u_0 = A_d x_0 for t = 0), m = 12 T.  A_d = I + 0.1 N(0,1)/sqrt(12) scaled
    so its spectral radius is at most 1.05; B_d ~ N(0, 0.1^2); Q = blkdiag(R, Q_x) per step
    with Q_x = diag U(1,10), R = diag U(0.1,1); c = 0; |u| <= 1, x free; x_0 ~ N(0, I)."""
    rng = np.random.default_rng(seed)
    if T is None:
        T = int(rng.integers(10, 51))
    Ad = np.eye(nx) + 0.1 * rng.standard_normal((nx, nx)) / np.sqrt(nx)
    rho = np.max(np.abs(np.linalg.eigvals(Ad)))
    if rho > 1.05:
        Ad *= 1.05 / rho
    Bd = 0.1 * rng.standard_normal((nx, nu))
    qx = rng.uniform(1.0, 10.0, nx)
    ru = rng.uniform(0.1, 1.0, nu)
    x0 = rng.standard_normal(nx)
    blk = nx + nu
    n = blk * T
    m = nx * T
    rows, cols, vals = [], [], []
    rhs = np.zeros(m)
    for t in range(T):
        r0 = nx * t
        ucol = blk * t
        xcol = blk * t + nu
        for a in range(nx):
            r = r0 + a
            if t > 0:
                prev = blk * (t - 1) + nu
                for b_ in range(nx):
                    rows.append(r); cols.append(prev + b_); vals.append(-Ad[a, b_])
            for b_ in range(nu):
                rows.append(r); cols.append(ucol + b_); vals.append(-Bd[a, b_])
            rows.append(r); cols.append(xcol + a); vals.append(1.0)
        if t == 0:
            rhs[0:nx] = Ad @ x0
    A = _csr(sp.coo_matrix((vals, (rows, cols)), shape=(m, n)))
    qd = np.tile(np.concatenate([ru, qx]), T)
    Q = _csr(sp.diags(qd).tocsr())
    c = np.zeros(n)
    lv = np.tile(np.concatenate([-np.ones(nu), np.full(nx, -INF)]), T)
    uv = np.tile(np.concatenate([np.ones(nu), np.full(nx, INF)]), T)
    return QP(n, m, Q, A, c, rhs.copy(), rhs.copy(), lv, uv, name=f"mpc_T{T}_s{seed}",
              meta={"T": T})


def mpc_batch(count=4096, seed=0):
    """``count`` MPC instances with independent seeds derived from ``seed``."""
    ss = np.random.SeedSequence(seed)
    seeds = [int(s.generate_state(1)[0]) for s in ss.spawn(count)]
    return [mpc_qp(seed=s) for s in seeds]


def lasso_qp(rows=20_000, cols=2_000, density=1e-3, lam_frac=0.01, seed=0) -> QP:
    """LASSO min ||Ax - b||^2 + lam ||x||_1 as the QP of Sec. 6.3:
    min y^T y + lam 1^T t  s.t.  y = A x - b,  -t <= x <= t.
    Variables (x, t, y); b is the last column of a random sparse design matrix and
    lam = lam_frac * ||A^T b||_inf as in the paper's setup."""
    rng = np.random.default_rng(seed)
    Dm = _sprandn(rng, rows, cols + 1, density)
    A = _csr(Dm[:, :cols])
    b = np.asarray(Dm[:, cols].todense()).ravel()
    lam = lam_frac * np.max(np.abs(A.T @ b)) if np.any(b) else lam_frac
    nx, nt, ny = cols, cols, rows
    N = nx + nt + ny
    Q = _csr(sp.diags(np.concatenate([np.zeros(nx + nt), 2.0 * np.ones(ny)])).tocsr())
    c = np.concatenate([np.zeros(nx), np.full(nt, lam), np.zeros(ny)])
    I = sp.identity(cols)
    top = sp.hstack([A, sp.csr_matrix((rows, nt)), -sp.identity(rows)])   # A x - y = b
    mid1 = sp.hstack([I, -I, sp.csr_matrix((cols, ny))])                  # x - t <= 0
    mid2 = sp.hstack([I, I, sp.csr_matrix((cols, ny))])                   # x + t >= 0
    Acon = _csr(sp.vstack([top, mid1, mid2]))
    lc = np.concatenate([b, np.full(cols, -INF), np.zeros(cols)])
    uc = np.concatenate([b, np.zeros(cols), np.full(cols, INF)])
    lv = np.full(N, -INF)
    uv = np.full(N, INF)
    # drop the all-zero quadratic rows from storage
    return QP(N, rows + 2 * cols, Q, Acon, c, lc, uc, lv, uv, name=f"lasso_{rows}x{cols}_s{seed}",
              meta={"lam": lam})


def equality_qp(n=30, m=10, seed=0) -> QP:
    """Equality-constrained QP with free variables and Q positive definite."""
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    Qd = M.T @ M / n + 0.5 * np.eye(n)
    Qd[np.abs(Qd) < 0.05] = 0.0
    Qd = 0.5 * (Qd + Qd.T) + 0.5 * np.eye(n)
    A = rng.standard_normal((m, n))
    A[rng.random((m, n)) < 0.5] = 0.0
    b = A @ rng.standard_normal(n)
    c = rng.standard_normal(n)
    return QP(n, m, _csr(Qd), _csr(A), c, b.copy(), b.copy(), np.full(n, -INF), np.full(n, INF),
              name=f"equality_qp_{n}x{m}_s{seed}")


def small_box_qp(n=6, m=3, seed=0) -> QP:
    """Small QP with boxes, one equality row and inequality rows (for brute force)."""
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    Qd = M.T @ M / n + 0.2 * np.eye(n)
    A = rng.standard_normal((m, n))
    x0 = rng.uniform(-0.5, 0.5, n)
    Ax0 = A @ x0
    lc = np.empty(m)
    uc = np.empty(m)
    lc[0] = uc[0] = Ax0[0]
    for i in range(1, m):
        if i % 2:
            lc[i], uc[i] = -INF, Ax0[i] + 0.1
        else:
            lc[i], uc[i] = Ax0[i] - 0.1, INF
    c = 3.0 * rng.standard_normal(n)
    lv = np.full(n, -1.0)
    uv = np.full(n, 1.0)
    lv[0] = -INF          # one half-bounded variable
    uv[1] = INF
    return QP(n, m, _csr(Qd), _csr(A), c, lc, uc, lv, uv, name=f"small_box_qp_{n}_s{seed}")


def infeasible_qp(n=8, m=4, seed=0) -> QP:
    """Two contradictory equality rows a^T x = b and a^T x = b + 1 (Sec. 5.1 certificate
    y = t (e_i - e_j) has A^T y = 0 and p(y) = -t < 0)."""
    qp = small_box_qp(n=n, m=m, seed=seed)
    A = qp.A.toarray()
    A = np.vstack([A, A[0:1]])
    lc = np.append(qp.lc, qp.lc[0] + 1.0)
    uc = np.append(qp.uc, qp.uc[0] + 1.0)
    return QP(n, m + 1, qp.Q, _csr(A), qp.c, lc, uc, qp.lv, qp.uv, name=f"infeasible_qp_{n}_s{seed}")


def unbounded_qp(n=6, seed=0) -> QP:
    """Q singular with Q d = 0, c^T d < 0, A d = 0, d free (Sec. 5.2 theorem)."""
    rng = np.random.default_rng(seed)
    d = np.zeros(n)
    d[0] = 1.0
    d[1] = 1.0
    B = rng.standard_normal((n, n))
    P = np.eye(n) - np.outer(d, d) / (d @ d)
    Qd = P @ (B.T @ B / n + np.eye(n)) @ P
    Qd = 0.5 * (Qd + Qd.T)
    # Q d = 0 bit for bit (column 1 = -column 0), so that it also holds after any
    # scaling that treats the two mirrored columns alike, and in FP32 storage
    Qd[:, 1] = -Qd[:, 0]
    Qd[1, :] = -Qd[0, :]
    Qd[1, 1] = Qd[0, 0]
    Qd[np.abs(Qd) < 1e-14] = 0.0
    A = rng.standard_normal((2, n))
    A[:, 1] = -A[:, 0]                      # A d = 0
    c = rng.standard_normal(n)
    c -= (c @ d) / (d @ d) * d
    c -= 1.0 * d                             # c^T d = -2
    lv = np.full(n, -INF)
    uv = np.full(n, INF)
    lv[2:] = -5.0
    uv[2:] = 5.0
    b = A @ rng.uniform(-1, 1, n)
    lc = np.array([b[0], -INF])
    uc = np.array([b[0], b[1] + 1.0])
    return QP(n, 2, _csr(Qd), _csr(A), c, lc, uc, lv, uv, name=f"unbounded_qp_{n}_s{seed}",
              meta={"d": d})


def serving_trace(rate_per_s=200.0, duration_s=2.0, seed=0, n_range=(1_000, 100_000),
                  factor_n=100_000, max_requests=None, mix=(0.70, 0.25, 0.05)):
    """Poisson arrival trace of a request mix: 70 % MPC (as ``mpc_qp``), 25 % random QPs as
    ``random_qp`` with n ~ U{1e3..1e5}, m = n/2, ~10 nonzeros per row (2 % of them made
    infeasible by a contradictory equality row), 5 % factor-model QPs with n = 1e5.
    Returns a list of (arrival_time_s, kind, seed, size) tuples; the QP is built on demand
    with ``build_request``."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t > duration_s:
            break
        u = rng.random()
        s = int(rng.integers(0, 2**31 - 1))
        if u < mix[0]:
            out.append((t, "mpc", s, 0))
        elif u < mix[0] + mix[1]:
            nsz = int(rng.integers(n_range[0], n_range[1] + 1))
            kind = "random_infeasible" if rng.random() < 0.02 else "random"
            out.append((t, kind, s, nsz))
        else:
            out.append((t, "factor", s, factor_n))
        if max_requests is not None and len(out) >= max_requests:
            break
    return out


def build_request(kind, seed, size):
    if kind == "mpc":
        return mpc_qp(seed=seed)
    if kind in ("random", "random_infeasible"):
        return random_qp(n=size, m=size // 2, n_eq=size // 4, m_rows=max(size // 4, 1), seed=seed,
                         per_row=10, infeasible=(kind == "random_infeasible"))
    if kind == "factor":
        return factor_portfolio(n=size, k=max(size // 100, 1), seed=seed)
    raise ValueError(kind)

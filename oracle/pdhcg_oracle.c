/*
 * pdhcg_oracle.c — plain FP64 CPU oracle of the PDHCG-II iteration.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code, header or constant table with the CUDA library.
 *
 * It follows the paper step by step, in the paper's order, with no blocking,
 * fusion or reordering:
 *   problem (QP) and its restricted Wolfe dual ........ Sec. 2, Eq. (QP), Eq. (dualQP)
 *   support function p(z; l, u), sign cones Y and R .... Sec. 2 (definitions after Eq. dualQP)
 *   PDHG step (primal prox solve, extrapolation, dual) .. Sec. 2.1, Eq. (pdhcg_update)
 *   primal subproblem: diagonal closed form, CG, BB-PG . Sec. 2.2 and Sec. 3.3
 *   structured Q = P + R^T R, applied matrix-free ...... Sec. 2.2 (oracle_solve_qr)
 *   reflected Halpern scheme ............................ Sec. 3.1
 *   tau = eta/omega, sigma = eta*omega, eta = 0.998/||A|| Sec. 3.2 (||A|| by Lanczos: reading)
 *   PID primal-weight update ............................ Sec. 3.2, Eq. (pid)
 *   adaptive inner tolerance ............................ Sec. 3.3
 *   KKT residuals r_primal, r_dual, r_gap ............... Sec. 4.2
 *   primal / dual infeasibility tests ................... Sec. 5.1, Sec. 5.2
 *
 * Where the paper is silent the oracle takes the readings listed in the
 * design notes (restart rule, Halpern index, PID gains, first inner tolerance,
 * norm estimate, initial point, Ruiz scaling, infeasibility tolerance).  Each
 * such place is marked "reading:" below.
 *
 * Parity pins: see tests/test_oracle_pins.py (dense KKT LU, active-set brute
 * force, constructed infeasible and unbounded instances, SVD norm, subproblem
 * optimality, LASSO against coordinate descent, the factored objective against
 * the explicitly formed one, factored scaling against scaling of a diagonal
 * R^T R, hand-derived closed forms in tests/golden, and a hand-derived trace of
 * the first four steps on a one-variable QP that fixes the adaptive inner
 * tolerance, the reflected Halpern weights and the step sizes, plus a point
 * where only the gap term of Sec. 4.2 is nonzero).  Parity unpinned:
 * iteration counts relative to the paper's own release (no instance or trace
 * is published).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include "pdhcg_oracle.h"

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

static double now_seconds(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

static double dot(const double* a, const double* b, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double norm2(const double* a, int64_t n) { return sqrt(dot(a, a, n)); }

static double norminf(const double* a, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s = fmax(s, fabs(a[i]));
  return s;
}

static double clampd(double v, double l, double u) {
  if (v < l) return l;
  if (v > u) return u;
  return v;
}

/* y = M x for a CSR matrix with values val (may differ from M->val). */
static void spmv(const oracle_csr* M, const double* val, const double* x, double* y) {
  for (int32_t i = 0; i < M->nrows; ++i) {
    double s = 0.0;
    for (int64_t k = M->rowptr[i]; k < M->rowptr[i + 1]; ++k) s += val[k] * x[M->col[k]];
    y[i] = s;
  }
}

/* y = M^T x, straight from the definition (column sums of M scaled by x). */
static void spmv_t(const oracle_csr* M, const double* val, const double* x, double* y) {
  for (int32_t j = 0; j < M->ncols; ++j) y[j] = 0.0;
  for (int32_t i = 0; i < M->nrows; ++i)
    for (int64_t k = M->rowptr[i]; k < M->rowptr[i + 1]; ++k) y[M->col[k]] += val[k] * x[i];
}

/* Sign cone Y_i of the dual variable (Sec. 2, cases by finiteness of l_c, u_c). */
static double proj_Y(double v, double lo, double hi) {
  int lf = isfinite(lo), uf = isfinite(hi);
  if (!lf && !uf) return 0.0;        /* {0}  */
  if (!lf && uf) return fmax(v, 0.0); /* R+   */
  if (lf && !uf) return fmin(v, 0.0); /* R-   */
  return v;                           /* R    */
}

/* Sign cone R_i of the reduced cost (Sec. 2, cases by finiteness of l_v, u_v). */
static double proj_R(double v, double lo, double hi) {
  int lf = isfinite(lo), uf = isfinite(hi);
  if (!lf && !uf) return 0.0;        /* {0}  */
  if (!lf && uf) return fmin(v, 0.0); /* R-   */
  if (lf && !uf) return fmax(v, 0.0); /* R+   */
  return v;                           /* R    */
}

/* Recession cone of the box [lo, hi], componentwise (Sec. 5.2; reading of the
 * garbled definition: {0} if both bounds are finite, R+ if only lo is, R- if
 * only hi is, R if neither is). */
static double proj_recc(double d, double lo, double hi) {
  int lf = isfinite(lo), uf = isfinite(hi);
  if (lf && uf) return 0.0;
  if (lf) return fmax(d, 0.0);
  if (uf) return fmin(d, 0.0);
  return d;
}

/* p(z; l, u) = u^T z^+ - l^T z^- (Sec. 2); a zero component contributes 0 even
 * when its bound is infinite. */
static double support_p(const double* z, const double* lo, const double* hi, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (z[i] > 0.0) s += hi[i] * z[i];
    else if (z[i] < 0.0) s -= lo[i] * (-z[i]);
  }
  return s;
}

void oracle_default_params(oracle_params* p) {
  memset(p, 0, sizeof(*p));
  p->eps_tol = 1e-6;
  p->eps_inf = 1e-8;
  p->time_limit_s = 3600.0;
  p->max_iter = 1000000;
  p->theta = 1.0;
  p->kp = 0.99;
  p->ki = 0.01;
  p->kd = 0.0;
  p->gamma_inner = 5e-4;
  p->eps_inner_min = 1e-9;
  p->eps_inner_first = 1e-2;
  p->k_eval = 64;
  p->inner = ORACLE_INNER_AUTO;
  p->max_inner_iter = 1000;
  p->ruiz_iters = 10;
  p->restart_sufficient = 0.2;
  p->restart_necessary = 0.8;
  p->restart_artificial = 0.36;
  p->power_max_iter = 1000;
  p->power_tol = 1e-8;
  p->eta_override = 0.0;
  p->omega0_override = 0.0;
  p->omega_clamp = 1e5;
}

/* ------------------------------------------------------------------ */
/* Setup: Ruiz equilibration (reading) and the norm estimate          */
/* ------------------------------------------------------------------ */

/* Ruiz equilibration of K = [Q A^T; A 0] in the infinity norm.  Each pass
 * divides every column j of K by sqrt(max_i |K_ij|) of the currently scaled
 * matrix.  The scaled entries are (Q_ij*D_i)*D_j and (A_ij*E_i)*D_j.
 * Reading: the paper names a "system scaling factor" but no scaling method. */
static void ruiz_impl(int32_t n, int32_t m, const oracle_csr* Q, const oracle_csr* R, const oracle_csr* A,
                      int32_t passes, double* D, double* E);

void oracle_ruiz(int32_t n, int32_t m, const oracle_csr* Q, const oracle_csr* A, int32_t passes,
                 double* D, double* E) {
  ruiz_impl(n, m, Q, NULL, A, passes, D, E);
}

void oracle_ruiz_qr(int32_t n, int32_t m, const oracle_csr* P, const oracle_csr* R, const oracle_csr* A,
                    int32_t passes, double* D, double* E) {
  ruiz_impl(n, m, P, R, A, passes, D, E);
}

/* With a structured Q = P + R^T R (reading): the column maximum of Q is taken
 * over the entries of P and the diagonal of R^T R (squared column norms of R).
 * By Cauchy-Schwarz each entry of R^T R is at most the geometric mean of the
 * two diagonal entries in its row and column, so the diagonal carries the size
 * of R^T R without forming it. */
static void ruiz_impl(int32_t n, int32_t m, const oracle_csr* Q, const oracle_csr* R, const oracle_csr* A,
                      int32_t passes, double* D, double* E) {
  double* rd = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  for (int32_t l = 0; R && l < R->nrows; ++l)
    for (int64_t k = R->rowptr[l]; k < R->rowptr[l + 1]; ++k) rd[R->col[k]] += R->val[k] * R->val[k];
  for (int32_t j = 0; j < n; ++j) D[j] = 1.0;
  for (int32_t i = 0; i < m; ++i) E[i] = 1.0;
  double* cn = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* rn = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  for (int32_t pass = 0; pass < passes; ++pass) {
    for (int32_t j = 0; j < n; ++j) cn[j] = 0.0;
    for (int32_t i = 0; i < m; ++i) rn[i] = 0.0;
    if (Q) {
      for (int32_t i = 0; i < n; ++i)
        for (int64_t k = Q->rowptr[i]; k < Q->rowptr[i + 1]; ++k) {
          int32_t j = Q->col[k];
          double v = fabs((Q->val[k] * D[i]) * D[j]);
          cn[j] = fmax(cn[j], v);
        }
    }
    for (int32_t j = 0; R && j < n; ++j) cn[j] = fmax(cn[j], (rd[j] * D[j]) * D[j]);
    for (int32_t i = 0; i < m; ++i)
      for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) {
        int32_t j = A->col[k];
        double v = fabs((A->val[k] * E[i]) * D[j]);
        cn[j] = fmax(cn[j], v);
        rn[i] = fmax(rn[i], v);
      }
    for (int32_t j = 0; j < n; ++j) D[j] = D[j] * (cn[j] > 0.0 ? 1.0 / sqrt(cn[j]) : 1.0);
    for (int32_t i = 0; i < m; ++i) E[i] = E[i] * (rn[i] > 0.0 ? 1.0 / sqrt(rn[i]) : 1.0);
  }
  free(cn);
  free(rn);
  free(rd);
}

/* Number of eigenvalues below x of the symmetric tridiagonal matrix with
 * diagonal a[0..k) and off-diagonal b[0..k-1): the number of negative pivots
 * of the LDL^T factorisation of T - x I (Sturm count). */
static int32_t sturm_below(const double* a, const double* b, int32_t k, double x) {
  int32_t c = 0;
  double d = 1.0;
  for (int32_t i = 0; i < k; ++i) {
    d = (a[i] - x) - (i > 0 ? (b[i - 1] * b[i - 1]) / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++c;
  }
  return c;
}

/* Largest eigenvalue of that tridiagonal matrix by bisection on the Sturm
 * count, from [max diagonal, Gershgorin bound] down to adjacent doubles.
 * Returns the upper end of the final interval. */
static double tridiag_max_eig(const double* a, const double* b, int32_t k) {
  double lo = a[0], hi = a[0];
  for (int32_t i = 0; i < k; ++i) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
    lo = fmax(lo, a[i]);
    hi = fmax(hi, a[i] + r);
  }
  hi = hi + 1e-12 * (fabs(hi) + 1e-300);
  for (int32_t it = 0; it < 2000; ++it) {
    const double x = 0.5 * (lo + hi);
    if (!(x > lo && x < hi)) break;
    if (sturm_below(a, b, k, x) == k) hi = x;
    else lo = x;
  }
  return hi;
}

/* ||A||_2 (reading: the paper fixes eta = 0.998/||A|| but not how ||A|| is
 * computed).  Lanczos on A^T A from v_1 = ones/sqrt(n), without
 * reorthogonalisation (its largest Ritz value still converges from below):
 *   t = A v_k, w = A^T t, alpha_k = ||t||^2, w -= alpha_k v_k + beta_{k-1} v_{k-1},
 *   beta_k = ||w||, v_{k+1} = w / beta_k.
 * The largest eigenvalue of the tridiagonal T_k (alpha, beta) is taken at
 * k = 8, 16, 24, 36, 54, ... (each check k + max(8, k/2) after the last) and at
 * max_iter; stop when two such values agree to tol relative, or when beta_k
 * vanishes (the Krylov space is invariant and T_k is exact).  *iters_out:
 * Lanczos steps taken. */
double oracle_norm_estimate(const oracle_csr* A, const double* val, int32_t max_iter, double tol,
                            int32_t* iters_out) {
  int32_t n = A->ncols, m = A->nrows;
  size_t nn = (size_t)(n > 0 ? n : 1);
  double* v = (double*)malloc(sizeof(double) * nn);
  double* vp = (double*)calloc(nn, sizeof(double));
  double* w = (double*)malloc(sizeof(double) * nn);
  double* t = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  double* al = (double*)malloc(sizeof(double) * (size_t)(max_iter > 0 ? max_iter : 1));
  double* be = (double*)malloc(sizeof(double) * (size_t)(max_iter > 0 ? max_iter : 1));
  for (int32_t j = 0; j < n; ++j) v[j] = 1.0 / sqrt((double)n);
  double lam = 0.0, lam_prev = -1.0, bprev = 0.0;
  int32_t next_check = 8, k = 0;
  for (k = 1; k <= max_iter; ++k) {
    spmv(A, val, v, t);
    spmv_t(A, val, t, w);
    const double alpha = dot(t, t, m);
    for (int32_t j = 0; j < n; ++j) w[j] = w[j] - alpha * v[j] - bprev * vp[j];
    const double beta = norm2(w, n);
    al[k - 1] = alpha;
    be[k - 1] = beta;
    const int invariant = !(beta > 1e-13 * sqrt(alpha * alpha + bprev * bprev));
    if (k == next_check || invariant || k == max_iter) {
      lam = tridiag_max_eig(al, be, k);
      if (invariant || (lam_prev >= 0.0 && fabs(lam - lam_prev) <= tol * lam)) break;
      lam_prev = lam;
      next_check += next_check / 2 > 8 ? next_check / 2 : 8;
    }
    for (int32_t j = 0; j < n; ++j) {
      vp[j] = v[j];
      v[j] = w[j] / beta;
    }
    bprev = beta;
  }
  if (iters_out) *iters_out = k > max_iter ? max_iter : k;
  free(v);
  free(vp);
  free(w);
  free(t);
  free(al);
  free(be);
  return sqrt(lam);
}

/* ------------------------------------------------------------------ */
/* Primal subproblem solvers (Sec. 2.2, Sec. 3.3)                      */
/*   min_{x in [lv,uv]} 1/2 x^T H x - b^T x,   H = Q + I/tau           */
/* ------------------------------------------------------------------ */

typedef struct {
  const oracle_csr* Q;   /* may be NULL (Q = 0) */
  const double* qval;    /* scaled values of Q  */
  const oracle_csr* R;   /* structured part Q = P + R^T R (Sec. 2.2): may be NULL */
  const double* rval;    /* scaled values of R  */
  double inv_tau;
  int32_t n;
  double* tmp;           /* length n (with R) */
  double* tk;            /* length k (with R) */
} hop_t;

/* out = Q v with Q = P + R^T R applied as P v + R^T (R v), never forming R^T R
 * (Sec. 2.2, structured quadratic objective). */
static void apply_Q(const oracle_csr* P, const double* pval, const oracle_csr* R, const double* rval,
                    int32_t n, const double* v, double* out, double* tmp, double* tk) {
  if (P) spmv(P, pval, v, out);
  else for (int32_t i = 0; i < n; ++i) out[i] = 0.0;
  if (R) {
    spmv(R, rval, v, tk);
    spmv_t(R, rval, tk, tmp);
    for (int32_t i = 0; i < n; ++i) out[i] += tmp[i];
  }
}

/* out = H v = Q v + v / tau */
static void apply_H(const hop_t* h, const double* v, double* out) {
  apply_Q(h->Q, h->qval, h->R, h->rval, h->n, v, out, h->tmp, h->tk);
  for (int32_t i = 0; i < h->n; ++i) out[i] += v[i] * h->inv_tau;
}

/* Conjugate gradient (Hestenes-Stiefel) on H x = b, warm-started at x, stopped
 * when ||b - H x||_2 <= eps or after max_it steps.  Returns the step count. */
static int32_t inner_cg(const hop_t* h, const double* b, double* x, double eps, int32_t max_it) {
  int32_t n = h->n;
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* p = (double*)malloc(sizeof(double) * (size_t)n);
  double* q = (double*)malloc(sizeof(double) * (size_t)n);
  apply_H(h, x, q);
  for (int32_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
  double rr = dot(r, r, n);
  int32_t j = 0;
  for (j = 0; j < max_it; ++j) {
    if (sqrt(rr) <= eps) break;
    if (j == 0) {
      for (int32_t i = 0; i < n; ++i) p[i] = r[i];
    }
    apply_H(h, p, q);
    double pq = dot(p, q, n);
    if (!(pq > 0.0)) break;
    double alpha = rr / pq;
    for (int32_t i = 0; i < n; ++i) x[i] += alpha * p[i];
    for (int32_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
    double rr_new = dot(r, r, n);
    double beta = rr_new / rr;
    for (int32_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    rr = rr_new;
  }
  free(r);
  free(p);
  free(q);
  return j;
}

/* Projected gradient with Barzilai-Borwein (BB1) steps over the box, warm
 * started at x (already in the box).  The step is s^T s / s^T (grad - grad_prev)
 * clamped to [alpha_min, tau] with alpha_min = 1 / (G + 1/tau), G a Gershgorin
 * bound on ||Q||; the first step is alpha_min.  Stops when the natural residual
 * ||x - proj(x - grad)||_2 <= eps or after max_it steps.  Returns the step count. */
static int32_t inner_bb(const hop_t* h, const double* b, const double* lv, const double* uv,
                        double gersh, double* x, double eps, int32_t max_it) {
  int32_t n = h->n;
  double tau = 1.0 / h->inv_tau;
  double alpha_min = 1.0 / (gersh + h->inv_tau);
  double alpha_max = tau;
  double* g = (double*)malloc(sizeof(double) * (size_t)n);
  double* xp = (double*)malloc(sizeof(double) * (size_t)n);
  double* gp = (double*)malloc(sizeof(double) * (size_t)n);
  apply_H(h, x, g);
  for (int32_t i = 0; i < n; ++i) g[i] = g[i] - b[i];
  int32_t j = 0;
  for (j = 0; j < max_it; ++j) {
    double nr = 0.0, ss = 0.0, sy = 0.0;
    for (int32_t i = 0; i < n; ++i) {
      double d = x[i] - clampd(x[i] - g[i], lv[i], uv[i]);
      nr += d * d;
    }
    if (sqrt(nr) <= eps) break;
    double alpha = alpha_min;
    if (j > 0) {
      for (int32_t i = 0; i < n; ++i) {
        double s = x[i] - xp[i];
        double yv = g[i] - gp[i];
        ss += s * s;
        sy += s * yv;
      }
      alpha = sy > 0.0 ? ss / sy : alpha_max;
      alpha = clampd(alpha, alpha_min, alpha_max);
    }
    for (int32_t i = 0; i < n; ++i) {
      xp[i] = x[i];
      gp[i] = g[i];
      x[i] = clampd(x[i] - alpha * g[i], lv[i], uv[i]);
    }
    apply_H(h, x, g);
    for (int32_t i = 0; i < n; ++i) g[i] = g[i] - b[i];
  }
  free(g);
  free(xp);
  free(gp);
  return j;
}

/* Exposed for unit pins: one inner solve on unscaled data. */
int32_t oracle_inner_solve(int32_t n, const oracle_csr* Q, const double* lv, const double* uv,
                           double tau, const double* b, double eps, int32_t max_it, int32_t method,
                           double* x) {
  hop_t h;
  h.R = NULL;
  h.rval = NULL;
  h.tk = NULL;
  h.Q = Q;
  h.qval = Q ? Q->val : NULL;
  h.inv_tau = 1.0 / tau;
  h.n = n;
  h.tmp = NULL;
  if (method == ORACLE_INNER_CG) return inner_cg(&h, b, x, eps, max_it);
  double gersh = 0.0;
  if (Q)
    for (int32_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t k = Q->rowptr[i]; k < Q->rowptr[i + 1]; ++k) s += fabs(Q->val[k]);
      gersh = fmax(gersh, s);
    }
  return inner_bb(&h, b, lv, uv, gersh, x, eps, max_it);
}

/* ------------------------------------------------------------------ */
/* KKT residuals (Sec. 4.2) on unscaled quantities                     */
/* ------------------------------------------------------------------ */

void oracle_kkt(int32_t n, int32_t m, const double* x, const double* y, const double* Ax,
                const double* ATy, const double* Qx, const double* c, const double* lc,
                const double* uc, const double* lv, const double* uv, double* out6) {
  /* primal residual */
  double viol = 0.0, bscale = 0.0;
  for (int32_t i = 0; i < m; ++i) {
    viol = fmax(viol, fabs(Ax[i] - clampd(Ax[i], lc[i], uc[i])));
    if (isfinite(lc[i])) bscale = fmax(bscale, fabs(lc[i]));
    if (isfinite(uc[i])) bscale = fmax(bscale, fabs(uc[i]));
  }
  double r_primal = viol / (1.0 + bscale);
  /* dual residual: r = Qx + c + A^T y must lie in R; rhat = proj_R(r) */
  double* rhat = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* mr = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double dviol = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    double r = Qx[j] + c[j] + ATy[j];
    rhat[j] = proj_R(r, lv[j], uv[j]);
    dviol = fmax(dviol, fabs(r - rhat[j]));
    mr[j] = -rhat[j];
  }
  double dscale = fmax(fmax(norminf(Qx, n), norminf(ATy, n)), norminf(c, n));
  double r_dual = dviol / (1.0 + dscale);
  /* duality gap */
  double xQx = dot(x, Qx, n);
  double cx = dot(c, x, n);
  double pr = support_p(mr, lv, uv, n);
  double py = support_p(y, lc, uc, m);
  double pobj = 0.5 * xQx + cx;
  double dobj = -pr - 0.5 * xQx - py;
  double gap = fabs(xQx + cx + pr + py);
  double r_gap = gap / (1.0 + fmax(fabs(pobj), fabs(0.5 * xQx + pr + py)));
  out6[0] = r_primal;
  out6[1] = r_dual;
  out6[2] = r_gap;
  out6[3] = pobj;
  out6[4] = dobj;
  out6[5] = 0.0;
  free(rhat);
  free(mr);
}

/* ------------------------------------------------------------------ */
/* PID primal-weight update (Sec. 3.2, Eq. pid)                        */
/* ------------------------------------------------------------------ */

/* One update at the end of a restarted round.  dx, dy are the norms of the
 * primal and dual movement over the round.  Reading: skip when either norm is
 * below 1e-10; clamp omega to [omega0/clamp, omega0*clamp]. */
void oracle_pid_update(double* log_omega, double* e_sum, double* e_prev, double dx, double dy,
                       double kp, double ki, double kd, double log_omega0, double clamp) {
  if (!(dx > 1e-10) || !(dy > 1e-10)) return;
  double omega = exp(*log_omega);
  double e = log(omega * dx / dy);
  *e_sum += e;
  double lw = *log_omega - (kp * e + ki * (*e_sum) + kd * (e - *e_prev));
  *e_prev = e;
  double lim = log(clamp);
  lw = clampd(lw, log_omega0 - lim, log_omega0 + lim);
  *log_omega = lw;
}

/* ------------------------------------------------------------------ */
/* The solver                                                          */
/* ------------------------------------------------------------------ */

static int csr_is_diagonal(const oracle_csr* Q) {
  if (!Q) return 1;
  for (int32_t i = 0; i < Q->nrows; ++i)
    for (int64_t k = Q->rowptr[i]; k < Q->rowptr[i + 1]; ++k)
      if (Q->col[k] != i && Q->val[k] != 0.0) return 0;
  return 1;
}

static int solve_impl(int32_t n, int32_t m, const oracle_csr* Q, const oracle_csr* R, const oracle_csr* A,
                      const double* c, const double* lc, const double* uc, const double* lv,
                      const double* uv, const oracle_params* prm, const double* x_init,
                      const double* y_init, double* x_out, double* y_out, oracle_result* res,
                      double* eps_trace, int32_t eps_trace_len);

int oracle_solve(int32_t n, int32_t m, const oracle_csr* Q, const oracle_csr* A, const double* c,
                 const double* lc, const double* uc, const double* lv, const double* uv,
                 const oracle_params* prm, const double* x_init, const double* y_init,
                 double* x_out, double* y_out, oracle_result* res, double* eps_trace,
                 int32_t eps_trace_len) {
  return solve_impl(n, m, Q, NULL, A, c, lc, uc, lv, uv, prm, x_init, y_init, x_out, y_out, res, eps_trace,
                    eps_trace_len);
}

/* Q = P + R^T R with R k x n, applied matrix-free (Sec. 2.2).  Readings: the
 * Ruiz factors come from P, A and the diagonal of R^T R (R^T R is never
 * formed); the scaled factor is R D; the bound on ||Q|| used by the BB step
 * range is the Gershgorin bound of the scaled P plus ||R D||_1 ||R D||_inf
 * (>= ||R D||_2^2). */
int oracle_solve_qr(int32_t n, int32_t m, const oracle_csr* P, const oracle_csr* R, const oracle_csr* A,
                    const double* c, const double* lc, const double* uc, const double* lv,
                    const double* uv, const oracle_params* prm, const double* x_init,
                    const double* y_init, double* x_out, double* y_out, oracle_result* res) {
  return solve_impl(n, m, P, R, A, c, lc, uc, lv, uv, prm, x_init, y_init, x_out, y_out, res, NULL, 0);
}

static int solve_impl(int32_t n, int32_t m, const oracle_csr* Q, const oracle_csr* R, const oracle_csr* A,
                      const double* c, const double* lc, const double* uc, const double* lv,
                      const double* uv, const oracle_params* prm, const double* x_init,
                      const double* y_init, double* x_out, double* y_out, oracle_result* res,
                      double* eps_trace, int32_t eps_trace_len) {
  double t_start = now_seconds();
  memset(res, 0, sizeof(*res));
  const int64_t nz_q = Q ? Q->rowptr[n] : 0;
  const int64_t nz_a = A->rowptr[m];
  size_t nn = (size_t)(n > 0 ? n : 1), mm = (size_t)(m > 0 ? m : 1);

  /* --- setup: scaling, scaled data (reading: Ruiz) --- */
  double* D = (double*)malloc(sizeof(double) * nn);
  double* E = (double*)malloc(sizeof(double) * mm);
  ruiz_impl(n, m, Q, R, A, prm->ruiz_iters, D, E);
  double* qv = (double*)malloc(sizeof(double) * (size_t)(nz_q > 0 ? nz_q : 1));
  double* av = (double*)malloc(sizeof(double) * (size_t)(nz_a > 0 ? nz_a : 1));
  for (int32_t i = 0; Q && i < n; ++i)
    for (int64_t k = Q->rowptr[i]; k < Q->rowptr[i + 1]; ++k) qv[k] = (Q->val[k] * D[i]) * D[Q->col[k]];
  for (int32_t i = 0; i < m; ++i)
    for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) av[k] = (A->val[k] * E[i]) * D[A->col[k]];
  double *cs = (double*)malloc(sizeof(double) * nn), *lvs = (double*)malloc(sizeof(double) * nn),
         *uvs = (double*)malloc(sizeof(double) * nn);
  double *lcs = (double*)malloc(sizeof(double) * mm), *ucs = (double*)malloc(sizeof(double) * mm);
  for (int32_t j = 0; j < n; ++j) {
    cs[j] = c[j] * D[j];
    lvs[j] = lv[j] / D[j];
    uvs[j] = uv[j] / D[j];
  }
  for (int32_t i = 0; i < m; ++i) {
    lcs[i] = lc[i] * E[i];
    ucs[i] = uc[i] * E[i];
  }
  double* qdiag = (double*)calloc(nn, sizeof(double));
  for (int32_t i = 0; Q && i < n; ++i)
    for (int64_t k = Q->rowptr[i]; k < Q->rowptr[i + 1]; ++k)
      if (Q->col[k] == i) qdiag[i] += qv[k];
  double gersh = 0.0;
  for (int32_t i = 0; Q && i < n; ++i) {
    double s = 0.0;
    for (int64_t k = Q->rowptr[i]; k < Q->rowptr[i + 1]; ++k) s += fabs(qv[k]);
    gersh = fmax(gersh, s);
  }
  /* structured part: scaled R D, and its contribution to the bound on ||Q|| */
  const int32_t kr = R ? R->nrows : 0;
  const int64_t nz_r = R ? R->rowptr[kr] : 0;
  double* rv = (double*)malloc(sizeof(double) * (size_t)(nz_r > 0 ? nz_r : 1));
  double* rtmp = (double*)malloc(sizeof(double) * nn);
  double* rtk = (double*)malloc(sizeof(double) * (size_t)(kr > 0 ? kr : 1));
  if (R) {
    double* colsum = (double*)calloc(nn, sizeof(double));
    double rowmax = 0.0;
    for (int32_t i = 0; i < kr; ++i) {
      double s = 0.0;
      for (int64_t k = R->rowptr[i]; k < R->rowptr[i + 1]; ++k) {
        rv[k] = R->val[k] * D[R->col[k]];
        s += fabs(rv[k]);
        colsum[R->col[k]] += fabs(rv[k]);
      }
      rowmax = fmax(rowmax, s);
    }
    gersh += rowmax * norminf(colsum, n);
    free(colsum);
  }

  /* --- step size eta = 0.998 / ||A|| (Sec. 3.2); norm by Lanczos (reading) --- */
  int32_t piters = 0;
  double normA = m > 0 ? oracle_norm_estimate(A, av, prm->power_max_iter, prm->power_tol, &piters) : 0.0;
  double eta = normA > 0.0 ? 0.998 / normA : 1.0;
  if (prm->eta_override > 0.0) eta = prm->eta_override;

  /* --- inner solver dispatch (Sec. 2.2; reading: AUTO = closed form for
   *     diagonal Q, BB-PG when any variable bound is finite, else CG) --- */
  int diagQ = csr_is_diagonal(Q) && !R;
  int any_box = 0;
  for (int32_t j = 0; j < n; ++j)
    if (isfinite(lv[j]) || isfinite(uv[j])) any_box = 1;
  int32_t method = prm->inner;
  if (method == ORACLE_INNER_AUTO) method = diagQ ? ORACLE_INNER_DIAG : (any_box ? ORACLE_INNER_BB : ORACLE_INNER_CG);
  if (method == ORACLE_INNER_DIAG && !diagQ) method = ORACLE_INNER_CG;
  res->inner_method = method;

  /* --- initial point (reading): x0 = proj_X(0) or the warm start, y0 = 0 or warm start --- */
  double *x = (double*)malloc(sizeof(double) * nn), *y = (double*)malloc(sizeof(double) * mm);
  double *xa = (double*)malloc(sizeof(double) * nn), *ya = (double*)malloc(sizeof(double) * mm);
  double *xp = (double*)malloc(sizeof(double) * nn), *yp = (double*)malloc(sizeof(double) * mm);
  double *xn = (double*)malloc(sizeof(double) * nn), *yn = (double*)malloc(sizeof(double) * mm);
  double *g = (double*)malloc(sizeof(double) * nn), *b = (double*)malloc(sizeof(double) * nn);
  double *xbar = (double*)malloc(sizeof(double) * nn), *axb = (double*)malloc(sizeof(double) * mm);
  for (int32_t j = 0; j < n; ++j) x[j] = clampd(x_init ? x_init[j] / D[j] : 0.0, lvs[j], uvs[j]);
  for (int32_t i = 0; i < m; ++i) y[i] = y_init ? proj_Y(y_init[i] / E[i], lcs[i], ucs[i]) : 0.0;
  memcpy(xa, x, sizeof(double) * nn);
  memcpy(ya, y, sizeof(double) * mm);

  /* initial primal weight (reading): ||c|| / ||finite bounds of S|| on scaled data */
  double cn = norm2(cs, n), bn2 = 0.0;
  for (int32_t i = 0; i < m; ++i) {
    if (isfinite(lcs[i])) bn2 += lcs[i] * lcs[i];
    if (isfinite(ucs[i])) bn2 += ucs[i] * ucs[i];
  }
  double bn = sqrt(bn2);
  double omega = (cn > 1e-10 && bn > 1e-10) ? cn / bn : 1.0;
  if (prm->omega0_override > 0.0) omega = prm->omega0_override;
  double log_omega = log(omega), log_omega0 = log(omega);
  double e_sum = 0.0, e_prev = 0.0;
  double tau = eta / omega, sigma = eta * omega;

  hop_t h;
  h.R = R;
  h.rval = rv;
  h.tk = rtk;
  h.Q = Q;
  h.qval = qv;
  h.n = n;
  h.tmp = rtmp;

  double eps_in = INFINITY, mv = 0.0;
  double fpr_anchor = 0.0, fpr_last = 0.0;
  int64_t k = 0;   /* Halpern index since the last restart */
  int64_t K = 0;   /* total PDHG steps */
  int status = 0;
  int64_t inner_total = 0, restarts = 0;
  double kkt[6] = {0, 0, 0, 0, 0, 0};

  double *ux = (double*)malloc(sizeof(double) * nn), *uy = (double*)malloc(sizeof(double) * mm);
  double *uAx = (double*)malloc(sizeof(double) * mm), *uATy = (double*)malloc(sizeof(double) * nn);
  double *uQx = (double*)malloc(sizeof(double) * nn);
  double *dd = (double*)malloc(sizeof(double) * nn), *ytil = (double*)malloc(sizeof(double) * mm);
  double *t_n = (double*)malloc(sizeof(double) * nn), *t_m = (double*)malloc(sizeof(double) * mm);

  for (;;) {
    double inv_tau = 1.0 / tau, inv_sigma = 1.0 / sigma;
    h.inv_tau = inv_tau;

    /* primal subproblem data: b = x/tau - c - A^T y (Sec. 2.1, Eq. primal_update) */
    spmv_t(A, av, y, g);
    for (int32_t j = 0; j < n; ++j) b[j] = x[j] * inv_tau - cs[j] - g[j];

    /* adaptive inner tolerance (Sec. 3.3).  reading: the first tolerance is
     * eps_inner_first * max(1, ||b||); afterwards the paper's rule with the
     * movement of the previous step. */
    if (K == 0) eps_in = prm->eps_inner_first * fmax(1.0, norm2(b, n));
    else eps_in = fmin(eps_in, fmax(prm->gamma_inner * omega * mv * inv_tau, prm->eps_inner_min));
    if (eps_trace && K < eps_trace_len) eps_trace[K] = eps_in;

    /* x+ = argmin over X of the prox subproblem (Sec. 2.2) */
    memcpy(xp, x, sizeof(double) * nn);
    if (method == ORACLE_INNER_DIAG) {
      for (int32_t j = 0; j < n; ++j) xp[j] = clampd(b[j] / (qdiag[j] + inv_tau), lvs[j], uvs[j]);
    } else if (method == ORACLE_INNER_CG) {
      inner_total += inner_cg(&h, b, xp, eps_in, prm->max_inner_iter);
    } else {
      inner_total += inner_bb(&h, b, lvs, uvs, gersh, xp, eps_in, prm->max_inner_iter);
    }

    /* extrapolation and dual step (Eq. extrapolation, Eq. dual_update) */
    for (int32_t j = 0; j < n; ++j) xbar[j] = 2.0 * xp[j] - x[j];
    spmv(A, av, xbar, axb);
    for (int32_t i = 0; i < m; ++i) {
      double v = y[i] * inv_sigma + axb[i];
      yp[i] = sigma * (v - clampd(v, lcs[i], ucs[i]));
    }

    /* fixed-point residual ||z - T(z)||_omega (reading: restart metric) */
    double dx2 = 0.0, dy2 = 0.0;
    for (int32_t j = 0; j < n; ++j) dx2 += (xp[j] - x[j]) * (xp[j] - x[j]);
    for (int32_t i = 0; i < m; ++i) dy2 += (yp[i] - y[i]) * (yp[i] - y[i]);
    double fpr = sqrt(omega * dx2 + dy2 / omega);

    /* reflected Halpern step (Sec. 3.1; reading: z+ = (k+1)/(k+2) ((1+theta) T(z) - theta z) + z0/(k+2)) */
    double wk = (double)(k + 1) / (double)(k + 2);
    double ak = 1.0 / (double)(k + 2);
    double mvh2 = 0.0;
    for (int32_t j = 0; j < n; ++j) {
      xn[j] = wk * ((1.0 + prm->theta) * xp[j] - prm->theta * x[j]) + ak * xa[j];
      mvh2 += (xn[j] - x[j]) * (xn[j] - x[j]);
    }
    for (int32_t i = 0; i < m; ++i) yn[i] = wk * ((1.0 + prm->theta) * yp[i] - prm->theta * y[i]) + ak * ya[i];

    if (k == 0) {
      fpr_anchor = fpr;
      fpr_last = fpr;
    }
    int do_restart = 0;
    int check = ((K + 1) % prm->k_eval == 0) || (K + 1 >= prm->max_iter);
    if (check) {
      /* KKT at T(z) on the original data (Sec. 4.2) */
      for (int32_t j = 0; j < n; ++j) ux[j] = xp[j] * D[j];
      for (int32_t i = 0; i < m; ++i) uy[i] = yp[i] * E[i];
      spmv(A, av, xp, uAx);
      for (int32_t i = 0; i < m; ++i) uAx[i] = uAx[i] / E[i];
      spmv_t(A, av, yp, uATy);
      for (int32_t j = 0; j < n; ++j) uATy[j] = uATy[j] / D[j];
      apply_Q(Q, qv, R, rv, n, xp, uQx, rtmp, rtk);
      for (int32_t j = 0; j < n; ++j) uQx[j] = uQx[j] / D[j];
      oracle_kkt(n, m, ux, uy, uAx, uATy, uQx, c, lc, uc, lv, uv, kkt);
      double rmax = fmax(kkt[0], fmax(kkt[1], kkt[2]));

      if (!isfinite(rmax)) status = ORACLE_NUMERICAL_ERROR;
      else if (rmax <= prm->eps_tol) status = ORACLE_OPTIMAL;

      /* infeasibility with Delta = T(z) - z (Sec. 5; reading of "consecutive iterates") */
      if (!status) {
        /* primal: ytil = proj_Y(Delta y), test A^T ytil in R and the dual improvement */
        for (int32_t i = 0; i < m; ++i) ytil[i] = proj_Y(yp[i] - y[i], lcs[i], ucs[i]);
        spmv_t(A, av, ytil, t_n);
        double pviol = 0.0;
        for (int32_t j = 0; j < n; ++j) {
          pviol = fmax(pviol, fabs(t_n[j] - proj_R(t_n[j], lvs[j], uvs[j])));
          t_n[j] = -t_n[j];
        }
        double pobj = support_p(t_n, lvs, uvs, n) + support_p(ytil, lcs, ucs, m);
        double neg = pobj < 0.0 ? -pobj : 0.0;
        if (neg > 0.0 && pviol <= prm->eps_inf * neg) {
          status = ORACLE_PRIMAL_INFEASIBLE;
          double s = norminf(ytil, m);
          for (int32_t i = 0; i < m; ++i) uy[i] = ytil[i] * E[i];
          double su = norminf(uy, m);
          for (int32_t i = 0; i < m; ++i) uy[i] = su > 0 ? uy[i] / su : 0.0;
          (void)s;
        }
      }
      if (!status) {
        /* dual: d = Delta x / ||Delta x||_inf (Sec. 5.2).  Reading: the printed
         * formula normalises Delta x itself; "projected" in the text refers to
         * x+ being the projection onto X, since projecting Delta x onto
         * Recc(X) would make the first term of the test vanish identically. */
        for (int32_t j = 0; j < n; ++j) dd[j] = xp[j] - x[j];
        double dn = norminf(dd, n);
        if (dn > 0.0) {
          for (int32_t j = 0; j < n; ++j) dd[j] = dd[j] / dn;
          double cd = dot(cs, dd, n);
          double v1 = 0.0, v2 = 0.0, v3 = 0.0;
          for (int32_t j = 0; j < n; ++j) v1 = fmax(v1, fabs(dd[j] - proj_recc(dd[j], lvs[j], uvs[j])));
          spmv(A, av, dd, t_m);
          for (int32_t i = 0; i < m; ++i) v2 = fmax(v2, fabs(t_m[i] - proj_recc(t_m[i], lcs[i], ucs[i])));
          if (Q || R) {
            apply_Q(Q, qv, R, rv, n, dd, t_n, rtmp, rtk);
            v3 = norminf(t_n, n);
          }
          if (cd < -prm->eps_tol && fmax(v1, fmax(v2, v3)) <= prm->eps_inf) {
            status = ORACLE_DUAL_INFEASIBLE;
            for (int32_t j = 0; j < n; ++j) ux[j] = dd[j] * D[j];
            double su = norminf(ux, n);
            for (int32_t j = 0; j < n; ++j) ux[j] = su > 0 ? ux[j] / su : 0.0;
          }
        }
      }
      if (!status && K + 1 >= prm->max_iter) status = ORACLE_ITERATION_LIMIT;
      if (!status && now_seconds() - t_start >= prm->time_limit_s) status = ORACLE_TIME_LIMIT;
      if (status) {
        K += 1;
        break;
      }

      /* restart test (reading: fixed-point-residual criteria) */
      if (k >= 1) {
        if (fpr <= prm->restart_sufficient * fpr_anchor) do_restart = 1;
        else if (fpr <= prm->restart_necessary * fpr_anchor && fpr > fpr_last) do_restart = 1;
        else if ((double)(k + 1) >= prm->restart_artificial * (double)(K + 1)) do_restart = 1;
      }
      fpr_last = fpr;
    }

    if (do_restart) {
      /* PID update of the primal weight over the finished round (Eq. pid):
       * movement between the round's first iterate (anchor) and its last (T(z)). */
      double ddx = 0.0, ddy = 0.0;
      for (int32_t j = 0; j < n; ++j) ddx += (xp[j] - xa[j]) * (xp[j] - xa[j]);
      for (int32_t i = 0; i < m; ++i) ddy += (yp[i] - ya[i]) * (yp[i] - ya[i]);
      oracle_pid_update(&log_omega, &e_sum, &e_prev, sqrt(ddx), sqrt(ddy), prm->kp, prm->ki, prm->kd,
                        log_omega0, prm->omega_clamp);
      omega = exp(log_omega);
      tau = eta / omega;
      sigma = eta * omega;
      memcpy(xa, xp, sizeof(double) * nn);
      memcpy(ya, yp, sizeof(double) * mm);
      mv = sqrt(dx2);
      memcpy(x, xp, sizeof(double) * nn);
      memcpy(y, yp, sizeof(double) * mm);
      k = 0;
      restarts += 1;
    } else {
      mv = sqrt(mvh2);
      memcpy(x, xn, sizeof(double) * nn);
      memcpy(y, yn, sizeof(double) * mm);
      k += 1;
    }
    K += 1;
  }

  if (status != ORACLE_DUAL_INFEASIBLE)
    for (int32_t j = 0; j < n; ++j) ux[j] = xp[j] * D[j];
  if (status != ORACLE_PRIMAL_INFEASIBLE)
    for (int32_t i = 0; i < m; ++i) uy[i] = yp[i] * E[i];
  if (x_out) memcpy(x_out, ux, sizeof(double) * (size_t)n);
  if (y_out && m > 0) memcpy(y_out, uy, sizeof(double) * (size_t)m);

  res->status = status;
  res->iterations = K;
  res->inner_iterations = inner_total;
  res->restarts = restarts;
  res->r_primal = kkt[0];
  res->r_dual = kkt[1];
  res->r_gap = kkt[2];
  res->primal_obj = kkt[3];
  res->dual_obj = kkt[4];
  res->eta = eta;
  res->omega = omega;
  res->norm_A = normA;
  res->power_iters = piters;
  res->solve_seconds = now_seconds() - t_start;

  free(D); free(E); free(qv); free(av); free(cs); free(lvs); free(uvs); free(lcs); free(ucs);
  free(qdiag); free(x); free(y); free(xa); free(ya); free(xp); free(yp); free(xn); free(yn);
  free(g); free(b); free(xbar); free(axb); free(ux); free(uy); free(uAx); free(uATy); free(uQx);
  free(dd); free(ytil); free(t_n); free(t_m); free(rv); free(rtmp); free(rtk);
  return 0;
}

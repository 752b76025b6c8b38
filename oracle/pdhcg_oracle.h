/*
 * pdhcg_oracle.h — interface of the FP64 CPU oracle (test infrastructure only).
 * Independent of the CUDA library: no shared header, type or constant.
 */
#ifndef PDHCG_ORACLE_H
#define PDHCG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* CSR matrix, 0-based, host memory. */
typedef struct {
  int32_t nrows, ncols;
  const int64_t* rowptr; /* nrows + 1 */
  const int32_t* col;    /* rowptr[nrows] */
  const double* val;     /* rowptr[nrows] */
} oracle_csr;

enum {
  ORACLE_INNER_AUTO = 0,
  ORACLE_INNER_DIAG = 1,
  ORACLE_INNER_CG = 2,
  ORACLE_INNER_BB = 3
};

enum {
  ORACLE_OPTIMAL = 1,
  ORACLE_PRIMAL_INFEASIBLE = 2,
  ORACLE_DUAL_INFEASIBLE = 3,
  ORACLE_ITERATION_LIMIT = 4,
  ORACLE_TIME_LIMIT = 5,
  ORACLE_NUMERICAL_ERROR = 6
};

typedef struct {
  double eps_tol, eps_inf, time_limit_s;
  int64_t max_iter;
  double theta, kp, ki, kd;
  double gamma_inner, eps_inner_min, eps_inner_first;
  int32_t k_eval, inner, max_inner_iter, ruiz_iters;
  double restart_sufficient, restart_necessary, restart_artificial;
  int32_t power_max_iter, pad0;
  double power_tol, eta_override, omega0_override, omega_clamp;
} oracle_params;

typedef struct {
  int32_t status, inner_method;
  int64_t iterations, inner_iterations, restarts;
  double r_primal, r_dual, r_gap, primal_obj, dual_obj;
  double eta, omega, norm_A, solve_seconds;
  int32_t power_iters, pad0;
} oracle_result;

void oracle_default_params(oracle_params* p);
void oracle_ruiz(int32_t n, int32_t m, const oracle_csr* Q, const oracle_csr* A, int32_t passes,
                 double* D, double* E);
/* The same for a structured Q = P + R^T R given by P (n x n, may be NULL) and
 * R (k x n): the column maxima include the scaled diagonal of R^T R. */
void oracle_ruiz_qr(int32_t n, int32_t m, const oracle_csr* P, const oracle_csr* R, const oracle_csr* A,
                    int32_t passes, double* D, double* E);
double oracle_norm_estimate(const oracle_csr* A, const double* val, int32_t max_iter, double tol,
                            int32_t* iters_out);
int32_t oracle_inner_solve(int32_t n, const oracle_csr* Q, const double* lv, const double* uv,
                           double tau, const double* b, double eps, int32_t max_it, int32_t method,
                           double* x);
void oracle_kkt(int32_t n, int32_t m, const double* x, const double* y, const double* Ax,
                const double* ATy, const double* Qx, const double* c, const double* lc,
                const double* uc, const double* lv, const double* uv, double* out6);
void oracle_pid_update(double* log_omega, double* e_sum, double* e_prev, double dx, double dy,
                       double kp, double ki, double kd, double log_omega0, double clamp);
int oracle_solve(int32_t n, int32_t m, const oracle_csr* Q, const oracle_csr* A, const double* c,
                 const double* lc, const double* uc, const double* lv, const double* uv,
                 const oracle_params* prm, const double* x_init, const double* y_init,
                 double* x_out, double* y_out, oracle_result* res, double* eps_trace,
                 int32_t eps_trace_len);

/* The same with Q = P + R^T R (R: k x n), applied as P v + R^T (R v). */
int oracle_solve_qr(int32_t n, int32_t m, const oracle_csr* P, const oracle_csr* R, const oracle_csr* A,
                    const double* c, const double* lc, const double* uc, const double* lv,
                    const double* uv, const oracle_params* prm, const double* x_init,
                    const double* y_init, double* x_out, double* y_out, oracle_result* res);

#ifdef __cplusplus
}
#endif
#endif

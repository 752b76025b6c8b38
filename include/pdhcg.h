/*
 * pdhcg.h — C ABI of the B300 (sm_103a) PDHCG-II solver library (libpdhcg.so).
 *
 * Problem (Sec. 2, Eq. QP):
 *     minimize   1/2 x^T Q x + c^T x
 *     subject to lc <= A x <= uc,   lv <= x <= uv
 * with Q symmetric positive semidefinite (full symmetric CSR storage, or NULL
 * for Q = 0), A an m x n CSR matrix, and +-INFINITY marking an absent bound
 * (an equality row has lc == uc).
 *
 * Method: the PDHCG-II iteration — the PDHG step of Sec. 2.1 (Eq. pdhcg_update)
 * with the primal subproblem solved by the diagonal closed form, conjugate
 * gradients or projected gradient with Barzilai-Borwein steps (Sec. 2.2), the
 * reflected Halpern scheme (Sec. 3.1), step sizes tau = eta/omega,
 * sigma = eta*omega with eta = 0.998/||A|| and the PID primal weight (Sec. 3.2,
 * Eq. pid), the adaptive inner tolerance (Sec. 3.3), the KKT stopping rule
 * (Sec. 4.2) and the infeasibility tests (Sec. 5.1, 5.2).  Every floating-point
 * step of the method runs in CUDA kernels on the device.
 *
 * Conventions for every entry point:
 *   - Return value: PDHCG_OK (0) on success, a negative PDHCG_E_* code on
 *     failure (pdhcg_strerror() names it; pdhcg_last_error() gives a detail
 *     message for the calling thread).  No C++ exception crosses the ABI.
 *   - Host pointers unless the name ends in _dev (then device pointers on the
 *     handle's device).  The library copies every input it keeps; the caller
 *     keeps ownership of its buffers.  Output arrays are caller-allocated.
 *   - A handle is not thread-safe: one thread at a time per handle.
 *   - CSR: 0-based, rowptr has nrows+1 entries, rowptr[0] = 0, nondecreasing;
 *     column indices in [0, ncols); duplicates are rejected; nnz < 2^31.
 */
#ifndef PDHCG_H
#define PDHCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PDHCG_API_VERSION 1

/* ---- return codes ---- */
#define PDHCG_OK 0
#define PDHCG_PENDING 1          /* pdhcg_poll: request not finished yet          */
#define PDHCG_E_INVALID (-1)     /* bad argument or malformed problem data        */
#define PDHCG_E_OOM (-2)         /* device allocation failed / over HBM budget    */
#define PDHCG_E_CUDA (-3)        /* a CUDA runtime call failed                    */
#define PDHCG_E_BUSY (-4)        /* server queue full; retry later                */
#define PDHCG_E_NOT_FOUND (-5)   /* unknown ticket                                */
#define PDHCG_E_DEVICE_TIMEOUT (-6) /* a bounded device-side wait gave up          */

/* ---- solver outcome (pdhcg_result.status) ---- */
#define PDHCG_UNSOLVED 0
#define PDHCG_OPTIMAL 1            /* max(r_primal, r_dual, r_gap) <= eps_tol (Sec. 4.2) */
#define PDHCG_PRIMAL_INFEASIBLE 2  /* Farkas ray found (Sec. 5.1); y_out holds it         */
#define PDHCG_DUAL_INFEASIBLE 3    /* unbounded direction found (Sec. 5.2); x_out holds it */
#define PDHCG_ITERATION_LIMIT 4
#define PDHCG_TIME_LIMIT 5
#define PDHCG_NUMERICAL_ERROR 6

/* ---- arithmetic of the iteration ---- */
#define PDHCG_FP64 0   /* matrix values, vectors and reductions in double                  */
#define PDHCG_FP32 1   /* FP32 matrix values, vectors and SpMV accumulation; FP64 inner
                          products, KKT norms, restart/PID decisions and certificates       */
#define PDHCG_MIXED 2  /* FP32 matrix values, FP64 vectors and accumulation                 */
#define PDHCG_DFLOAT 3 /* FP32 matrix values; vectors and accumulation in double-float (an
                          unevaluated sum of two FP32 values, ~48-bit significand) on the
                          FP32 pipe; FP64 inner products, KKT norms and decisions as above  */

/* ---- primal subproblem solver (Sec. 2.2) ---- */
#define PDHCG_INNER_AUTO 0  /* diagonal Q: closed form; else finite bounds: BB; else CG */
#define PDHCG_INNER_DIAG 1  /* closed form; only valid for diagonal Q                    */
#define PDHCG_INNER_CG 2    /* conjugate gradients; only valid when no bound is finite   */
#define PDHCG_INNER_BB 3    /* projected gradient with Barzilai-Borwein steps            */
#define PDHCG_INNER_CG_LIFTED 4 /* every finite variable bound becomes a row e_j^T x of A
                                   (with that bound as its row bounds) and the variables
                                   become free, so the subproblem is an unconstrained SPD
                                   solve: closed form for diagonal Q, else CG.  The
                                   solution's y holds the original rows' duals only;
                                   residuals and iterations refer to the lifted problem */

typedef struct {
  int32_t nrows, ncols;
  int64_t nnz;
  const int64_t* rowptr; /* nrows + 1 */
  const int32_t* col;    /* nnz       */
  const double* val;     /* nnz       */
} pdhcg_csr;

/* Solver parameters.  Fill with pdhcg_default_params() first; struct_size is
 * checked so that older callers keep working when fields are appended. */
typedef struct {
  uint32_t struct_size;
  int32_t precision;          /* PDHCG_FP64 (default) / PDHCG_FP32 / PDHCG_MIXED / PDHCG_DFLOAT */
  double eps_tol;             /* KKT tolerance, Sec. 4.2 (1e-6)                              */
  double eps_inf;             /* infeasibility tolerance eps_inf, Sec. 5 (1e-8)              */
  double time_limit_s;        /* wall-clock limit measured on the device timer (3600)        */
  int64_t max_iter;           /* outer PDHG steps (1e6)                                      */
  double theta;               /* Halpern reflection parameter, Sec. 3.1 (1.0)                */
  double kp, ki, kd;          /* PID gains, Eq. pid (0.99, 0.01, 0.0)                        */
  double gamma_inner;         /* gamma of the adaptive inner tolerance, Sec. 3.3 (5e-4)      */
  double eps_inner_min;       /* eps_min, Sec. 3.3 (1e-9)                                    */
  double eps_inner_first;     /* first inner tolerance = this * max(1, ||b||) (1e-2)         */
  int32_t k_eval;             /* KKT / infeasibility / restart check period (64)             */
  int32_t inner;              /* PDHCG_INNER_*                                               */
  int32_t max_inner_iter;     /* cap on CG / BB steps per outer step (1000)                  */
  int32_t ruiz_iters;         /* Ruiz equilibration passes, 0 = no scaling (10)              */
  double restart_sufficient;  /* restart if FPR <= this * FPR(anchor) (0.2)                  */
  double restart_necessary;   /* ... or FPR <= this * FPR(anchor) and FPR grew (0.8)         */
  double restart_artificial;  /* ... or round length >= this * total steps (0.36)            */
  int32_t power_max_iter;     /* cap on Lanczos steps of the ||A||_2 estimate (1000)         */
  int32_t lanes_override;     /* force lanes per CSR row (1..32, power of 2); 0 = tuned      */
  double power_tol;           /* relative change of the ||A||_2 estimate that stops it (1e-8)*/
  double eta_override;        /* > 0: use this eta instead of 0.998/||A||                    */
  double omega0_override;     /* > 0: use this initial primal weight                         */
  double omega_clamp;         /* omega kept within [omega0/c, omega0*c] (1e5)                */
  int32_t group_blocks;       /* CTAs per instance in pdhcg_solve: 0 = auto                  */
  int32_t device_timeout_ms;  /* bound on any device-side wait (8000)                        */
  /* Row layout (read at create; 0 = default): rows are sorted by length inside
   * windows of sell_sigma rows and packed 32 to a slice, one lane per row
   * (1024); rows longer than long_row get a warp each (64); rows of huge_row
   * entries or more a whole CTA (2048). */
  int32_t sell_sigma, long_row, huge_row;
  int32_t pool_ctas_per_sm;   /* cap on resident pool CTAs per SM in batched solves: 0 = as
                                 many as fit                                                 */
  int32_t pipeline;           /* pdhcg_solve of a large problem as a CUDA graph of one kernel
                                 per phase, with device-driven conditional nodes: 0 = when
                                 the problem is large enough to fill the GPU (and Q is not
                                 structured), 1 = always (error if the graph cannot be
                                 built), -1 = never (the persistent multi-CTA kernel)         */
  int32_t pool_threads;       /* threads of a pool CTA, the one-CTA solve of a small problem
                                 (alone, batched or served): 0 = 256 (two per SM), or 128
                                 (four per SM when a problem's vectors fit a quarter of the
                                 SM's shared memory).  Part of the arithmetic's definition:
                                 the two widths sum in different orders, and a problem gives
                                 the same bits alone, batched or served only at one width.
                                 A batch takes its first problem's value.  In a batched
                                 launch that also holds multi-CTA groups the pool CTAs are
                                 256 threads wide whatever this says                          */
} pdhcg_params;

typedef struct {
  int32_t status;             /* PDHCG_OPTIMAL, ... (see above)                              */
  int32_t inner_method;       /* the PDHCG_INNER_* actually used                             */
  int64_t iterations;         /* outer PDHG steps                                            */
  int64_t inner_iterations;   /* CG / BB steps summed over all outer steps                   */
  int64_t restarts;
  double r_primal, r_dual, r_gap; /* Sec. 4.2 residuals at the returned point (unscaled data)*/
  double primal_obj, dual_obj;
  double eta, omega, norm_A;  /* step size, final primal weight, ||A||_2 estimate (scaled) */
  double solve_seconds;       /* device-timer duration of the solve                          */
  int32_t power_iters;        /* Lanczos steps taken by the ||A||_2 estimate                 */
  int32_t precision;
  double latency_seconds;     /* serving loop: pdhcg_submit to result ready (wall clock); 0 otherwise */
  int32_t form;               /* how the solve ran: 0 one CTA (pool), 1 a multi-CTA group of the
                                 persistent kernel, 2 the pipeline graph (pdhcg_params.pipeline) */
  int32_t reserved;
} pdhcg_result;

typedef struct pdhcg_problem pdhcg_t;
typedef struct pdhcg_server pdhcg_server_t;

/* Fill p with the defaults listed above.  Returns PDHCG_E_INVALID for NULL. */
int pdhcg_default_params(pdhcg_params* p);

/* Validate the problem, copy it to the device and run the setup of the method
 * on the device: Ruiz equilibration of [Q A^T; A 0] (reading of the paper's
 * "system scaling"), the Lanczos estimate of ||A||_2 for
 * eta = 0.998/||A|| (Sec. 3.2), Gershgorin bound of Q for the BB step range,
 * and the initial primal weight.  Q may be NULL (LP).  A must be given even
 * when m = 0 (nrows = 0).  lc, uc: m entries; c, lv, uv: n entries.
 * cuda_stream: a cudaStream_t (NULL = the default stream) used for all work on
 * this handle.  On success *out owns device memory released by pdhcg_destroy.
 * Errors: E_INVALID (shape, NaN, lc > uc, lv > uv, lc = +inf, non-symmetric Q,
 * duplicate entries), E_OOM, E_CUDA. */
int pdhcg_create(const pdhcg_csr* Q, const pdhcg_csr* A, const double* c, const double* lc,
                 const double* uc, const double* lv, const double* uv, const pdhcg_params* params,
                 void* cuda_stream, pdhcg_t** out);

/* Structured quadratic term Q = P + R^T R (Sec. 2.2): P n x n symmetric (or NULL
 * for P = 0), R k x n (k >= 1).  R^T R is never formed: every product with Q is
 * P v + R^T (R v), the k-vector R v taken by a phase of its own.  Other
 * arguments and ownership as pdhcg_create.  Scaling reads the Ruiz factors off
 * P and A only; the step range of the BB inner solver bounds ||R D||_2^2 by
 * ||R D||_1 ||R D||_inf.  The handle works with every solve entry point. */
int pdhcg_create_qr(const pdhcg_csr* P, const pdhcg_csr* R, const pdhcg_csr* A, const double* c,
                    const double* lc, const double* uc, const double* lv, const double* uv,
                    const pdhcg_params* params, void* cuda_stream, pdhcg_t** out);

/* One problem of a batch creation (same meaning as the pdhcg_create arguments). */
typedef struct {
  const pdhcg_csr* Q; /* NULL = no quadratic term */
  const pdhcg_csr* A;
  const double *c, *lc, *uc, *lv, *uv;
} pdhcg_problem_data;

/* Create count handles at once: host validation runs on several threads, all
 * handles share one device allocation (released with the last handle), every
 * input is staged through pinned memory, and the device setup of all problems
 * runs in one launch (one CTA per problem).  On failure no handle is created
 * and pdhcg_last_error() names the first bad problem.  out: count handles. */
int pdhcg_create_batch(int count, const pdhcg_problem_data* problems, const pdhcg_params* params,
                       void* cuda_stream, pdhcg_t** out);

/* Solve from host buffers (blocking).  x0 (n) / y0 (m) are optional warm
 * starts (NULL = x = proj_X(0), y = 0).  x_out (n) / y_out (m) may be NULL.
 * Host<->device copies of the warm start and of the result are part of the call.
 * For PDHCG_PRIMAL_INFEASIBLE y_out holds the ray (infinity norm 1); for
 * PDHCG_DUAL_INFEASIBLE x_out holds the ray. */
int pdhcg_solve(pdhcg_t* prob, const double* x0, const double* y0, pdhcg_result* res,
                double* x_out, double* y_out);

/* Same with device-resident buffers (double, on the handle's device); the
 * result struct is still returned in host memory.  Blocking. */
int pdhcg_solve_dev(pdhcg_t* prob, const double* x0_dev, const double* y0_dev, pdhcg_result* res,
                    double* x_out_dev, double* y_out_dev);

/* Solve count independent problems in one persistent launch: every CTA takes
 * the next unsolved instance from a device work queue and solves it alone
 * (instances whose size calls for it run on groups of CTAs).  All handles must
 * share precision and stream.  x_out / y_out: arrays of count host pointers
 * (each may be NULL), or NULL.  res: count results. */
int pdhcg_solve_batch(pdhcg_t* const* probs, int count, pdhcg_result* res, double* const* x_out,
                      double* const* y_out);

/* Allocation-free form of pdhcg_solve_batch.  The paper has no counterpart: it
 * solves one QP per call; this is a deployment interface of this library.
 *
 * For callers that must not allocate while solving: a real-time loop (e.g. a
 * model-predictive controller re-solving every control period) cannot take the
 * latency of cudaMalloc or the device-wide synchronisation of cudaFree, and a
 * process whose device memory is fully reserved by its own pool or budget would
 * see such an allocation fail.  The per-call scratch (solver states, instance
 * descriptors, work queue) lives in one static device array of about 1.1 MB per
 * device, so this call makes no cudaMalloc / cudaFree or other allocating call.
 *
 * probs, count: as pdhcg_solve_batch (same precision, device and stream);
 *   0 <= count <= PDHCG_NOALLOC_MAX_INSTANCES, else PDHCG_E_INVALID with a
 *   message naming the limit.
 * res: count results in host memory, or NULL.
 * x_out_dev / y_out_dev: arrays of count DEVICE pointers (double, n_i resp. m_i
 *   elements on the handles' device; each may be NULL), or NULL.  The kernel
 *   writes the solutions there directly; the caller owns these buffers.
 * Blocking: returns after the launch finished.  The queue cursor and error flag
 *   in the scratch must start at zero, and every call resets them (with the
 *   states and descriptors) before its launch.
 * Set-up: the first call on each device looks up the scratch's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call before
 *   any stream capture on that device.  The call copies from host memory and
 *   synchronises its stream, so it must not be called while that stream is
 *   being captured into a CUDA graph.
 * Concurrency: the scratch is one per device per process, so overlapping calls
 *   would race on it; the library serialises calls on a process-wide lock.
 * Results equal pdhcg_solve_batch's for the same handles. */
#define PDHCG_NOALLOC_MAX_INSTANCES 1024
int pdhcg_solve_batch_noalloc(pdhcg_t* const* probs, int count, pdhcg_result* res,
                              double* const* x_out_dev, double* const* y_out_dev);

/* ---- autotuner of the launch shape and row layout ----
 * The paper has no counterpart (its kernels are not described).  Candidate
 * settings of the row layout (sell_sigma, long_row, huge_row) and of the launch
 * shape (for a single problem: the pipeline form against the persistent kernel
 * at several group_blocks; for a batch: pool_threads and pool_ctas_per_sm) are
 * timed on the device with CUDA events over a fixed number of PDHG steps of
 * the given problems (count == 1: one multi-CTA solve; count > 1: one batched
 * launch), and the fastest is written into *params.  The defaults are kept
 * unless a candidate is faster by more than 3 %.  Results are cached per
 * shape class (precision, batch or single, inner solver, size and row-length
 * histogram bucket) for the life of the process: a later call of the same
 * class returns the cached choice without timing (out->from_cache = 1).
 * params: in, the base parameters; out, with the chosen fields set.
 * The call creates and destroys its own handles and synchronises stream.
 * Errors as pdhcg_create_batch. */
typedef struct {
  int32_t sell_sigma, long_row, huge_row, group_blocks, pool_ctas_per_sm; /* chosen (0 = default) */
  int32_t pipeline;                 /* chosen pdhcg_params.pipeline                              */
  int32_t candidates;               /* configurations timed (0 when taken from the cache)       */
  int32_t from_cache;               /* 1: the shape class was tuned before in this process       */
  double seconds_per_step;          /* chosen configuration: device seconds per PDHG step       */
  double default_seconds_per_step;  /* the defaults, timed the same way                          */
  int32_t pool_threads;             /* chosen pdhcg_params.pool_threads (0 = default)            */
  int32_t reserved;
} pdhcg_tuning;
int pdhcg_autotune(int count, const pdhcg_problem_data* problems, pdhcg_params* params, void* cuda_stream,
                   pdhcg_tuning* out);

/* eta used by the iteration and the ||A||_2 estimate of the scaled A (Sec. 3.2). */
int pdhcg_get_eta(const pdhcg_t* prob, double* eta, double* norm_A);

/* Scaling vectors: x_original = D .* x_scaled, y_original = E .* y_scaled. */
int pdhcg_get_scaling(const pdhcg_t* prob, double* D, double* E);

/* Sizes of a handle: n, m, device bytes held. */
int pdhcg_get_info(const pdhcg_t* prob, int32_t* n, int32_t* m, size_t* device_bytes);

/* CUDA device ordinal the handle's data lives on (the device current at create). */
int pdhcg_get_device(const pdhcg_t* prob, int32_t* device);

/* Profiling aid: device-timer seconds of the last pdhcg_solve / pdhcg_solve_dev /
 * pdhcg_solve_batch of this handle, as seen by one thread of the first CTA
 * (all zero unless the library was built with PDHCG_PHASE_TIMERS=1), split into 8
 * categories: [0] Phase I (A^T y, subproblem start), [1] inner-solver row phases
 * (Q p), [2] inner-solver elementwise phases, [3] Phase II (A xbar, dual step,
 * Halpern), [4] KKT / infeasibility checks, [5] group barriers and reductions,
 * [6] restarts and output, [7] unused. */
int pdhcg_get_phase_times(const pdhcg_t* prob, double* seconds8);

void pdhcg_destroy(pdhcg_t* prob);

/* ---- serving loop (continuous batching) ----
 * A host scheduler thread admits submitted problems while their device
 * footprint fits hbm_budget_bytes and a slot (max_slots) is free, keeps every
 * live solve's iterates and restart state resident on the device, and packs
 * all live solves into shared persistent launches that each advance every live
 * solve for a slice of about 10 ms of device time (each solve pauses at the
 * first 16-step boundary past it, so slots of unequal cost stop together);
 * finished solves free their slot and memory at the next slice boundary, where
 * waiting requests are admitted.  The paper solves one problem at a time and
 * has no counterpart of this loop. */
typedef struct {
  uint64_t submitted, admitted, completed, rejected;
  uint64_t launches;
  int32_t live, queued;
  size_t hbm_in_use;
  /* scheduler wall time so far: admission (creation and device setup of the
   * admitted problems), slices (launch to end), retirement (results back) */
  double admit_seconds, slice_seconds, retire_seconds;
} pdhcg_server_stats;

int pdhcg_server_create(size_t hbm_budget_bytes, int max_slots, const pdhcg_params* params,
                        void* cuda_stream, pdhcg_server_t** out);
/* Copy the problem into the server's queue (non-blocking).  Returns
 * PDHCG_E_BUSY if the queue holds max_queue requests already, PDHCG_E_OOM if
 * the problem alone can never fit the budget.  *ticket identifies it. */
int pdhcg_submit(pdhcg_server_t* srv, const pdhcg_csr* Q, const pdhcg_csr* A, const double* c,
                 const double* lc, const double* uc, const double* lv, const double* uv,
                 uint64_t* ticket);
/* PDHCG_PENDING while queued or running; PDHCG_OK once finished, filling res
 * and (optionally) x_out / y_out; the ticket is then forgotten. */
int pdhcg_poll(pdhcg_server_t* srv, uint64_t ticket, pdhcg_result* res, double* x_out,
               double* y_out);
int pdhcg_server_get_stats(pdhcg_server_t* srv, pdhcg_server_stats* stats);
void pdhcg_server_destroy(pdhcg_server_t* srv);

const char* pdhcg_strerror(int code);
const char* pdhcg_last_error(void);

/* Self-test of the bounded device waits (failure detection without a fault).
 * Every spin-wait of the solve kernel (the group barrier, queue waits) gives
 * up after params.device_timeout_ms, sets a device error flag and returns, so
 * that the host reports PDHCG_E_DEVICE_TIMEOUT and the context stays usable.
 * This call makes both kinds of wait run out on purpose, on the current
 * device: a two-CTA group barrier whose second CTA never arrives, and a wait
 * on a flag that nothing sets, each limited to timeout_us microseconds
 * (1 .. 1e7).  Returns PDHCG_E_DEVICE_TIMEOUT when both gave up and reported
 * it (the designed outcome), PDHCG_E_CUDA if a wait did not report, and
 * PDHCG_E_INVALID for a timeout out of range.  *waited_seconds (may be NULL):
 * device time spent in the two waits. */
int pdhcg_selftest_bounded_wait(int32_t timeout_us, double* waited_seconds);

#ifdef __cplusplus
}
#endif
#endif /* PDHCG_H */

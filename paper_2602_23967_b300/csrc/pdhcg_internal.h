// pdhcg_internal.h — layouts shared by the host layer and the CUDA kernels of libpdhcg.
#pragma once
#include <cstdint>

#include "pdhcg.h"

namespace pdhcg {

// Reduction slots available per group reduction (the KKT / infeasibility check
// uses the most).
constexpr int kSlots = 24;
// Bytes of one group's barrier block (34 lines of 128 bytes).
constexpr size_t kBarBytes = 34 * 128;

// Bound-type code of a row or variable: bit 0 = lower bound finite,
// bit 1 = upper bound finite.
enum : int8_t { kFree = 0, kLowOnly = 1, kUpOnly = 2, kBoxed = 3 };

// Parameters the device loop reads (host fills from pdhcg_params).
struct DevParams {
  double eps_tol, eps_inf, time_limit_ns;
  int64_t max_iter;
  double theta, kp, ki, kd;
  double gamma_inner, eps_inner_min, eps_inner_first;
  double restart_sufficient, restart_necessary, restart_artificial, omega_clamp;
  int32_t k_eval, max_inner_iter;
};

// Scalar state of one solve, FP64, kept in device memory between launches so a
// solve can be paused at a check boundary and resumed (serving loop).
struct SolverState {
  int64_t K;            // PDHG steps done
  int64_t k;            // Halpern index since the last restart
  int64_t inner_total;  // CG / BB steps
  int64_t restarts;
  double omega, log_omega, log_omega0, e_sum, e_prev;
  double tau, sigma, eta, norm_A;
  double eps_in, mv, fpr_anchor, fpr_last;
  double r_primal, r_dual, r_gap, pobj, dobj;
  double t_start_ns, t_end_ns;
  double gersh, omega0;
  double bscale, cinf;  // max(||lc||_inf, ||uc||_inf) over finite entries; ||c||_inf
  // device-timer nanoseconds seen by thread 0 of the group's first CTA, per
  // category: 0 Phase I, 1 inner row phases, 2 inner elementwise, 3 Phase II,
  // 4 checks, 5 group barriers/reductions, 6 restarts and output, 7 unused
  double tm[8];
  int32_t status;       // PDHCG_* status, 0 while running
  int32_t cur;          // which of the two x / y buffers holds the current iterate
  int32_t started;      // 0 until the first launch initialised the iterates
  int32_t method;       // PDHCG_INNER_DIAG / CG / BB
  int32_t power_iters;
  int32_t device_error; // a bounded device wait gave up
  int32_t form;         // how the last launch ran it: 0 pool CTA, 1 multi-CTA group, 2 pipeline graph
  int32_t pad_;
};

// With FP32 matrix values, lo holds each scaled value's rounding remainder
// float(v - double(float(v))), so val + lo reproduces the FP64 value to about
// 2^-48 relative (used by the KKT checks and the defect correction); null in
// FP64 mode.
template <class T>
struct Csr {
  int32_t nrows = 0;
  int32_t nnz = 0;
  const int32_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const T* val = nullptr;
  const float* lo = nullptr;
};

// SELL-C-sigma slices (C = 32 rows, one per lane) of one matrix of a row space.
// Element j of slot (slice s, lane l) sits at ptr[s] + 32*j + l; padding has
// value 0.  Rows listed as long / huge are not in the slices.
template <class T>
struct Sell {
  const int64_t* ptr = nullptr;  // nslices + 1
  const int32_t* col = nullptr;
  const T* val = nullptr;
  const float* lo = nullptr;     // remainders in slice order (see Csr)
};

// Row space (the n variable rows, or the m constraint rows) in SELL form.
struct SpaceLayout {
  int32_t nslices = 0, nlong = 0, nhuge = 0;
  const int32_t* perm = nullptr;   // nslices*32 row ids (-1 = padding slot)
  const int32_t* longs = nullptr;  // rows summed by one warp each (CSR)
  const int32_t* huges = nullptr;  // rows summed by a whole CTA each (CSR)
  // per-CTA ranges of slices / long rows / huge rows (part_blocks + 1 each; null = all)
  const int32_t* slice_part = nullptr;
  const int32_t* long_part = nullptr;
  const int32_t* huge_part = nullptr;
};

// Everything a kernel needs to know about one instance.  MatT: matrix value
// type; VecT: iterate / vector type.
template <class MatT, class VecT>
struct Inst {
  int32_t n = 0, m = 0;
  int32_t has_q = 0;
  int32_t lanes_var = 4, lanes_con = 4;  // CSR lanes per row in the n-space / m-space phases
  Csr<MatT> Q, A, AT;                    // scaled matrices; AT is the explicit transpose of A
  Sell<MatT> Qs, As, ATs;                // the same values in SELL form
  SpaceLayout vsp, csp;                  // variable-row and constraint-row spaces
  // Row partitions for multi-CTA groups: var_part / con_part hold part_blocks+1
  // row offsets (nnz-balanced); long rows sit alone in their range.
  const int32_t* var_part = nullptr;
  const int32_t* con_part = nullptr;
  int32_t part_blocks = 0;
  int32_t long_row = 1 << 30;            // rows at least this long use the whole CTA
  // Structured objective Q = P + R^T R (Sec. 2.2): Q / Qs hold [P | R^T] with
  // columns n.. n+k-1 addressing R v, which a phase over the k rows of R puts in
  // rt1 (rt2: a second product in the checks).  k = 0: plain Q.
  int32_t k = 0;
  Csr<MatT> R;
  Sell<MatT> Rsl;
  SpaceLayout rsp;
  VecT* rt1 = nullptr;
  VecT* rt2 = nullptr;
  // scaled problem data.  With FP32 matrix values c, lc and uc are the
  // defect-corrected copies the iteration reads (reset from c_o, lc_o, uc_o at
  // the start of a solve, shifted at every check).
  VecT *c = nullptr, *lc = nullptr, *uc = nullptr;
  const VecT *lv = nullptr, *uv = nullptr, *qdiag = nullptr;
  const int8_t *vtype = nullptr, *ctype = nullptr;
  // original-space data for the KKT residuals (double)
  const double *D = nullptr, *E = nullptr, *c_o = nullptr, *lv_o = nullptr, *uv_o = nullptr,
               *lc_o = nullptr, *uc_o = nullptr;
  double bscale = 0.0;  // max(||lc||_inf, ||uc||_inf) over finite entries
  double cinf = 0.0;    // ||c||_inf
  // iterate / work vectors
  VecT *xb0 = nullptr, *xb1 = nullptr, *yb0 = nullptr, *yb1 = nullptr;
  VecT *xT = nullptr, *yT = nullptr, *xa = nullptr, *ya = nullptr;
  VecT *r = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr;
  VecT *bv = nullptr, *grad = nullptr, *gprev = nullptr, *xprev = nullptr;
  VecT* xbar = nullptr;  // 2 x+ - x, written once x+ is known (one gather per nonzero in Phase II)
  // warm start and outputs (device, double; may be null)
  const double *x_init = nullptr, *y_init = nullptr;
  double *x_out = nullptr, *y_out = nullptr;
  SolverState* st = nullptr;
  DevParams prm;
};

// Shared-memory bytes the vectors of an (n, m) instance take when a pool CTA
// keeps them on chip: 9 n-vectors (+4 for CG / BB), 6 m-vectors, bound codes,
// and the SELL slice offsets of the row spaces (at most n/32 + 1 slices each;
// A^T's and A's, and Q's with an inner solver).
inline __host__ __device__ size_t smem_vector_bytes(int n, int m, int method, size_t vec_bytes) {
  const bool inner = method == 2 || method == 3;
  const size_t nv = 9 + (inner ? 4 : 0);
  auto al = [](size_t b) { return (b + 15) & ~size_t(15); };
  const size_t ptrs = (inner ? 2 : 1) * al((size_t(n) / 32 + 2) * 8) + al((size_t(m) / 32 + 2) * 8);
  return nv * al(size_t(n) * vec_bytes) + 6 * al(size_t(m) * vec_bytes) + al(size_t(n)) + al(size_t(m)) + ptrs;
}

// How one launch of the solve kernel maps CTAs to instances.
struct LaunchPlan {
  // Multi-CTA groups occupy CTAs [0, group_blocks); group g owns
  // [g_first[g], g_first[g] + g_nblk[g]) and solves instance g_inst[g].
  int32_t ngroups = 0;
  int32_t group_blocks = 0;
  const int32_t* g_first = nullptr;
  const int32_t* g_nblk = nullptr;
  const int32_t* g_inst = nullptr;
  unsigned long long* g_bar = nullptr;  // barrier blocks, kBarBytes per group (zeroed before launch)
  double* g_part = nullptr;             // partial sums: group g at g_part_off[g], 2*kSlots*nblk
  const int64_t* g_part_off = nullptr;
  // Remaining CTAs take single-CTA instances from a queue.
  int32_t npool = 0;
  const int32_t* pool_inst = nullptr;
  int32_t* pool_next = nullptr;         // atomic cursor (zeroed before launch)
  // Slice limits for the serving loop: a solve pauses at the first check
  // boundary after it has done iter_budget steps in this launch (0 = none).
  int64_t iter_budget = 0;
  // Serving slices: a single-CTA solve also pauses, at a step boundary, once
  // this many nanoseconds of device time have passed since it resumed (0 = none),
  // so that every slot of a launch stops at about the same time.
  uint64_t slice_ns = 0;
  // Pool CTAs copy an instance's vectors into dynamic shared memory when they
  // fit in this many bytes (0 = never); see smem_vector_bytes().
  int64_t smem_vec_bytes = 0;
  // Threads of a pool CTA in a launch without groups: 256 (the group kernel's
  // width) or 128 (the narrow pool kernel); see pdhcg_params.pool_threads.
  int32_t pool_bs = 256;
  uint64_t timeout_ns = 8000000000ull;  // bound on any device wait
  int32_t* err = nullptr;               // set to 1 when a bounded wait gave up
  // Some instance has a structured Q = P + R^T R: launch the kernel variant
  // with the R phases (the plain variant has none of their cost).
  int32_t structured = 0;
  // Every pool instance uses the closed form (diagonal Q) and none is
  // structured: launch the variant without the CG / BB code.
  int32_t diag_only = 0;
};

}  // namespace pdhcg

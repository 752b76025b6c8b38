// host_problem.h — host-side representation of a pdhcg_t handle.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "pdhcg_internal.h"

namespace pdhcg {

void set_error(const std::string& msg);

// Validated, canonical host copy of a problem (integer layout work only: the
// method's arithmetic all runs on the device).
struct HostQP {
  int32_t n = 0, m = 0;
  int32_t m_user = 0;  // rows of the caller's problem (m also counts lifted bound rows)
  // structured objective Q = P + R^T R (Sec. 2.2): R is k x n; the Q arrays then
  // hold [P | R^T] (n x (n + k)), i.e. Q v = [P | R^T] [v; R v]
  int32_t k = 0;
  std::vector<int32_t> Rp, Rc;
  std::vector<double> Rv;
  bool has_q = false, diag_q = true, any_box = false;
  std::vector<int32_t> Qp, Qc, Ap, Ac, ATp, ATc;
  std::vector<double> Qv, Av, ATv;
  std::vector<double> c, lc, uc, lv, uv;
  std::vector<int8_t> vtype, ctype;
};

// Validate and canonicalise; returns PDHCG_OK or PDHCG_E_INVALID (with set_error).
int build_host_qp(const pdhcg_csr* Q, const pdhcg_csr* A, const double* c, const double* lc,
                  const double* uc, const double* lv, const double* uv, HostQP* out,
                  const pdhcg_csr* R = nullptr);
// PDHCG_INNER_CG_LIFTED: append a row e_j^T for every variable with a finite
// bound (row bounds = that variable's bounds) and make every variable free.
void lift_box_rows(HostQP* h);

// SELL-C-sigma layout of a row space with up to two matrices (integer part;
// values are filled on the device from the scaled CSR values).
struct SellHost {
  int32_t nslices = 0;
  std::vector<int32_t> perm;   // nslices*32, -1 = padding
  std::vector<int32_t> longs;  // rows handled warp-per-row
  std::vector<int32_t> huges;  // rows handled CTA-per-row
  std::vector<int64_t> ptr[2];
  std::vector<int32_t> col[2];
};
constexpr int kSellSigma = 1024;
constexpr int64_t kLongRow = 64;
constexpr int64_t kHugeRow = 2048;
// Row layout: rows sorted by length inside windows of sigma rows; rows longer
// than long_row are summed by a warp each, rows of huge_row or more by a CTA.
struct SellLayout {
  int32_t sigma = kSellSigma;
  int64_t long_row = kLongRow;
  int64_t huge_row = kHugeRow;
};
// The layout a params struct asks for (0 fields = the defaults above).
SellLayout sell_layout_of(const pdhcg_params& p);
void build_sell(int32_t nrows, int nmat, const std::vector<int32_t>* rp[2],
                const std::vector<int32_t>* ci[2], SellHost* out, const SellLayout& lay = SellLayout{});
// Autotuner selection: the index of the fastest timing, except that candidate
// 0 (the defaults) is kept unless another one is faster by more than the
// relative margin; negative or non-finite timings (failed runs) never win.
int pick_fastest(const std::vector<double>& seconds, double margin);
// Split items with the given weights into nblk contiguous ranges (nblk + 1 bounds).
std::vector<int32_t> split_balanced(const std::vector<int64_t>& w, int nblk);

// Batched and served solves: an instance whose PDHG step touches fewer than
// this many nonzeros and vector entries runs on one pool CTA; a larger one on
// a multi-CTA group.
constexpr int64_t kGroupWork = 150000;

// Device bytes a problem will hold (for admission control).
size_t device_footprint(const HostQP& h, int precision);

struct PartitionSet {
  int nblk = 0;
  int32_t* d_buf = nullptr;  // 11 tables of nblk + 1 entries
  bool owned = false;        // d_buf is a cudaMalloc of its own (else it lives in the arena)
  int32_t *v_slice = nullptr, *v_long = nullptr, *v_huge = nullptr;
  int32_t *c_slice = nullptr, *c_long = nullptr, *c_huge = nullptr;
  int32_t *v_even = nullptr, *c_even = nullptr;  // even row splits for elementwise work
  int32_t *r_slice = nullptr, *r_long = nullptr, *r_huge = nullptr;  // rows of R (structured Q)
};

}  // namespace pdhcg

struct pdhcg_problem;

namespace pdhcg {

struct CreateInput {
  const pdhcg_csr *Q, *A;
  const double *c, *lc, *uc, *lv, *uv;
  const pdhcg_csr* R = nullptr;  // structured objective: Q + R^T R
};

// Memory sources a long-running caller (the serving loop) hands to creation so
// that it neither allocates nor frees synchronously: the arena comes from
// `pool` in stream order on the creation stream and is freed with
// cudaFreeAsync on that stream; the pinned staging buffer is reused (grown
// only when too small).
struct CreateAlloc {
  cudaMemPool_t pool = nullptr;
  void** pinned = nullptr;
  size_t* pinned_bytes = nullptr;
};

// Create count handles (shared allocation when count > 1).  In pdhcg_api.cu.
// pool_only: handles are solved by single CTAs only (no multi-CTA scratch).
int create_impl(int count, const CreateInput* in, const pdhcg_params* params, void* stream,
                pdhcg_problem** out, bool pool_only, const CreateAlloc* alloc = nullptr);
// Device bytes the handle of `in` would hold (host-side preparation only).
int footprint_of(const CreateInput& in, const pdhcg_params& prm, size_t* bytes);
SolverState initial_state(const pdhcg_problem* P);
void fill_result(const pdhcg_problem* P, const SolverState& S, pdhcg_result* res);
// One pooled launch advancing every handle by at most iter_budget PDHG steps
// (0 = no step limit) and, when slice_ns > 0, until about slice_ns of device
// time has passed (checked every 16 steps), with handle i's state at d_states[slots ? slots[i] : i]
// on the device and its solution written to x_out[i] / y_out[i] (device, may
// be null).  scratch (device, scratch_bytes) holds the launch descriptors when
// large enough; the caller then synchronises the stream before reusing it.
// Without it the call allocates a temporary buffer and blocks until done.
// Handles whose batch_nblk is above one run on multi-CTA groups: with
// group_stream given, in a cooperative launch of their own on that stream
// (ordered after the copies on the handles' stream by ev_ready, and before
// later work there by ev_done); without it, in one cooperative launch whose
// remaining CTAs serve the pool.  A large handle that finds no room sits this
// launch out when a step or time limit makes it a slice.
int launch_pool_slice(pdhcg_problem* const* probs, int count, SolverState* d_states,
                      double* const* x_out, double* const* y_out, int64_t iter_budget,
                      const int* slots = nullptr, void* scratch = nullptr, size_t scratch_bytes = 0,
                      uint64_t slice_ns = 0, cudaStream_t group_stream = nullptr,
                      cudaEvent_t ev_ready = nullptr, cudaEvent_t ev_done = nullptr);
// Bytes of device scratch one launch over count instances needs, ngroups of
// them on multi-CTA groups of group_ctas CTAs in total.
size_t batch_scratch_bytes(int count, int ngroups, int group_ctas);
int check_params_c(const pdhcg_params* p);

}  // namespace pdhcg

// Opaque handle of the C ABI.
struct pdhcg_problem {
  int device = 0;
  cudaStream_t stream = nullptr;
  pdhcg_params prm{};
  int precision = PDHCG_FP64;
  int method = PDHCG_INNER_DIAG;
  int32_t n = 0, m = 0;
  int32_t m_user = 0;  // rows the caller sees (m may add lifted bound rows)
  int32_t k = 0;       // rows of R in a structured objective Q = P + R^T R (0: none)
  int64_t nnzQ = 0, nnzA = 0, nnzR = 0;
  bool has_q = false;
  int lanes_var = 4, lanes_con = 4;
  // host copies kept for partitioning
  std::vector<int32_t> Qp, Ap, ATp;
  std::vector<int32_t> Rp;
  pdhcg::SellHost vsell, csell;  // integer SELL layouts (var space: AT [+ Q], con space: A)
  pdhcg::SellHost rsell;         // rows of R (structured objective)
  int32_t *r_perm = nullptr, *r_longs = nullptr, *r_huges = nullptr;
  int64_t* sRp = nullptr;
  int32_t* sRc = nullptr;
  void* sRv = nullptr;  // MatT
  size_t rsell_cols = 0;
  int32_t *Rp_d = nullptr, *Rc_d = nullptr;
  double* Rv_o = nullptr;
  void* Rs = nullptr;               // MatT, scaled R D
  // FP32 matrix values only: rounding remainders of the scaled values (float),
  // CSR order and SELL order (null in FP64 mode)
  float *Qs_lo = nullptr, *As_lo = nullptr, *ATs_lo = nullptr, *Rs_lo = nullptr;
  float *sQv_lo = nullptr, *sAv_lo = nullptr, *sATv_lo = nullptr, *sRv_lo = nullptr;
  void *rt1 = nullptr, *rt2 = nullptr;  // VecT, R v products (k each)
  // device SELL arrays
  int32_t *v_perm = nullptr, *v_longs = nullptr, *v_huges = nullptr;
  int32_t *c_perm = nullptr, *c_longs = nullptr, *c_huges = nullptr;
  int64_t *sATp = nullptr, *sQp = nullptr, *sAp = nullptr;
  int32_t *sATc = nullptr, *sQc = nullptr, *sAc = nullptr;
  void *sATv = nullptr, *sQv = nullptr, *sAv = nullptr;  // MatT
  size_t vsell_cols[2] = {0, 0}, csell_cols = 0;  // SELL element counts
  // device arena (possibly a slice of an allocation shared by a batch of handles)
  void* arena = nullptr;
  size_t arena_bytes = 0;
  size_t input_bytes = 0;              // uploaded prefix of the arena
  std::shared_ptr<void> arena_owner;  // frees the allocation with its last handle
  // typed device pointers (void* so the handle is precision-agnostic)
  int32_t *Qp_d = nullptr, *Qc_d = nullptr, *Ap_d = nullptr, *Ac_d = nullptr, *ATp_d = nullptr,
          *ATc_d = nullptr;
  double *Qv_o = nullptr, *Av_o = nullptr, *ATv_o = nullptr;
  void *Qs = nullptr, *As = nullptr, *ATs = nullptr;  // MatT
  double *c_o = nullptr, *lv_o = nullptr, *uv_o = nullptr, *lc_o = nullptr, *uc_o = nullptr;
  double *D = nullptr, *E = nullptr, *Dn = nullptr, *En = nullptr, *pv = nullptr, *pu = nullptr, *pw = nullptr,
         *pt = nullptr;
  void *c = nullptr, *lv = nullptr, *uv = nullptr, *lc = nullptr, *uc = nullptr, *qdiag = nullptr;
  int8_t *vtype = nullptr, *ctype = nullptr;
  void *xb0 = nullptr, *xb1 = nullptr, *yb0 = nullptr, *yb1 = nullptr, *xT = nullptr, *yT = nullptr,
       *xa = nullptr, *ya = nullptr, *r = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr,
       *bv = nullptr, *grad = nullptr, *gprev = nullptr, *xprev = nullptr, *xbar = nullptr;
  double *x_stage = nullptr, *y_stage = nullptr, *x_init_stage = nullptr, *y_init_stage = nullptr;
  pdhcg::SolverState* st = nullptr;
  // launch scratch: desc, plan arrays, barrier counter, partials
  void* inst_d = nullptr;  // one Inst<MatT, VecT>
  int32_t* plan_i32 = nullptr;           // g_first, g_nblk, g_inst, pool_inst, pool_next, err
  unsigned long long* bar = nullptr;
  int64_t* part_off = nullptr;
  double* part = nullptr;                // 2 * kSlots * max_blk
  int max_blk = 0;
  std::map<int, pdhcg::PartitionSet> partitions;
  // batched and served solves: CTAs of this instance's group (1 = a pool CTA),
  // and for batch_nblk > 1 its partition tables, uploaded with the inputs
  int batch_nblk = 1;
  int32_t* batch_part = nullptr;
  std::vector<int32_t> batch_tables;
  // pipeline form of pdhcg_solve (built at the first solve that uses it)
  int pipe_grid = 0;
  void* pipe_scratch = nullptr;        // PipeState, then kSlots * pipe_grid partial sums
  cudaGraphExec_t pipe_exec = nullptr;
  // setup results
  pdhcg::SolverState setup_state{};
  pdhcg::SolverState last_state{};  // state at the end of the last pdhcg_solve / _dev
};

// pdhcg_api.cu — the C ABI of include/pdhcg.h: create / solve / solve_batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>
#include <thread>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "host_problem.h"
#include "launch.h"
#include "setup_kernel.cuh"

namespace pdhcg {

const char* last_error_cstr();

template <class M, class V>
struct Prec {
  using Mat = M;
  using Vec = V;
};

template <class F>
int dispatch_precision(int precision, F&& f) {
  switch (precision) {
    case PDHCG_FP64: return f(Prec<double, double>{});
    case PDHCG_FP32: return f(Prec<float, float>{});
    case PDHCG_MIXED: return f(Prec<float, double>{});
    case PDHCG_DFLOAT: return f(Prec<float, dfloat>{});
    default: set_error("unknown precision"); return PDHCG_E_INVALID;
  }
}

int cuda_fail(cudaError_t e, const char* where) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? PDHCG_E_OOM : PDHCG_E_CUDA;
}

#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

size_t mat_bytes(int precision) { return precision == PDHCG_FP64 ? 8 : 4; }
size_t vec_bytes(int precision) { return precision == PDHCG_FP32 ? 4 : 8; }

// Carves 256-byte aligned buffers out of one allocation (first a sizing pass).
struct Carver {
  char* base = nullptr;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += std::max<size_t>(count, 1) * sizeof(T);
    return p;
  }
  void* take_bytes(size_t elems, size_t esize) {
    off = (off + 255) & ~size_t(255);
    void* p = base ? base + off : nullptr;
    off += std::max<size_t>(elems, 1) * esize;
    return p;
  }
};

// Device layout of one handle.  Everything uploaded from the host comes first
// (one contiguous prefix, copied with a single transfer); computed and work
// arrays follow.  With external_state the SolverState lives outside the arena.
void carve(pdhcg_problem* P, Carver& cv, bool external_state = false) {
  const size_t n = size_t(P->n), m = size_t(P->m), nq = size_t(P->nnzQ), na = size_t(P->nnzA);
  const size_t mb = mat_bytes(P->precision), vb = vec_bytes(P->precision);
  // ---- uploaded inputs ----
  P->Qp_d = cv.take<int32_t>(n + 1);
  P->Qc_d = cv.take<int32_t>(nq);
  P->Ap_d = cv.take<int32_t>(m + 1);
  P->Ac_d = cv.take<int32_t>(na);
  P->ATp_d = cv.take<int32_t>(n + 1);
  P->ATc_d = cv.take<int32_t>(na);
  P->Qv_o = cv.take<double>(nq);
  P->Av_o = cv.take<double>(na);
  P->ATv_o = cv.take<double>(na);
  P->c_o = cv.take<double>(n);
  P->lv_o = cv.take<double>(n);
  P->uv_o = cv.take<double>(n);
  P->lc_o = cv.take<double>(m);
  P->uc_o = cv.take<double>(m);
  P->vtype = cv.take<int8_t>(n);
  P->ctype = cv.take<int8_t>(m);
  P->v_perm = cv.take<int32_t>(P->vsell.perm.size());
  P->v_longs = cv.take<int32_t>(P->vsell.longs.size());
  P->v_huges = cv.take<int32_t>(P->vsell.huges.size());
  P->c_perm = cv.take<int32_t>(P->csell.perm.size());
  P->c_longs = cv.take<int32_t>(P->csell.longs.size());
  P->c_huges = cv.take<int32_t>(P->csell.huges.size());
  P->sATp = cv.take<int64_t>(P->vsell.ptr[0].size());
  P->sQp = cv.take<int64_t>(P->vsell.ptr[1].size());
  P->sAp = cv.take<int64_t>(P->csell.ptr[0].size());
  P->sATc = cv.take<int32_t>(P->vsell_cols[0] + 16);
  P->sQc = cv.take<int32_t>(P->vsell_cols[1] + 16);
  P->sAc = cv.take<int32_t>(P->csell_cols + 16);
  if (P->k > 0) {
    const size_t k = size_t(P->k), nr = size_t(P->nnzR);
    P->Rp_d = cv.take<int32_t>(k + 1);
    P->Rc_d = cv.take<int32_t>(nr);
    P->Rv_o = cv.take<double>(nr);
    P->r_perm = cv.take<int32_t>(P->rsell.perm.size());
    P->r_longs = cv.take<int32_t>(P->rsell.longs.size());
    P->r_huges = cv.take<int32_t>(P->rsell.huges.size());
    P->sRp = cv.take<int64_t>(P->rsell.ptr[0].size());
    P->sRc = cv.take<int32_t>(P->rsell_cols + 16);
  }
  if (P->batch_nblk > 1) P->batch_part = cv.take<int32_t>(11 * (size_t(P->batch_nblk) + 1));
  if (!external_state) P->st = cv.take<SolverState>(1);
  P->input_bytes = (cv.off + 255) & ~size_t(255);
  // ---- computed on the device ----
  P->Qs = cv.take_bytes(nq, mb);
  P->As = cv.take_bytes(na, mb);
  P->ATs = cv.take_bytes(na, mb);
  P->sATv = cv.take_bytes(P->vsell_cols[0] + 16, mb);
  P->sQv = cv.take_bytes(P->vsell_cols[1] + 16, mb);
  P->sAv = cv.take_bytes(P->csell_cols + 16, mb);
  if (P->k > 0) {
    P->Rs = cv.take_bytes(size_t(P->nnzR), mb);
    P->sRv = cv.take_bytes(P->rsell_cols + 16, mb);
    P->rt1 = cv.take_bytes(size_t(P->k), vb);
    P->rt2 = cv.take_bytes(size_t(P->k), vb);
  }
  if (mb == 4) {  // FP32 matrix values: their rounding remainders (FP64-accurate checks)
    P->Qs_lo = cv.take<float>(nq);
    P->As_lo = cv.take<float>(na);
    P->ATs_lo = cv.take<float>(na);
    P->sATv_lo = cv.take<float>(P->vsell_cols[0] + 16);
    P->sQv_lo = cv.take<float>(P->vsell_cols[1] + 16);
    P->sAv_lo = cv.take<float>(P->csell_cols + 16);
    if (P->k > 0) {
      P->Rs_lo = cv.take<float>(size_t(P->nnzR));
      P->sRv_lo = cv.take<float>(P->rsell_cols + 16);
    }
  }
  P->D = cv.take<double>(n);
  P->E = cv.take<double>(m);
  P->Dn = cv.take<double>(n);
  P->En = cv.take<double>(m);
  P->pv = cv.take<double>(n);
  P->pu = cv.take<double>(n);
  P->pw = cv.take<double>(n);
  P->pt = cv.take<double>(m);
  P->c = cv.take_bytes(n, vb);
  P->lv = cv.take_bytes(n, vb);
  P->uv = cv.take_bytes(n, vb);
  P->qdiag = cv.take_bytes(n, vb);
  P->lc = cv.take_bytes(m, vb);
  P->uc = cv.take_bytes(m, vb);
  void** nvecs[] = {&P->xb0, &P->xb1, &P->xT, &P->xa, &P->r, &P->p0, &P->p1, &P->q,
                    &P->bv, &P->grad, &P->gprev, &P->xprev, &P->xbar};
  for (void** pp : nvecs) *pp = cv.take_bytes(n, vb);
  void** mvecs[] = {&P->yb0, &P->yb1, &P->yT, &P->ya};
  for (void** pp : mvecs) *pp = cv.take_bytes(m, vb);
  P->x_stage = cv.take<double>(n);
  P->y_stage = cv.take<double>(m);
  P->x_init_stage = cv.take<double>(n);
  P->y_init_stage = cv.take<double>(m);
  P->inst_d = cv.take_bytes(1, sizeof(Inst<double, double>));
  P->plan_i32 = cv.take<int32_t>(16);
  P->bar = static_cast<unsigned long long*>(cv.take_bytes(kBarBytes, 1));
  P->part_off = cv.take<int64_t>(1);
  P->part = cv.take<double>(size_t(2) * kSlots * size_t(std::max(P->max_blk, 1)));
}

// Copy the uploaded inputs of P into a host staging image of its arena prefix.
void pack_inputs(const pdhcg_problem* P, const HostQP& h, char* stage) {
  const char* base = static_cast<const char*>(P->arena);
  auto put = [&](const void* dst, const void* src, size_t bytes) {
    if (bytes) std::memcpy(stage + (static_cast<const char*>(dst) - base), src, bytes);
  };
  const size_t n = size_t(h.n), m = size_t(h.m);
  put(P->Qp_d, h.Qp.data(), sizeof(int32_t) * (n + 1));
  put(P->Qc_d, h.Qc.data(), sizeof(int32_t) * h.Qc.size());
  put(P->Ap_d, h.Ap.data(), sizeof(int32_t) * (m + 1));
  put(P->Ac_d, h.Ac.data(), sizeof(int32_t) * h.Ac.size());
  put(P->ATp_d, h.ATp.data(), sizeof(int32_t) * (n + 1));
  put(P->ATc_d, h.ATc.data(), sizeof(int32_t) * h.ATc.size());
  put(P->Qv_o, h.Qv.data(), sizeof(double) * h.Qv.size());
  put(P->Av_o, h.Av.data(), sizeof(double) * h.Av.size());
  put(P->ATv_o, h.ATv.data(), sizeof(double) * h.ATv.size());
  put(P->c_o, h.c.data(), sizeof(double) * n);
  put(P->lv_o, h.lv.data(), sizeof(double) * n);
  put(P->uv_o, h.uv.data(), sizeof(double) * n);
  put(P->lc_o, h.lc.data(), sizeof(double) * m);
  put(P->uc_o, h.uc.data(), sizeof(double) * m);
  put(P->vtype, h.vtype.data(), n);
  put(P->ctype, h.ctype.data(), m);
  put(P->v_perm, P->vsell.perm.data(), sizeof(int32_t) * P->vsell.perm.size());
  put(P->v_longs, P->vsell.longs.data(), sizeof(int32_t) * P->vsell.longs.size());
  put(P->v_huges, P->vsell.huges.data(), sizeof(int32_t) * P->vsell.huges.size());
  put(P->c_perm, P->csell.perm.data(), sizeof(int32_t) * P->csell.perm.size());
  put(P->c_longs, P->csell.longs.data(), sizeof(int32_t) * P->csell.longs.size());
  put(P->c_huges, P->csell.huges.data(), sizeof(int32_t) * P->csell.huges.size());
  put(P->sATp, P->vsell.ptr[0].data(), sizeof(int64_t) * P->vsell.ptr[0].size());
  put(P->sQp, P->vsell.ptr[1].data(), sizeof(int64_t) * P->vsell.ptr[1].size());
  put(P->sAp, P->csell.ptr[0].data(), sizeof(int64_t) * P->csell.ptr[0].size());
  put(P->sATc, P->vsell.col[0].data(), sizeof(int32_t) * P->vsell.col[0].size());
  put(P->sQc, P->vsell.col[1].data(), sizeof(int32_t) * P->vsell.col[1].size());
  put(P->sAc, P->csell.col[0].data(), sizeof(int32_t) * P->csell.col[0].size());
  if (P->k > 0) {
    put(P->Rp_d, h.Rp.data(), sizeof(int32_t) * h.Rp.size());
    put(P->Rc_d, h.Rc.data(), sizeof(int32_t) * h.Rc.size());
    put(P->Rv_o, h.Rv.data(), sizeof(double) * h.Rv.size());
    put(P->r_perm, P->rsell.perm.data(), sizeof(int32_t) * P->rsell.perm.size());
    put(P->r_longs, P->rsell.longs.data(), sizeof(int32_t) * P->rsell.longs.size());
    put(P->r_huges, P->rsell.huges.data(), sizeof(int32_t) * P->rsell.huges.size());
    put(P->sRp, P->rsell.ptr[0].data(), sizeof(int64_t) * P->rsell.ptr[0].size());
    put(P->sRc, P->rsell.col[0].data(), sizeof(int32_t) * P->rsell.col[0].size());
  }
  if (P->batch_nblk > 1) put(P->batch_part, P->batch_tables.data(), sizeof(int32_t) * P->batch_tables.size());
  if (static_cast<const char*>(static_cast<const void*>(P->st)) >= base &&
      static_cast<const char*>(static_cast<const void*>(P->st)) < base + P->input_bytes) {
    SolverState S{};
    S.method = P->method;
    put(P->st, &S, sizeof(S));
  }
}

int lanes_for(double avg) {
  int L = 2;
  while (L < 32 && L * 2 <= avg) L *= 2;
  return L;
}

// nnz-balanced row partition into nblk ranges; rows of length >= long_thr get a range alone.
std::vector<int32_t> partition_rows(const std::vector<int64_t>& len, int nblk, int64_t long_thr) {
  const int32_t R = int32_t(len.size());
  int64_t total = 0;
  for (int64_t l : len) total += l + 2;
  double target = std::max(1.0, std::ceil(double(total) / nblk));
  std::vector<int32_t> b;
  for (int attempt = 0; attempt < 200; ++attempt) {
    b.assign(1, 0);
    int64_t acc = 0;
    for (int32_t r = 0; r < R; ++r) {
      if (len[r] >= long_thr) {
        if (b.back() < r) b.push_back(r);
        b.push_back(r + 1);
        acc = 0;
        continue;
      }
      acc += len[r] + 2;
      if (double(acc) >= target) {
        b.push_back(r + 1);
        acc = 0;
      }
    }
    if (b.back() < R) b.push_back(R);
    if (int(b.size()) - 1 <= nblk) break;
    target *= 1.1;
  }
  while (int(b.size()) - 1 < nblk) b.push_back(R);
  return b;
}

// Elementwise phases split [0, n) and [0, m) evenly over the CTAs of a group.
std::vector<int32_t> even_split(int32_t rows, int nblk) {
  std::vector<int32_t> b(size_t(nblk) + 1);
  for (int k = 0; k <= nblk; ++k) b[size_t(k)] = int32_t((int64_t(rows) * k) / nblk);
  return b;
}

// The 11 row-partition tables of a group of nblk CTAs (nblk + 1 entries each):
// SELL slices / long rows / huge rows of the variable space, the same for the
// constraint space, even element splits of both, and the three tables of the
// rows of R.  Host work only.
std::vector<int32_t> partition_tables(const pdhcg_problem* P, int nblk) {
  auto slice_w = [](const SellHost& sh, int nmat) {
    std::vector<int64_t> w(size_t(sh.nslices), 0);
    for (int k = 0; k < nmat; ++k)
      for (int32_t s = 0; s < sh.nslices; ++s) w[size_t(s)] += sh.ptr[k][size_t(s) + 1] - sh.ptr[k][size_t(s)] + 8;
    return w;
  };
  auto row_w = [](const std::vector<int32_t>& rows, const std::vector<int32_t>* rp0,
                  const std::vector<int32_t>* rp1) {
    std::vector<int64_t> w(rows.size(), 0);
    for (size_t i = 0; i < rows.size(); ++i) {
      const int32_t r = rows[i];
      w[i] = (*rp0)[size_t(r) + 1] - (*rp0)[size_t(r)] + (rp1 && !rp1->empty() ? (*rp1)[size_t(r) + 1] - (*rp1)[size_t(r)] : 0) + 8;
    }
    return w;
  };
  const std::vector<int32_t>* qrp = P->has_q ? &P->Qp : nullptr;
  std::vector<int32_t> tabs[6] = {
      split_balanced(slice_w(P->vsell, P->has_q ? 2 : 1), nblk),
      split_balanced(row_w(P->vsell.longs, &P->ATp, qrp), nblk),
      split_balanced(row_w(P->vsell.huges, &P->ATp, qrp), nblk),
      split_balanced(slice_w(P->csell, 1), nblk),
      split_balanced(row_w(P->csell.longs, &P->Ap, nullptr), nblk),
      split_balanced(row_w(P->csell.huges, &P->Ap, nullptr), nblk)};
  std::vector<int32_t> ev = even_split(P->n, nblk), ec = even_split(P->m, nblk);
  // huge rows go to the last CTAs (their slice share is balanced separately)
  for (int t : {2, 5}) {
    std::vector<int32_t>& b = tabs[t];
    const int32_t nh = b.back();
    for (int k = 0; k <= nblk; ++k) b[size_t(k)] = std::max(0, std::min(nh, k - (nblk - nh)));
  }
  // rows of R (structured objective): slices, long and huge rows like the other spaces
  std::vector<int32_t> rt[3];
  if (P->k > 0) {
    rt[0] = split_balanced(slice_w(P->rsell, 1), nblk);
    rt[1] = split_balanced(row_w(P->rsell.longs, &P->Rp, nullptr), nblk);
    rt[2] = split_balanced(row_w(P->rsell.huges, &P->Rp, nullptr), nblk);
    const int32_t nh = rt[2].back();
    for (int k = 0; k <= nblk; ++k) rt[2][size_t(k)] = std::max(0, std::min(nh, k - (nblk - nh)));
  } else {
    for (auto& t : rt) t.assign(size_t(nblk) + 1, 0);
  }
  std::vector<int32_t> flat;
  flat.reserve(11 * (size_t(nblk) + 1));
  for (auto& t : tabs) flat.insert(flat.end(), t.begin(), t.end());
  flat.insert(flat.end(), ev.begin(), ev.end());
  flat.insert(flat.end(), ec.begin(), ec.end());
  for (auto& t : rt) flat.insert(flat.end(), t.begin(), t.end());
  return flat;
}

// The device tables of a PartitionSet at d (11 * (nblk + 1) int32).
void bind_partition(PartitionSet& ps, int32_t* d, int nblk) {
  const size_t per = size_t(nblk) + 1;
  ps.nblk = nblk;
  ps.d_buf = d;
  ps.v_slice = d;
  ps.v_long = d + per;
  ps.v_huge = d + 2 * per;
  ps.c_slice = d + 3 * per;
  ps.c_long = d + 4 * per;
  ps.c_huge = d + 5 * per;
  ps.v_even = d + 6 * per;
  ps.c_even = d + 7 * per;
  ps.r_slice = d + 8 * per;
  ps.r_long = d + 9 * per;
  ps.r_huge = d + 10 * per;
}

int get_partition(pdhcg_problem* P, int nblk, PartitionSet** out) {
  auto it = P->partitions.find(nblk);
  if (it != P->partitions.end()) {
    *out = &it->second;
    return PDHCG_OK;
  }
  const std::vector<int32_t> flat = partition_tables(P, nblk);
  int32_t* d = nullptr;
  CK(cudaMalloc(&d, sizeof(int32_t) * flat.size()));
  const cudaError_t e = cudaMemcpy(d, flat.data(), sizeof(int32_t) * flat.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_fail(e, "partition tables");
  }
  PartitionSet ps;
  bind_partition(ps, d, nblk);
  ps.owned = true;
  auto res = P->partitions.emplace(nblk, ps);
  *out = &res.first->second;
  return PDHCG_OK;
}

DevParams dev_params(const pdhcg_params& p) {
  DevParams d;
  d.eps_tol = p.eps_tol;
  d.eps_inf = p.eps_inf;
  d.time_limit_ns = p.time_limit_s * 1e9;
  d.max_iter = p.max_iter;
  d.theta = p.theta;
  d.kp = p.kp;
  d.ki = p.ki;
  d.kd = p.kd;
  d.gamma_inner = p.gamma_inner;
  d.eps_inner_min = p.eps_inner_min;
  d.eps_inner_first = p.eps_inner_first;
  d.restart_sufficient = p.restart_sufficient;
  d.restart_necessary = p.restart_necessary;
  d.restart_artificial = p.restart_artificial;
  d.omega_clamp = p.omega_clamp;
  d.k_eval = p.k_eval;
  d.max_inner_iter = p.max_inner_iter;
  return d;
}

template <class MatT, class VecT>
Inst<MatT, VecT> make_inst(const pdhcg_problem* P) {
  Inst<MatT, VecT> I;
  I.n = P->n;
  I.m = P->m;
  I.has_q = P->has_q ? 1 : 0;
  I.lanes_var = P->lanes_var;
  I.lanes_con = P->lanes_con;
  I.Q = Csr<MatT>{P->n, int32_t(P->nnzQ), P->Qp_d, P->Qc_d, static_cast<const MatT*>(P->Qs), P->Qs_lo};
  I.A = Csr<MatT>{P->m, int32_t(P->nnzA), P->Ap_d, P->Ac_d, static_cast<const MatT*>(P->As), P->As_lo};
  I.AT = Csr<MatT>{P->n, int32_t(P->nnzA), P->ATp_d, P->ATc_d, static_cast<const MatT*>(P->ATs), P->ATs_lo};
  I.ATs = Sell<MatT>{P->sATp, P->sATc, static_cast<const MatT*>(P->sATv), P->sATv_lo};
  I.Qs = Sell<MatT>{P->sQp, P->sQc, static_cast<const MatT*>(P->sQv), P->sQv_lo};
  I.As = Sell<MatT>{P->sAp, P->sAc, static_cast<const MatT*>(P->sAv), P->sAv_lo};
  I.vsp.nslices = P->vsell.nslices;
  I.vsp.nlong = int32_t(P->vsell.longs.size());
  I.vsp.nhuge = int32_t(P->vsell.huges.size());
  I.vsp.perm = P->v_perm;
  I.vsp.longs = P->v_longs;
  I.vsp.huges = P->v_huges;
  I.csp.nslices = P->csell.nslices;
  I.csp.nlong = int32_t(P->csell.longs.size());
  I.csp.nhuge = int32_t(P->csell.huges.size());
  I.csp.perm = P->c_perm;
  I.csp.longs = P->c_longs;
  I.csp.huges = P->c_huges;
  I.c = static_cast<VecT*>(P->c);
  I.lv = static_cast<const VecT*>(P->lv);
  I.uv = static_cast<const VecT*>(P->uv);
  I.lc = static_cast<VecT*>(P->lc);
  I.uc = static_cast<VecT*>(P->uc);
  I.qdiag = static_cast<const VecT*>(P->qdiag);
  I.vtype = P->vtype;
  I.ctype = P->ctype;
  I.D = P->D;
  I.E = P->E;
  I.c_o = P->c_o;
  I.lv_o = P->lv_o;
  I.uv_o = P->uv_o;
  I.lc_o = P->lc_o;
  I.uc_o = P->uc_o;
  I.bscale = P->setup_state.bscale;
  I.cinf = P->setup_state.cinf;
  I.xb0 = static_cast<VecT*>(P->xb0);
  I.xb1 = static_cast<VecT*>(P->xb1);
  I.yb0 = static_cast<VecT*>(P->yb0);
  I.yb1 = static_cast<VecT*>(P->yb1);
  I.xT = static_cast<VecT*>(P->xT);
  I.yT = static_cast<VecT*>(P->yT);
  I.xa = static_cast<VecT*>(P->xa);
  I.ya = static_cast<VecT*>(P->ya);
  I.r = static_cast<VecT*>(P->r);
  I.p0 = static_cast<VecT*>(P->p0);
  I.p1 = static_cast<VecT*>(P->p1);
  I.q = static_cast<VecT*>(P->q);
  I.bv = static_cast<VecT*>(P->bv);
  I.grad = static_cast<VecT*>(P->grad);
  I.gprev = static_cast<VecT*>(P->gprev);
  I.xprev = static_cast<VecT*>(P->xprev);
  I.xbar = static_cast<VecT*>(P->xbar);
  I.st = P->st;
  I.prm = dev_params(P->prm);
  if (P->k > 0) {
    I.k = P->k;
    I.R = Csr<MatT>{P->k, int32_t(P->nnzR), P->Rp_d, P->Rc_d, static_cast<const MatT*>(P->Rs), P->Rs_lo};
    I.Rsl = Sell<MatT>{P->sRp, P->sRc, static_cast<const MatT*>(P->sRv), P->sRv_lo};
    I.rsp.nslices = P->rsell.nslices;
    I.rsp.nlong = int32_t(P->rsell.longs.size());
    I.rsp.nhuge = int32_t(P->rsell.huges.size());
    I.rsp.perm = P->r_perm;
    I.rsp.longs = P->r_longs;
    I.rsp.huges = P->r_huges;
    I.rt1 = static_cast<VecT*>(P->rt1);
    I.rt2 = static_cast<VecT*>(P->rt2);
  }
  return I;
}

template <class MatT, class VecT>
void set_partition(Inst<MatT, VecT>& I, const PartitionSet& ps, const pdhcg_problem* P) {
  I.vsp.slice_part = ps.v_slice;
  I.vsp.long_part = ps.v_long;
  I.vsp.huge_part = ps.v_huge;
  I.csp.slice_part = ps.c_slice;
  I.csp.long_part = ps.c_long;
  I.csp.huge_part = ps.c_huge;
  I.var_part = ps.v_even;
  I.con_part = ps.c_even;
  I.rsp.slice_part = ps.r_slice;
  I.rsp.long_part = ps.r_long;
  I.rsp.huge_part = ps.r_huge;
  I.part_blocks = ps.nblk;
  (void)P;
}

SolverState initial_state(const pdhcg_problem* P) {
  SolverState S = P->setup_state;
  S.K = 0;
  S.k = 0;
  S.inner_total = 0;
  S.restarts = 0;
  S.omega = S.omega0;
  S.log_omega = std::log(S.omega0);
  S.log_omega0 = S.log_omega;
  S.e_sum = 0.0;
  S.e_prev = 0.0;
  S.tau = S.eta / S.omega;
  S.sigma = S.eta * S.omega;
  S.eps_in = INFINITY;
  S.mv = 0.0;
  S.fpr_anchor = 0.0;
  S.fpr_last = 0.0;
  S.r_primal = S.r_dual = S.r_gap = S.pobj = S.dobj = 0.0;
  S.t_start_ns = S.t_end_ns = 0.0;
  S.status = 0;
  S.cur = 0;
  S.started = 0;
  S.method = P->method;
  S.device_error = 0;
  for (double& t : S.tm) t = 0.0;
  return S;
}

void fill_result(const pdhcg_problem* P, const SolverState& S, pdhcg_result* res) {
  std::memset(res, 0, sizeof(*res));
  res->status = S.status;
  res->inner_method = S.method;
  res->iterations = S.K;
  res->inner_iterations = S.inner_total;
  res->restarts = S.restarts;
  res->r_primal = S.r_primal;
  res->r_dual = S.r_dual;
  res->r_gap = S.r_gap;
  res->primal_obj = S.pobj;
  res->dual_obj = S.dobj;
  res->eta = S.eta;
  res->omega = S.omega;
  res->norm_A = S.norm_A;
  res->solve_seconds = (S.t_end_ns - S.t_start_ns) * 1e-9;
  res->power_iters = S.power_iters;
  res->precision = P->precision;
  res->form = S.form;
}

// CTAs of one cooperative group: the solve kernel's co-residency, or (setup)
// the setup kernel's, which may be lower.
int max_group_blocks(int precision, bool setup) {
  KernelLimits kl{};
  int rc = dispatch_precision(precision, [&](auto tag) {
    using M = typename decltype(tag)::Mat;
    using V = typename decltype(tag)::Vec;
    cudaError_t e = kernel_limits<M, V>(&kl);
    return e == cudaSuccess ? PDHCG_OK : cuda_fail(e, "kernel_limits");
  });
  if (rc) return rc;
  return setup ? std::min(kl.max_coresident_group, kl.max_coresident_setup) : kl.max_coresident_group;
}

int cached_max_group_blocks(int precision, bool setup = false) {
  static std::mutex mu;
  static int cache[2][4][64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  int* slot = (dev >= 0 && dev < 64) ? &cache[setup ? 1 : 0][precision][dev] : nullptr;
  if (slot && *slot > 0) return *slot;
  const int mb = max_group_blocks(precision, setup);
  if (mb > 0 && slot) *slot = mb;
  return mb;
}

// Largest per-instance vector footprint a pool CTA keeps in shared memory.
#ifndef PDHCG_SMEM_VEC_BUDGET_KB
#define PDHCG_SMEM_VEC_BUDGET_KB 110
#endif
constexpr size_t kSmemVecBudget = size_t(PDHCG_SMEM_VEC_BUDGET_KB) * 1024;


size_t smem_need(const pdhcg_problem* P) {
  return smem_vector_bytes(P->n, P->m, P->method, vec_bytes(P->precision));
}

// Threads of the pool CTA that solves P alone, batched or served.
int pool_width(const pdhcg_problem* P) { return P->prm.pool_threads == 128 ? kPoolBS : kGroupBS; }

int choose_group_blocks(const pdhcg_problem* P, int maxblk) {
  if (P->prm.group_blocks > 0) return std::min(P->prm.group_blocks, maxblk);
  const int64_t work = (P->method != PDHCG_INNER_DIAG ? P->nnzQ + P->nnzR : 0) + 2 * P->nnzA + P->n + P->m;
  if (work < 150000) return 1;
  return int(std::max<int64_t>(2, std::min<int64_t>(maxblk, work / 8192)));
}

// Batched and served solves: instances below kGroupWork (nonzeros and vector
// entries one PDHG step touches, inner products counted once) run on one pool
// CTA each; larger ones on a multi-CTA group of about one CTA per
// kWorkPerGroupCta, at most kMaxBatchGroup.
#ifndef PDHCG_WORK_PER_GROUP_CTA
#define PDHCG_WORK_PER_GROUP_CTA 65536
#endif
constexpr int64_t kWorkPerGroupCta = PDHCG_WORK_PER_GROUP_CTA;
#ifndef PDHCG_MAX_BATCH_GROUP
#define PDHCG_MAX_BATCH_GROUP 32
#endif
constexpr int kMaxBatchGroup = PDHCG_MAX_BATCH_GROUP;

int batch_group_blocks(const pdhcg_problem* P) {
  const int64_t work = (P->method != PDHCG_INNER_DIAG ? P->nnzQ + P->nnzR : 0) + 2 * P->nnzA + P->n + P->m;
  if (work < kGroupWork) return 1;
  return int(std::max<int64_t>(2, std::min<int64_t>(kMaxBatchGroup, work / kWorkPerGroupCta)));
}

// Pooled handles: the group size for batched launches and its partition tables
// (uploaded with the inputs, so no launch has to allocate them).
void set_batch_grouping(pdhcg_problem* P) {
  P->batch_nblk = batch_group_blocks(P);
  if (P->batch_nblk > 1) P->batch_tables = partition_tables(P, P->batch_nblk);
}

template <class M, class V>
SetupArgs<M, V> make_setup_args(const pdhcg_problem* P, const PartitionSet* ps) {
  SetupArgs<M, V> a{};
  a.n = P->n;
  a.m = P->m;
  a.has_q = P->has_q ? 1 : 0;
  a.ruiz_iters = P->prm.ruiz_iters;
  a.power_max_iter = P->prm.power_max_iter;
  a.lanes_var = P->lanes_var;
  a.lanes_con = P->lanes_con;
  a.power_tol = P->prm.power_tol;
  a.eta_override = P->prm.eta_override;
  a.omega0_override = P->prm.omega0_override;
  a.Qp = P->Qp_d;
  a.Qc = P->Qc_d;
  a.Ap = P->Ap_d;
  a.Ac = P->Ac_d;
  a.ATp = P->ATp_d;
  a.ATc = P->ATc_d;
  a.Qv_o = P->Qv_o;
  a.Av_o = P->Av_o;
  a.ATv_o = P->ATv_o;
  a.c_o = P->c_o;
  a.lv_o = P->lv_o;
  a.uv_o = P->uv_o;
  a.lc_o = P->lc_o;
  a.uc_o = P->uc_o;
  a.var_part = ps ? ps->v_even : nullptr;
  a.con_part = ps ? ps->c_even : nullptr;
  a.D = P->D;
  a.E = P->E;
  a.Dn = P->Dn;
  a.En = P->En;
  a.pv = P->pv;
  a.pu = P->pu;
  a.pw = P->pw;
  a.pt = P->pt;
  a.Qs = static_cast<M*>(P->Qs);
  a.As = static_cast<M*>(P->As);
  a.ATs = static_cast<M*>(P->ATs);
  a.c = static_cast<V*>(P->c);
  a.lv = static_cast<V*>(P->lv);
  a.uv = static_cast<V*>(P->uv);
  a.lc = static_cast<V*>(P->lc);
  a.uc = static_cast<V*>(P->uc);
  a.qdiag = static_cast<V*>(P->qdiag);
  a.st = P->st;
  a.vsp.nslices = P->vsell.nslices;
  a.vsp.nlong = int32_t(P->vsell.longs.size());
  a.vsp.nhuge = int32_t(P->vsell.huges.size());
  a.vsp.perm = P->v_perm;
  a.vsp.longs = P->v_longs;
  a.vsp.huges = P->v_huges;
  a.csp.nslices = P->csell.nslices;
  a.csp.nlong = int32_t(P->csell.longs.size());
  a.csp.nhuge = int32_t(P->csell.huges.size());
  a.csp.perm = P->c_perm;
  a.csp.longs = P->c_longs;
  a.csp.huges = P->c_huges;
  if (ps) {
    a.vsp.slice_part = ps->v_slice;
    a.vsp.long_part = ps->v_long;
    a.vsp.huge_part = ps->v_huge;
    a.csp.slice_part = ps->c_slice;
    a.csp.long_part = ps->c_long;
    a.csp.huge_part = ps->c_huge;
  }
  a.sATp = P->sATp;
  a.sQp = P->sQp;
  a.sAp = P->sAp;
  a.sATc = P->sATc;
  a.sQc = P->sQc;
  a.sAc = P->sAc;
  a.sATv = static_cast<M*>(P->sATv);
  a.sQv = static_cast<M*>(P->sQv);
  a.sAv = static_cast<M*>(P->sAv);
  a.Qs_lo = P->Qs_lo;
  a.As_lo = P->As_lo;
  a.ATs_lo = P->ATs_lo;
  a.sATv_lo = P->sATv_lo;
  a.sQv_lo = P->sQv_lo;
  a.sAv_lo = P->sAv_lo;
  a.Rs_lo = P->Rs_lo;
  a.sRv_lo = P->sRv_lo;
  if (P->k > 0) {
    a.k = P->k;
    a.Rp = P->Rp_d;
    a.Rc = P->Rc_d;
    a.Rv_o = P->Rv_o;
    a.Rs = static_cast<M*>(P->Rs);
    a.rsp.nslices = P->rsell.nslices;
    a.rsp.perm = P->r_perm;
    a.sRp = P->sRp;
    a.sRv = static_cast<M*>(P->sRv);
  }
  return a;
}

int run_setup(pdhcg_problem* P) {
  const int lim = cached_max_group_blocks(P->precision, true);
  if (lim < 0) return lim;
  const int nblk = choose_group_blocks(P, std::max(1, std::min(P->max_blk, lim)));
  PartitionSet* ps = nullptr;
  if (nblk > 1) {
    int rc = get_partition(P, nblk, &ps);
    if (rc) return rc;
  }
  CK(cudaMemsetAsync(P->bar, 0, kBarBytes, P->stream));
  CK(cudaMemsetAsync(P->plan_i32, 0, sizeof(int32_t) * 16, P->stream));
  return dispatch_precision(P->precision, [&](auto tag) {
    using M = typename decltype(tag)::Mat;
    using V = typename decltype(tag)::Vec;
    SetupArgs<M, V> a = make_setup_args<M, V>(P, ps);
    const uint64_t tmo = uint64_t(std::max(P->prm.device_timeout_ms, 1)) * 1000000ull;
    cudaError_t e = launch_setup<M, V>(a, nblk, P->bar, P->part, P->plan_i32 + 5, tmo, P->stream);
    if (e != cudaSuccess) return cuda_fail(e, "setup launch");
    CK(cudaMemcpyAsync(&P->setup_state, P->st, sizeof(SolverState), cudaMemcpyDeviceToHost, P->stream));
    int32_t err = 0;
    CK(cudaMemcpyAsync(&err, P->plan_i32 + 5, sizeof(int32_t), cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    if (err) {
      set_error("setup: a bounded device wait gave up");
      return PDHCG_E_DEVICE_TIMEOUT;
    }
    return PDHCG_OK;
  });
}


// Problems at least this large (the work measure of choose_group_blocks) run
// pdhcg_solve in the pipeline form when params.pipeline is 0.
constexpr int64_t kPipelineWork = int64_t(1) << 21;

bool use_pipeline(const pdhcg_problem* P) {
  if (P->prm.pipeline < 0 || P->k > 0 || P->max_blk <= 1) return false;
  if (P->prm.pipeline > 0) return true;
  const int64_t work = (P->method != PDHCG_INNER_DIAG ? P->nnzQ : 0) + 2 * P->nnzA + P->n + P->m;
  return work >= kPipelineWork;
}

// One solve in the pipeline form: descriptor and initial state up, one graph
// launch, state back.  The graph is built at the first call.
int solve_pipeline(pdhcg_problem* P, const double* x0_d, const double* y0_d, pdhcg_result* res,
                   double* x_out_d, double* y_out_d) {
  return dispatch_precision(P->precision, [&](auto tag) -> int {
    using M = typename decltype(tag)::Mat;
    using V = typename decltype(tag)::Vec;
    if (!P->pipe_exec) {
      int sms = 0;
      CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device));
      const int per_sm = pipeline_blocks_per_sm<M, V>();
      if (per_sm < 1) {
        set_error("pipeline: its kernels cannot be resident");
        return PDHCG_E_CUDA;
      }
      const int grid = per_sm * sms;
      if (!P->pipe_scratch) CK(cudaMalloc(&P->pipe_scratch, kPipeStateBytes + sizeof(double) * kSlots * size_t(grid)));
      PartitionSet* ps = nullptr;
      int rc = get_partition(P, grid, &ps);
      if (rc) return rc;
      double* part = reinterpret_cast<double*>(static_cast<char*>(P->pipe_scratch) + kPipeStateBytes);
      cudaGraphExec_t ex = nullptr;
      const cudaError_t e = pipeline_build<M, V>(static_cast<const Inst<M, V>*>(P->inst_d), grid, P->method,
                                                 P->pipe_scratch, part, &ex);
      if (e != cudaSuccess) return cuda_fail(e, "pipeline graph");
      P->pipe_exec = ex;
      P->pipe_grid = grid;
    }
    PartitionSet* ps = nullptr;
    int rc = get_partition(P, P->pipe_grid, &ps);
    if (rc) return rc;
    SolverState S = initial_state(P);
    CK(cudaMemcpyAsync(P->st, &S, sizeof(S), cudaMemcpyHostToDevice, P->stream));
    Inst<M, V> I = make_inst<M, V>(P);
    I.x_init = x0_d;
    I.y_init = y0_d;
    I.x_out = x_out_d;
    I.y_out = y_out_d;
    set_partition(I, *ps, P);
    CK(cudaMemcpyAsync(P->inst_d, &I, sizeof(I), cudaMemcpyHostToDevice, P->stream));
    CK(cudaMemsetAsync(P->pipe_scratch, 0, kPipeStateBytes, P->stream));
    CK(cudaGraphLaunch(P->pipe_exec, P->stream));
    CK(cudaMemcpyAsync(&S, P->st, sizeof(S), cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
#if PDHCG_PIPE_TIMERS
    {  // the kernels' device times into the phase-time categories
      PipeClockView v{};
      CK(cudaMemcpy(&v, P->pipe_scratch, sizeof(v), cudaMemcpyDeviceToHost));
      const int cat[12] = {7, 0, 1, 2, 2, 1, 6, 3, 4, 6, 6, 6};
      for (double& t : S.tm) t = 0.0;
      for (int k = 0; k < 12; ++k) S.tm[cat[k]] += double(v.ns_busy[k]);
      S.tm[5] += double(v.ns_gap);
    }
#endif
    if (res) fill_result(P, S, res);
    P->last_state = S;
    return PDHCG_OK;
  });
}

// One solve of one handle (device pointers for warm start / outputs).
int solve_one(pdhcg_problem* P, const double* x0_d, const double* y0_d, pdhcg_result* res,
              double* x_out_d, double* y_out_d) {
  CK(cudaSetDevice(P->device));
  if (use_pipeline(P)) {
    const int rc = solve_pipeline(P, x0_d, y0_d, res, x_out_d, y_out_d);
    if (rc == PDHCG_OK || P->prm.pipeline > 0) return rc;
    // automatic choice: the persistent kernel when the graph is unavailable
    P->prm.pipeline = -1;
  }
  const int nblk = choose_group_blocks(P, P->max_blk);
  PartitionSet* ps = nullptr;
  if (nblk > 1) {
    int rc = get_partition(P, nblk, &ps);
    if (rc) return rc;
  }
  SolverState S = initial_state(P);
  CK(cudaMemcpyAsync(P->st, &S, sizeof(S), cudaMemcpyHostToDevice, P->stream));
  int rc = dispatch_precision(P->precision, [&](auto tag) {
    using M = typename decltype(tag)::Mat;
    using V = typename decltype(tag)::Vec;
    Inst<M, V> I = make_inst<M, V>(P);
    I.x_init = x0_d;
    I.y_init = y0_d;
    I.x_out = x_out_d;
    I.y_out = y_out_d;
    if (ps) set_partition(I, *ps, P);
    CK(cudaMemcpyAsync(P->inst_d, &I, sizeof(I), cudaMemcpyHostToDevice, P->stream));
    // plan_i32: [0] g_first [1] g_nblk [2] g_inst [3] pool_inst [4] pool_next [5] err
    int32_t hp[16] = {0, nblk, 0, 0, 0, 0};
    CK(cudaMemcpyAsync(P->plan_i32, hp, sizeof(hp), cudaMemcpyHostToDevice, P->stream));
    CK(cudaMemsetAsync(P->bar, 0, kBarBytes, P->stream));
    int64_t zero = 0;
    CK(cudaMemcpyAsync(P->part_off, &zero, sizeof(zero), cudaMemcpyHostToDevice, P->stream));
    LaunchPlan plan;
    plan.structured = P->k > 0;
    plan.err = P->plan_i32 + 5;
    plan.timeout_ns = uint64_t(std::max(P->prm.device_timeout_ms, 1)) * 1000000ull;
    int grid = 1;
    if (nblk > 1) {
      plan.ngroups = 1;
      plan.group_blocks = nblk;
      plan.g_first = P->plan_i32 + 0;
      plan.g_nblk = P->plan_i32 + 1;
      plan.g_inst = P->plan_i32 + 2;
      plan.g_bar = P->bar;
      plan.g_part = P->part;
      plan.g_part_off = P->part_off;
      grid = nblk;
    } else {
      plan.npool = 1;
      plan.pool_inst = P->plan_i32 + 3;
      plan.pool_next = P->plan_i32 + 4;
      plan.diag_only = P->method == PDHCG_INNER_DIAG && P->k == 0;
      plan.smem_vec_bytes = int64_t(std::min(smem_need(P), kSmemVecBudget));
      plan.pool_bs = pool_width(P);
    }
    cudaError_t e = launch_solve<M, V>(static_cast<const Inst<M, V>*>(P->inst_d), plan, grid, P->stream);
    if (e != cudaSuccess) return cuda_fail(e, "solve launch");
    return PDHCG_OK;
  });
  if (rc) return rc;
  CK(cudaMemcpyAsync(&S, P->st, sizeof(S), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  if (S.device_error) {
    set_error("solve: a bounded device wait gave up");
    return PDHCG_E_DEVICE_TIMEOUT;
  }
  if (res) fill_result(P, S, res);
  P->last_state = S;
  return PDHCG_OK;
}

}  // namespace pdhcg

using namespace pdhcg;

extern "C" {

int pdhcg_default_params(pdhcg_params* p) {
  if (!p) return PDHCG_E_INVALID;
  std::memset(p, 0, sizeof(*p));
  p->struct_size = sizeof(pdhcg_params);
  p->precision = PDHCG_FP64;
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
  p->inner = PDHCG_INNER_AUTO;
  p->max_inner_iter = 1000;
  p->ruiz_iters = 10;
  p->restart_sufficient = 0.2;
  p->restart_necessary = 0.8;
  p->restart_artificial = 0.36;
  p->power_max_iter = 1000;
  p->lanes_override = 0;
  p->power_tol = 1e-8;
  p->eta_override = 0.0;
  p->omega0_override = 0.0;
  p->omega_clamp = 1e5;
  p->group_blocks = 0;
  p->device_timeout_ms = 8000;
  p->sell_sigma = 0;
  p->long_row = 0;
  p->huge_row = 0;
  p->pool_ctas_per_sm = 0;
  p->pipeline = 0;
  p->pool_threads = 0;
  return PDHCG_OK;
}

static int check_params(const pdhcg_params* p) {
  if (!p || p->struct_size != sizeof(pdhcg_params)) {
    set_error("params: struct_size mismatch (call pdhcg_default_params first)");
    return PDHCG_E_INVALID;
  }
  if (p->precision < 0 || p->precision > 3 || p->k_eval < 1 || p->max_iter < 1 ||
      !(p->eps_tol > 0) || !(p->eps_inf > 0) || p->max_inner_iter < 0 || p->ruiz_iters < 0 ||
      p->inner < 0 || p->inner > 4 || !(p->omega_clamp >= 1.0) || p->power_max_iter < 1 ||
      (p->lanes_override != 0 && (p->lanes_override > 32 || (p->lanes_override & (p->lanes_override - 1)))) ||
      p->sell_sigma < 0 || p->long_row < 0 || p->huge_row < 0 || p->pool_ctas_per_sm < 0 ||
      p->pipeline < -1 || p->pipeline > 1 ||
      (p->pool_threads != 0 && p->pool_threads != 128 && p->pool_threads != 256) ||
      sell_layout_of(*p).long_row >= sell_layout_of(*p).huge_row) {
    set_error("params: value out of range");
    return PDHCG_E_INVALID;
  }
  return PDHCG_OK;
}

}  // extern "C"

namespace pdhcg {

// Host side of creation: validate, canonicalise, choose the inner solver, build
// the SELL layouts.  No device work.
int prepare_problem(const CreateInput& in, const pdhcg_params& prm, void* stream, pdhcg_problem** out,
                    HostQP* h) {
  int rc = build_host_qp(in.Q, in.A, in.c, in.lc, in.uc, in.lv, in.uv, h, in.R);
  if (rc) return rc;
  int method = prm.inner;
  if (method == PDHCG_INNER_CG_LIFTED) {
    lift_box_rows(h);
    method = PDHCG_INNER_AUTO;  // no finite variable bound is left
  }
  if (method == PDHCG_INNER_AUTO) method = h->diag_q ? PDHCG_INNER_DIAG : (h->any_box ? PDHCG_INNER_BB : PDHCG_INNER_CG);
  if (method == PDHCG_INNER_DIAG && !h->diag_q) {
    set_error("inner = DIAG needs a diagonal Q");
    return PDHCG_E_INVALID;
  }
  if (method == PDHCG_INNER_CG && h->any_box) {
    set_error("inner = CG needs every variable free (no finite bound)");
    return PDHCG_E_INVALID;
  }
  auto* P = new (std::nothrow) pdhcg_problem();
  if (!P) return PDHCG_E_OOM;
  P->prm = prm;
  P->precision = prm.precision;
  P->method = method;
  P->n = h->n;
  P->m = h->m;
  P->m_user = h->m_user;
  P->nnzQ = int64_t(h->Qc.size());
  P->nnzA = int64_t(h->Ac.size());
  P->has_q = h->has_q;
  P->stream = static_cast<cudaStream_t>(stream);
  P->Qp = h->Qp;
  P->Ap = h->Ap;
  P->ATp = h->ATp;
  {
    const double avg_q = P->n ? double(P->nnzQ) / P->n : 0.0;
    const double avg_at = P->n ? double(P->nnzA) / P->n : 0.0;
    const double avg_a = P->m ? double(P->nnzA) / P->m : 0.0;
    P->lanes_var = lanes_for(method == PDHCG_INNER_DIAG ? avg_at : std::max(avg_q, avg_at));
    P->lanes_con = lanes_for(avg_a);
    if (prm.lanes_override) P->lanes_var = P->lanes_con = prm.lanes_override;
  }
  const SellLayout lay = sell_layout_of(prm);
  const std::vector<int32_t>* vrp[2] = {&h->ATp, &h->Qp};
  const std::vector<int32_t>* vci[2] = {&h->ATc, &h->Qc};
  build_sell(h->n, h->has_q ? 2 : 1, vrp, vci, &P->vsell, lay);
  const std::vector<int32_t>* crp[2] = {&h->Ap, nullptr};
  const std::vector<int32_t>* cci[2] = {&h->Ac, nullptr};
  build_sell(h->m, 1, crp, cci, &P->csell, lay);
  P->vsell_cols[0] = P->vsell.col[0].size();
  P->vsell_cols[1] = P->vsell.col[1].size();
  P->csell_cols = P->csell.col[0].size();
  if (h->k > 0) {
    P->k = h->k;
    P->nnzR = int64_t(h->Rc.size());
    P->Rp = h->Rp;
    const std::vector<int32_t>* rrp[2] = {&h->Rp, nullptr};
    const std::vector<int32_t>* rci[2] = {&h->Rc, nullptr};
    build_sell(h->k, 1, rrp, rci, &P->rsell, lay);
    P->rsell_cols = P->rsell.col[0].size();
  }
  *out = P;
  return PDHCG_OK;
}


// Create count handles: one device allocation, one staging transfer per handle,
// and (count > 1) one pooled setup launch.
int create_impl(int count, const CreateInput* in, const pdhcg_params* params, void* stream,
                pdhcg_t** out, bool pool_only, const CreateAlloc* alloc) {
  pdhcg_params prm;
  if (params) {
    int rc = check_params(params);
    if (rc) return rc;
    prm = *params;
  } else {
    pdhcg_default_params(&prm);
  }
  std::vector<pdhcg_problem*> P(static_cast<size_t>(count), nullptr);
  std::vector<HostQP> H(static_cast<size_t>(count));
  std::vector<int> rcs(static_cast<size_t>(count), PDHCG_OK);
  std::vector<std::string> errs(static_cast<size_t>(count));
  {
    const int nth = std::max(1, std::min<int>(count, int(std::thread::hardware_concurrency())));
    std::atomic<int> nextq(0);
    auto work = [&]() {
      for (int i = nextq++; i < count; i = nextq++) {
        rcs[size_t(i)] = prepare_problem(in[i], prm, stream, &P[size_t(i)], &H[size_t(i)]);
        if (rcs[size_t(i)]) errs[size_t(i)] = last_error_cstr();
      }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nth; ++t) th.emplace_back(work);
    work();
    for (auto& t : th) t.join();
  }
  auto cleanup = [&]() {
    for (auto* q : P) delete q;
  };
  for (int i = 0; i < count; ++i)
    if (rcs[size_t(i)]) {
      set_error("problem " + std::to_string(i) + ": " + errs[size_t(i)]);
      cleanup();
      return rcs[size_t(i)];
    }
  int dev = 0;
  cudaGetDevice(&dev);
  const int mb = cached_max_group_blocks(prm.precision);
  if (mb < 0) {
    cleanup();
    return mb;
  }
  const bool batch = count > 1;
  const bool pooled = batch || pool_only;
  // sizes and offsets inside one allocation
  std::vector<size_t> off(static_cast<size_t>(count));
  size_t total = batch ? ((sizeof(SolverState) * size_t(count) + 255) & ~size_t(255)) : 0;
  size_t stage_total = 0;
  for (int i = 0; i < count; ++i) {
    P[size_t(i)]->device = dev;
    P[size_t(i)]->max_blk = pooled ? 1 : std::max(mb, 1);
    if (pooled) {
      P[size_t(i)]->prm.group_blocks = 1;
      set_batch_grouping(P[size_t(i)]);
    }
    Carver sizing;
    carve(P[size_t(i)], sizing, batch);
    P[size_t(i)]->arena_bytes = (sizing.off + 255) & ~size_t(255);
    off[size_t(i)] = total;
    total += P[size_t(i)]->arena_bytes;
    stage_total += P[size_t(i)]->input_bytes;
  }
  void* raw = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool from_pool = alloc && alloc->pool;
  cudaError_t e = from_pool ? cudaMallocFromPoolAsync(&raw, total, alloc->pool, s) : cudaMalloc(&raw, total);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "cudaMalloc(arena)");
  }
  std::shared_ptr<void> owner = from_pool ? std::shared_ptr<void>(raw, [s](void* q) { cudaFreeAsync(q, s); })
                                          : std::shared_ptr<void>(raw, [](void* q) { cudaFree(q); });
  SolverState* states = batch ? static_cast<SolverState*>(raw) : nullptr;
  for (int i = 0; i < count; ++i) {
    pdhcg_problem* Pi = P[size_t(i)];
    Pi->arena = static_cast<char*>(raw) + off[size_t(i)];
    Pi->arena_owner = owner;
    if (batch) Pi->st = states + i;
    Carver real;
    real.base = static_cast<char*>(Pi->arena);
    carve(Pi, real, batch);
  }
  // stage the inputs in pinned memory and copy each handle's prefix.  Without a
  // caller-owned buffer, the process-wide staging buffer is reused (grown when
  // too small; pinning hundreds of MB per call costs more than the copy).
  static std::mutex g_stage_mu;
  static void* g_stage = nullptr;
  static size_t g_stage_bytes = 0;
  std::unique_lock<std::mutex> stage_lock(g_stage_mu, std::defer_lock);
  CreateAlloc shared_stage;
  if (!(alloc && alloc->pinned && alloc->pinned_bytes)) {
    stage_lock.lock();
    shared_stage.pool = alloc ? alloc->pool : nullptr;
    shared_stage.pinned = &g_stage;
    shared_stage.pinned_bytes = &g_stage_bytes;
    alloc = &shared_stage;
  }
  void* stage = nullptr;
  const bool reuse = alloc && alloc->pinned && alloc->pinned_bytes;
  if (reuse && *alloc->pinned_bytes >= stage_total && *alloc->pinned) {
    stage = *alloc->pinned;
  } else {
    if (reuse && *alloc->pinned) {
      cudaFreeHost(*alloc->pinned);
      *alloc->pinned = nullptr;
      *alloc->pinned_bytes = 0;
    }
    const size_t want = reuse ? std::max<size_t>(stage_total + stage_total / 4, size_t(64) << 20)
                              : std::max<size_t>(stage_total, 1);
    e = cudaMallocHost(&stage, want);
    if (e != cudaSuccess) {
      cleanup();
      return cuda_fail(e, "cudaMallocHost(stage)");
    }
    if (reuse) {
      *alloc->pinned = stage;
      *alloc->pinned_bytes = want;
    }
  }
  std::vector<size_t> soff(static_cast<size_t>(count) + 1, 0);
  for (int i = 0; i < count; ++i) soff[size_t(i) + 1] = soff[size_t(i)] + P[size_t(i)]->input_bytes;
  {
    // pack in parallel (host memory bandwidth), copy in order
    const int nth = std::max(1, std::min<int>(count / 64 + 1, int(std::thread::hardware_concurrency())));
    std::atomic<int> nextp(0);
    auto work = [&]() {
      for (int i = nextp++; i < count; i = nextp++)
        pack_inputs(P[size_t(i)], H[size_t(i)], static_cast<char*>(stage) + soff[size_t(i)]);
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nth; ++t) th.emplace_back(work);
    work();
    for (auto& t : th) t.join();
  }
  std::vector<SolverState> hstates(batch ? size_t(count) : 0);
  for (int i = 0; i < count; ++i) {
    pdhcg_problem* Pi = P[size_t(i)];
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(Pi->arena, static_cast<char*>(stage) + soff[size_t(i)], Pi->input_bytes,
                          cudaMemcpyHostToDevice, s);
    if (batch) {
      hstates[size_t(i)] = SolverState{};
      hstates[size_t(i)].method = Pi->method;
    }
  }
  if (batch && e == cudaSuccess)
    e = cudaMemcpyAsync(states, hstates.data(), sizeof(SolverState) * size_t(count), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (!reuse) cudaFreeHost(stage);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "upload");
  }
  int rc = PDHCG_OK;
  if (!batch) {
    rc = run_setup(P[0]);
  } else {
    rc = dispatch_precision(prm.precision, [&](auto tag) -> int {
      using M = typename decltype(tag)::Mat;
      using V = typename decltype(tag)::Vec;
      std::vector<SetupArgs<M, V>> args(static_cast<size_t>(count));
      for (int i = 0; i < count; ++i) args[size_t(i)] = make_setup_args<M, V>(P[size_t(i)], nullptr);
      const size_t abytes = sizeof(SetupArgs<M, V>) * args.size(), fbytes = 0;
      char* dscratch = nullptr;
      // stream-ordered scratch: a plain cudaFree would wait for every kernel on
      // the device, including a solve running on another stream
      struct ScratchGuard {
        char* p;
        cudaStream_t s;
        ~ScratchGuard() {
          if (p) (void)cudaFreeAsync(p, s);
        }
      };
      if (from_pool) CK(cudaMallocFromPoolAsync(reinterpret_cast<void**>(&dscratch), abytes + fbytes + 256,
                                                alloc->pool, s));
      else CK(cudaMallocAsync(reinterpret_cast<void**>(&dscratch), abytes + fbytes + 256, s));
      ScratchGuard guard{dscratch, s};
      int32_t* ctl = reinterpret_cast<int32_t*>(dscratch + abytes + fbytes);
      CK(cudaMemcpyAsync(dscratch, args.data(), abytes, cudaMemcpyHostToDevice, s));
      CK(cudaMemsetAsync(ctl, 0, 2 * sizeof(int32_t), s));
      const uint64_t tmo = uint64_t(std::max(prm.device_timeout_ms, 1)) * 1000000ull;
      cudaError_t e2 = launch_setup_pool<M, V>(reinterpret_cast<SetupArgs<M, V>*>(dscratch), count, ctl,
                                               ctl + 1, tmo, s);
      if (e2 != cudaSuccess) return cuda_fail(e2, "batched setup");
      CK(cudaMemcpyAsync(hstates.data(), states, sizeof(SolverState) * size_t(count), cudaMemcpyDeviceToHost, s));
      int32_t err = 0;
      CK(cudaMemcpyAsync(&err, ctl + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (err) {
        set_error("batched setup: a bounded device wait gave up");
        return PDHCG_E_DEVICE_TIMEOUT;
      }
      for (int i = 0; i < count; ++i) P[size_t(i)]->setup_state = hstates[size_t(i)];
      return PDHCG_OK;
    });
  }
  if (rc) {
    cleanup();
    return rc;
  }
  for (int i = 0; i < count; ++i) {
    for (int k = 0; k < 2; ++k) {
      std::vector<int32_t>().swap(P[size_t(i)]->vsell.col[k]);
      std::vector<int32_t>().swap(P[size_t(i)]->csell.col[k]);
    }
    if (P[size_t(i)]->batch_nblk > 1) {
      PartitionSet ps;
      bind_partition(ps, P[size_t(i)]->batch_part, P[size_t(i)]->batch_nblk);
      P[size_t(i)]->partitions[P[size_t(i)]->batch_nblk] = ps;
      std::vector<int32_t>().swap(P[size_t(i)]->batch_tables);
    }
    out[i] = P[size_t(i)];
  }
  return PDHCG_OK;
}

int footprint_of(const CreateInput& in, const pdhcg_params& prm, size_t* bytes) {
  HostQP h;
  pdhcg_problem* P = nullptr;
  int rc = prepare_problem(in, prm, nullptr, &P, &h);
  if (rc) return rc;
  P->max_blk = 1;
  set_batch_grouping(P);
  Carver sizing;
  carve(P, sizing, false);
  *bytes = ((sizing.off + 255) & ~size_t(255)) + (1u << 12);
  delete P;
  return PDHCG_OK;
}

int check_params_c(const pdhcg_params* p) { return check_params(p); }

// ---- persistent launches over many instances (batched solves and serving slices) ----
//
// Small instances run on pool CTAs that take them from an atomic queue.  An
// instance whose batch_group_blocks() is above one runs on a multi-CTA group
// of the group-size kernel, in a cooperative launch (every group's CTAs
// co-resident).  Two ways to combine them:
//   * one launch (batched solves): the cooperative launch's CTAs beyond the
//     groups serve the pool; groups take at most half of the co-resident CTAs
//     while pool instances wait;
//   * two launches (serving slices, group_stream given): the pool keeps its own
//     128-thread kernel, so a small request's arithmetic does not depend on
//     what else is live, and the groups run in a cooperative launch of their
//     own on group_stream (created at low priority, so waiting pool CTAs are
//     scheduled first), concurrently; groups take at most half of the
//     co-resident CTAs while pool instances are live.
// A large instance that finds no room runs on a pool CTA (skip_unplaced =
// false), or sits the launch out (skip_unplaced = true: a serving slice, where
// it gets its group in a later slice).
//
// Device scratch, carved from d: the descriptors, the queue, the group
// tables, one zeroed barrier block and the partial sums per group.

size_t batch_scratch_bytes(int count, int ngroups, int group_ctas) {
  Carver c;
  c.take_bytes(size_t(std::max(count, 1)), sizeof(Inst<double, double>));
  c.take<int32_t>(size_t(count) + 8);
  c.take<int32_t>(3 * size_t(std::max(ngroups, 1)));
  c.take<int64_t>(size_t(std::max(ngroups, 1)));
  c.take_bytes(size_t(std::max(ngroups, 1)) * kBarBytes, 1);
  c.take<double>(size_t(2) * kSlots * size_t(std::max(group_ctas, 1)));
  return c.off + 256;
}

struct BatchGroups {
  std::vector<int32_t> inst, nblk;  // group g: instance, CTAs
  std::vector<int32_t> pool;        // pool instances in queue order
  int ctas = 0;                     // CTAs of all groups
};

// Which instances get groups (in the caller's order) within gcap group CTAs.
BatchGroups plan_groups(pdhcg_problem* const* probs, const int32_t* order, int count, int gcap,
                        bool skip_unplaced) {
  BatchGroups b;
  for (int q = 0; q < count; ++q) {
    const int i = order[q];
    const int nb = batch_group_blocks(probs[i]);
    if (nb > 1 && b.ctas + nb <= gcap) {
      b.inst.push_back(i);
      b.nblk.push_back(nb);
      b.ctas += nb;
    } else if (nb <= 1 || !skip_unplaced) {
      b.pool.push_back(i);
    }
  }
  return b;
}

// Streams and events of the two-launch form.
struct SplitLaunch {
  cudaStream_t group_stream = nullptr;
  cudaEvent_t ready = nullptr, done = nullptr;  // inputs copied / groups finished
};

template <class M, class V>
int launch_batch(pdhcg_problem* const* probs, int count, std::vector<Inst<M, V>>& hi, const int32_t* order,
                 int64_t iter_budget, uint64_t slice_ns, char* d, size_t bytes, cudaStream_t s,
                 bool skip_unplaced, const SplitLaunch* split) {
  const pdhcg_problem* P0 = probs[0];
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P0->device));
  size_t need = 0;  // vectors of the largest pool instance, up to the budget
  int nsmall = 0;
  for (int i = 0; i < count; ++i) {
    const bool small = batch_group_blocks(probs[i]) <= 1;
    if (small) need = std::max(need, std::min(smem_need(probs[i]), kSmemVecBudget));
    nsmall += small;
  }
  const bool any_large = nsmall < count;
  // co-resident CTAs of the cooperative launch (its dynamic shared memory:
  // the pool vectors in the one-launch form, none in the two-launch form)
  const size_t coop_smem = split ? 0 : need;
  const int cap = any_large ? std::max(1, group_blocks_per_sm<M, V>(coop_smem)) * sms : 0;
  int gcap = cap;
  if (nsmall > 0) gcap = split ? cap / 2 : std::max(0, cap - std::min(nsmall, cap / 2));
  BatchGroups bg;
  if (any_large) bg = plan_groups(probs, order, count, gcap, skip_unplaced);
  else bg.pool.assign(order, order + count);
  const int ng = int(bg.inst.size());
  if (batch_scratch_bytes(count, ng, bg.ctas) > bytes) {
    set_error("batched launch: scratch too small");
    return PDHCG_E_INVALID;
  }
  if (ng == 0 && bg.pool.empty()) return PDHCG_OK;
  // group instances: their partitions (precomputed for pooled handles)
  std::vector<int64_t> part_off(size_t(std::max(ng, 1)), 0);
  for (int g = 0; g < ng; ++g) {
    pdhcg_problem* P = probs[bg.inst[size_t(g)]];
    PartitionSet* ps = nullptr;
    int rc = get_partition(P, bg.nblk[size_t(g)], &ps);
    if (rc) return rc;
    set_partition(hi[size_t(bg.inst[size_t(g)])], *ps, P);
    if (g + 1 < ng) part_off[size_t(g) + 1] = part_off[size_t(g)] + int64_t(2) * kSlots * bg.nblk[size_t(g)];
  }
  Carver cv;
  cv.base = d;
  void* d_inst = cv.take_bytes(size_t(std::max(count, 1)), sizeof(Inst<double, double>));
  int32_t* d_pool = cv.take<int32_t>(size_t(count) + 8);
  int32_t* d_gtab = cv.take<int32_t>(3 * size_t(std::max(ng, 1)));
  int64_t* d_poff = cv.take<int64_t>(size_t(std::max(ng, 1)));
  unsigned long long* d_bar =
      static_cast<unsigned long long*>(cv.take_bytes(size_t(std::max(ng, 1)) * kBarBytes, 1));
  double* d_part = cv.take<double>(size_t(2) * kSlots * size_t(std::max(bg.ctas, 1)));
  const int npool = int(bg.pool.size());
  std::vector<int32_t> qw(size_t(npool) + 8, 0);
  for (size_t q = 0; q < bg.pool.size(); ++q) qw[q] = bg.pool[q];
  std::vector<int32_t> gt(3 * size_t(std::max(ng, 1)), 0);
  for (int g = 0, first = 0; g < ng; ++g) {
    gt[size_t(g)] = first;
    gt[size_t(ng + g)] = bg.nblk[size_t(g)];
    gt[size_t(2 * ng + g)] = bg.inst[size_t(g)];
    first += bg.nblk[size_t(g)];
  }
  CK(cudaMemcpyAsync(d_inst, hi.data(), sizeof(Inst<M, V>) * size_t(count), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_pool, qw.data(), sizeof(int32_t) * qw.size(), cudaMemcpyHostToDevice, s));
  if (ng > 0) {
    CK(cudaMemcpyAsync(d_gtab, gt.data(), sizeof(int32_t) * gt.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_poff, part_off.data(), sizeof(int64_t) * size_t(ng), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(d_bar, 0, size_t(ng) * kBarBytes, s));
  }
  LaunchPlan base;
  for (int i = 0; i < count; ++i) base.structured |= probs[i]->k > 0;
  base.iter_budget = iter_budget;
  base.slice_ns = slice_ns;
  base.timeout_ns = uint64_t(std::max(P0->prm.device_timeout_ms, 1)) * 1000000ull;
  base.err = d_pool + npool + 1;
  LaunchPlan pool = base;  // pool CTAs
  pool.diag_only = 1;
  for (int i : bg.pool) pool.diag_only &= probs[i]->method == PDHCG_INNER_DIAG && probs[i]->k == 0;
  pool.npool = npool;
  pool.pool_inst = d_pool;
  pool.pool_next = d_pool + npool;
  pool.smem_vec_bytes = int64_t(need);
  LaunchPlan grp = base;   // the groups (and, in the one-launch form, the pool too)
  if (ng > 0) {
    grp.ngroups = ng;
    grp.group_blocks = bg.ctas;
    grp.g_first = d_gtab;
    grp.g_nblk = d_gtab + ng;
    grp.g_inst = d_gtab + 2 * ng;
    grp.g_bar = d_bar;
    grp.g_part = d_part;
    grp.g_part_off = d_poff;
  }
  const Inst<M, V>* di = static_cast<const Inst<M, V>*>(d_inst);
  if (ng > 0 && !split) {  // one cooperative launch: groups, then pool CTAs
    grp.npool = pool.npool;
    grp.pool_inst = pool.pool_inst;
    grp.pool_next = pool.pool_next;
    grp.smem_vec_bytes = pool.smem_vec_bytes;
    const cudaError_t e = launch_solve<M, V>(di, grp, std::min(cap, bg.ctas + npool), s);
    if (e != cudaSuccess) return cuda_fail(e, "batched launch");
    return PDHCG_OK;
  }
  if (ng > 0) {  // the groups' cooperative launch on the second stream, after the copies above
    CK(cudaEventRecord(split->ready, s));
    CK(cudaStreamWaitEvent(split->group_stream, split->ready, 0));
    const cudaError_t e = launch_solve<M, V>(di, grp, bg.ctas, split->group_stream);
    if (e != cudaSuccess) return cuda_fail(e, "group launch");
  }
  if (npool > 0) {
    // As many pool CTAs per SM as registers allow (or pool_ctas_per_sm); each
    // keeps what fits of its instance's vectors in its share of shared memory.
    const int bs = pool_width(P0);
    int per_sm = std::max(1, pool_blocks_per_sm<M, V>(0, bs));
    if (P0->prm.pool_ctas_per_sm > 0) per_sm = std::min(per_sm, P0->prm.pool_ctas_per_sm);
    pool.pool_bs = bs;
    pool.smem_vec_bytes = int64_t(std::min(need, pool_smem_for<M, V>(per_sm, bs)));
    per_sm = std::min(per_sm, std::max(1, pool_blocks_per_sm<M, V>(size_t(pool.smem_vec_bytes), bs)));
    const cudaError_t e = launch_solve<M, V>(di, pool, std::max(1, std::min(npool, per_sm * sms)), s);
    if (e != cudaSuccess) {
      if (ng > 0) (void)cudaStreamSynchronize(split->group_stream);
      return cuda_fail(e, "pool launch");
    }
  }
  if (ng > 0) {  // later work on s (state read-back) waits for the groups too
    CK(cudaEventRecord(split->done, split->group_stream));
    CK(cudaStreamWaitEvent(s, split->done, 0));
  }
  return PDHCG_OK;
}

int launch_pool_slice(pdhcg_problem* const* probs, int count, SolverState* d_states, double* const* x_out,
                      double* const* y_out, int64_t iter_budget, const int* slots, void* scratch,
                      size_t scratch_bytes, uint64_t slice_ns, cudaStream_t group_stream, cudaEvent_t ev_ready,
                      cudaEvent_t ev_done) {
  if (count <= 0) return PDHCG_OK;
  const pdhcg_problem* P0 = probs[0];
  CK(cudaSetDevice(P0->device));
  cudaStream_t s = P0->stream;
  return dispatch_precision(P0->precision, [&](auto tag) -> int {
    using M = typename decltype(tag)::Mat;
    using V = typename decltype(tag)::Vec;
    std::vector<Inst<M, V>> hi(static_cast<size_t>(count));
    std::vector<int32_t> order(static_cast<size_t>(count));
    int ngmax = 0, ctas = 0;
    for (int i = 0; i < count; ++i) {
      hi[size_t(i)] = make_inst<M, V>(probs[i]);
      hi[size_t(i)].st = d_states + (slots ? slots[i] : i);
      hi[size_t(i)].x_out = x_out ? x_out[i] : nullptr;
      hi[size_t(i)].y_out = y_out ? y_out[i] : nullptr;
      order[size_t(i)] = i;
      const int nb = batch_group_blocks(probs[i]);
      if (nb > 1) {
        ngmax++;
        ctas += nb;
      }
    }
    const size_t need = batch_scratch_bytes(count, ngmax, ctas);
    char* d = static_cast<char*>(scratch);
    std::unique_ptr<char, void (*)(char*)> guard(nullptr, [](char* q) { cudaFree(q); });
    if (!d || scratch_bytes < need) {
      CK(cudaMalloc(&d, need));
      guard.reset(d);
    }
    SplitLaunch split{group_stream, ev_ready, ev_done};
    int rc = launch_batch<M, V>(probs, count, hi, order.data(), iter_budget, slice_ns, d,
                                guard ? need : scratch_bytes, s, slice_ns > 0 || iter_budget > 0,
                                group_stream ? &split : nullptr);
    if (rc) {
      if (guard) (void)cudaStreamSynchronize(s);
      return rc;
    }
    // the descriptors must outlive the launch: synchronise before a temporary
    // buffer is freed (a caller's scratch stays valid until it synchronises)
    if (guard) CK(cudaStreamSynchronize(s));
    return PDHCG_OK;
  });
}

}  // namespace pdhcg

extern "C" {

int pdhcg_create(const pdhcg_csr* Q, const pdhcg_csr* A, const double* c, const double* lc,
                 const double* uc, const double* lv, const double* uv, const pdhcg_params* params,
                 void* cuda_stream, pdhcg_t** out) {
  if (!out) {
    set_error("out is NULL");
    return PDHCG_E_INVALID;
  }
  *out = nullptr;
  CreateInput in{Q, A, c, lc, uc, lv, uv};
  return create_impl(1, &in, params, cuda_stream, out, false);
}

int pdhcg_create_qr(const pdhcg_csr* P, const pdhcg_csr* R, const pdhcg_csr* A, const double* c,
                    const double* lc, const double* uc, const double* lv, const double* uv,
                    const pdhcg_params* params, void* cuda_stream, pdhcg_t** out) {
  if (!out || !R) {
    set_error("create_qr: out and R must be given");
    return PDHCG_E_INVALID;
  }
  *out = nullptr;
  CreateInput in{P, A, c, lc, uc, lv, uv, R};
  return create_impl(1, &in, params, cuda_stream, out, false);
}

int pdhcg_create_batch(int count, const pdhcg_problem_data* problems, const pdhcg_params* params,
                       void* cuda_stream, pdhcg_t** out) {
  if (count < 0 || (count > 0 && (!problems || !out))) {
    set_error("create_batch: bad arguments");
    return PDHCG_E_INVALID;
  }
  if (count == 0) return PDHCG_OK;
  for (int i = 0; i < count; ++i) out[i] = nullptr;
  std::vector<CreateInput> in(static_cast<size_t>(count));
  for (int i = 0; i < count; ++i)
    in[size_t(i)] = CreateInput{problems[i].Q, problems[i].A, problems[i].c, problems[i].lc,
                                problems[i].uc, problems[i].lv, problems[i].uv};
  return create_impl(count, in.data(), params, cuda_stream, out, false);
}

int pdhcg_solve(pdhcg_t* P, const double* x0, const double* y0, pdhcg_result* res, double* x_out,
                double* y_out) {
  if (!P) {
    set_error("NULL handle");
    return PDHCG_E_INVALID;
  }
  CK(cudaSetDevice(P->device));
  const size_t n = size_t(P->n), m = size_t(P->m), mu = size_t(P->m_user);
  if (x0) CK(cudaMemcpyAsync(P->x_init_stage, x0, sizeof(double) * n, cudaMemcpyHostToDevice, P->stream));
  if (y0 && m) {
    // lifted bound rows (if any) start with a zero dual
    if (mu < m) CK(cudaMemsetAsync(P->y_init_stage + mu, 0, sizeof(double) * (m - mu), P->stream));
    if (mu) CK(cudaMemcpyAsync(P->y_init_stage, y0, sizeof(double) * mu, cudaMemcpyHostToDevice, P->stream));
  }
  int rc = solve_one(P, x0 ? P->x_init_stage : nullptr, (y0 && m) ? P->y_init_stage : nullptr, res,
                     P->x_stage, P->y_stage);
  if (rc) return rc;
  if (x_out) CK(cudaMemcpyAsync(x_out, P->x_stage, sizeof(double) * n, cudaMemcpyDeviceToHost, P->stream));
  if (y_out && mu) CK(cudaMemcpyAsync(y_out, P->y_stage, sizeof(double) * mu, cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  return PDHCG_OK;
}

int pdhcg_solve_dev(pdhcg_t* P, const double* x0_dev, const double* y0_dev, pdhcg_result* res,
                    double* x_out_dev, double* y_out_dev) {
  if (!P) {
    set_error("NULL handle");
    return PDHCG_E_INVALID;
  }
  if (P->m_user == P->m) return solve_one(P, x0_dev, y0_dev, res, x_out_dev, y_out_dev);
  // lifted bound rows: the caller's y buffers hold only the original rows
  CK(cudaSetDevice(P->device));
  const size_t m = size_t(P->m), mu = size_t(P->m_user);
  if (y0_dev) {
    CK(cudaMemsetAsync(P->y_init_stage + mu, 0, sizeof(double) * (m - mu), P->stream));
    if (mu) CK(cudaMemcpyAsync(P->y_init_stage, y0_dev, sizeof(double) * mu, cudaMemcpyDeviceToDevice, P->stream));
  }
  int rc = solve_one(P, x0_dev, y0_dev ? P->y_init_stage : nullptr, res, x_out_dev, P->y_stage);
  if (rc) return rc;
  if (y_out_dev && mu) {
    CK(cudaMemcpyAsync(y_out_dev, P->y_stage, sizeof(double) * mu, cudaMemcpyDeviceToDevice, P->stream));
    CK(cudaStreamSynchronize(P->stream));
  }
  return PDHCG_OK;
}

int pdhcg_get_eta(const pdhcg_t* P, double* eta, double* norm_A) {
  if (!P) return PDHCG_E_INVALID;
  if (eta) *eta = P->setup_state.eta;
  if (norm_A) *norm_A = P->setup_state.norm_A;
  return PDHCG_OK;
}

int pdhcg_get_scaling(const pdhcg_t* P, double* D, double* E) {
  if (!P) return PDHCG_E_INVALID;
  CK(cudaSetDevice(P->device));
  if (D) CK(cudaMemcpy(D, P->D, sizeof(double) * size_t(P->n), cudaMemcpyDeviceToHost));
  if (E && P->m_user) CK(cudaMemcpy(E, P->E, sizeof(double) * size_t(P->m_user), cudaMemcpyDeviceToHost));
  return PDHCG_OK;
}

int pdhcg_get_phase_times(const pdhcg_t* P, double* seconds8) {
  if (!P || !seconds8) return PDHCG_E_INVALID;
  for (int k = 0; k < 8; ++k) seconds8[k] = P->last_state.tm[k] * 1e-9;
  return PDHCG_OK;
}

int pdhcg_get_info(const pdhcg_t* P, int32_t* n, int32_t* m, size_t* bytes) {
  if (!P) return PDHCG_E_INVALID;
  if (n) *n = P->n;
  if (m) *m = P->m_user;
  if (bytes) *bytes = P->arena_bytes;
  return PDHCG_OK;
}

int pdhcg_get_device(const pdhcg_t* P, int32_t* device) {
  if (!P || !device) return PDHCG_E_INVALID;
  *device = P->device;
  return PDHCG_OK;
}

void pdhcg_destroy(pdhcg_t* P) {
  if (!P) return;
  cudaSetDevice(P->device);
  if (P->stream) cudaStreamSynchronize(P->stream);
  for (auto& kv : P->partitions)
    if (kv.second.owned) cudaFree(kv.second.d_buf);
  if (P->pipe_exec) cudaGraphExecDestroy(P->pipe_exec);
  if (P->pipe_scratch) cudaFree(P->pipe_scratch);
  P->arena_owner.reset();  // frees the allocation with its last handle
  delete P;
}

const char* pdhcg_strerror(int code) {
  switch (code) {
    case PDHCG_OK: return "ok";
    case PDHCG_PENDING: return "pending";
    case PDHCG_E_INVALID: return "invalid argument or problem data";
    case PDHCG_E_OOM: return "out of device memory / over budget";
    case PDHCG_E_CUDA: return "CUDA error";
    case PDHCG_E_BUSY: return "busy";
    case PDHCG_E_NOT_FOUND: return "unknown ticket";
    case PDHCG_E_DEVICE_TIMEOUT: return "bounded device wait gave up";
    default: return "unknown error";
  }
}

const char* pdhcg_last_error(void) { return last_error_cstr(); }

}  // extern "C"

// ---- batched solves: one persistent launch, CTAs pull instances from a queue ----
namespace pdhcg {

struct BatchScratch {
  int device = -1;
  void* buf = nullptr;
  size_t bytes = 0;
};
static std::mutex g_batch_mu;
static std::vector<BatchScratch> g_batch_scratch;

static int batch_buffer(int device, size_t bytes, void** out) {
  for (auto& b : g_batch_scratch)
    if (b.device == device) {
      if (b.bytes < bytes) {
        cudaFree(b.buf);
        b.buf = nullptr;
        b.bytes = 0;
        CK(cudaMalloc(&b.buf, bytes));
        b.bytes = bytes;
      }
      *out = b.buf;
      return PDHCG_OK;
    }
  BatchScratch b;
  b.device = device;
  CK(cudaMalloc(&b.buf, bytes));
  b.bytes = bytes;
  g_batch_scratch.push_back(b);
  *out = b.buf;
  return PDHCG_OK;
}

int solve_batch_impl(pdhcg_t* const* probs, int count, pdhcg_result* res, double* const* x_out,
                     double* const* y_out, int64_t iter_budget) {
  if (count < 0 || (count > 0 && !probs)) {
    set_error("solve_batch: bad arguments");
    return PDHCG_E_INVALID;
  }
  if (count == 0) return PDHCG_OK;
  const pdhcg_problem* P0 = probs[0];
  for (int i = 0; i < count; ++i) {
    if (!probs[i] || probs[i]->precision != P0->precision || probs[i]->device != P0->device ||
        probs[i]->stream != P0->stream) {
      set_error("solve_batch: handles must be non-NULL and share precision, device and stream");
      return PDHCG_E_INVALID;
    }
  }
  std::lock_guard<std::mutex> lk(g_batch_mu);
  CK(cudaSetDevice(P0->device));
  cudaStream_t s = P0->stream;
  size_t sum_n = 0, sum_m = 0;
  std::vector<size_t> xoff(static_cast<size_t>(count)), yoff(static_cast<size_t>(count));
  for (int i = 0; i < count; ++i) {
    xoff[i] = sum_n;
    yoff[i] = sum_m;
    sum_n += size_t(probs[i]->n);
    sum_m += size_t(probs[i]->m);
  }
  // longest-processing-time-first order for the work queue
  std::vector<int32_t> order(static_cast<size_t>(count));
  std::vector<int64_t> work(static_cast<size_t>(count));
  int ngmax = 0, gctas = 0;
  for (int i = 0; i < count; ++i) {
    work[i] = (probs[i]->method != PDHCG_INNER_DIAG ? 4 * probs[i]->nnzQ : 0) + 2 * probs[i]->nnzA +
              probs[i]->n + probs[i]->m;
    order[i] = i;
    const int nb = batch_group_blocks(probs[i]);
    if (nb > 1) {
      ngmax++;
      gctas += nb;
    }
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
  Carver sizing;
  sizing.take<SolverState>(size_t(count));
  sizing.take<double>(sum_n);
  sizing.take<double>(sum_m);
  const size_t launch_bytes = batch_scratch_bytes(count, ngmax, gctas);
  sizing.take_bytes(launch_bytes, 1);
  void* buf = nullptr;
  int rc = batch_buffer(P0->device, sizing.off + 256, &buf);
  if (rc) return rc;
  Carver cv;
  cv.base = static_cast<char*>(buf);
  SolverState* d_st = cv.take<SolverState>(size_t(count));
  double* d_x = cv.take<double>(sum_n);
  double* d_y = cv.take<double>(sum_m);
  char* d_launch = static_cast<char*>(cv.take_bytes(launch_bytes, 1));

  std::vector<SolverState> hs(static_cast<size_t>(count));
  for (int i = 0; i < count; ++i) hs[i] = initial_state(probs[i]);

  rc = dispatch_precision(P0->precision, [&](auto tag) {
    using M = typename decltype(tag)::Mat;
    using V = typename decltype(tag)::Vec;
    std::vector<Inst<M, V>> hi(static_cast<size_t>(count));
    for (int i = 0; i < count; ++i) {
      hi[i] = make_inst<M, V>(probs[i]);
      hi[i].st = d_st + i;
      hi[i].x_out = d_x + xoff[i];
      hi[i].y_out = d_y + yoff[i];
    }
    CK(cudaMemcpyAsync(d_st, hs.data(), sizeof(SolverState) * size_t(count), cudaMemcpyHostToDevice, s));
    // every instance is placed: one that finds no group runs on a pool CTA
    int lrc = launch_batch<M, V>(const_cast<pdhcg_problem* const*>(probs), count, hi, order.data(), iter_budget, 0,
                                 d_launch, launch_bytes, s, false, nullptr);
    if (lrc) {
      (void)cudaStreamSynchronize(s);
      return lrc;
    }
    CK(cudaMemcpyAsync(hs.data(), d_st, sizeof(SolverState) * size_t(count), cudaMemcpyDeviceToHost, s));
    return PDHCG_OK;
  });
  if (rc) return rc;
  std::vector<double> hx, hy;
  const bool want_x = x_out != nullptr, want_y = y_out != nullptr;
  if (want_x) {
    hx.resize(sum_n);
    CK(cudaMemcpyAsync(hx.data(), d_x, sizeof(double) * sum_n, cudaMemcpyDeviceToHost, s));
  }
  if (want_y && sum_m) {
    hy.resize(sum_m);
    CK(cudaMemcpyAsync(hy.data(), d_y, sizeof(double) * sum_m, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  bool dev_err = false;
  for (int i = 0; i < count; ++i) {
    if (hs[i].device_error) dev_err = true;
    probs[i]->last_state = hs[i];
    if (res) fill_result(probs[i], hs[i], res + i);
    if (want_x && x_out[i]) std::memcpy(x_out[i], hx.data() + xoff[i], sizeof(double) * size_t(probs[i]->n));
    if (want_y && y_out[i] && probs[i]->m_user)
      std::memcpy(y_out[i], hy.data() + yoff[i], sizeof(double) * size_t(probs[i]->m_user));
  }
  if (dev_err) {
    set_error("solve_batch: a bounded device wait gave up");
    return PDHCG_E_DEVICE_TIMEOUT;
  }
  return PDHCG_OK;
}

}  // namespace pdhcg

extern "C" int pdhcg_solve_batch(pdhcg_t* const* probs, int count, pdhcg_result* res,
                                 double* const* x_out, double* const* y_out) {
  return pdhcg::solve_batch_impl(probs, count, res, x_out, y_out, 0);
}

// ---- batched solve with static device scratch (no allocation) ----
//
// pdhcg_solve_batch above keeps its per-call scratch (solver states, instance
// descriptors, work queue, solution staging) in a device buffer that it grows
// with cudaMalloc / cudaFree.  This variant serves callers that must not
// allocate while solving: a real-time loop (a model-predictive controller
// re-solving its QPs every control period) cannot take the latency of
// cudaMalloc, nor the device-wide synchronisation of cudaFree; and a process
// whose device memory is already reserved in full by its own pool or budget
// would fail such an allocation with out-of-memory in mid-run.  Its scratch is
// one file-scope device array of fixed size, so it allocates no device, pinned
// or host-heap memory on the success path.
namespace pdhcg {

// At most this many instances per call (states + descriptors + queue words).
constexpr int kNoAllocMaxInstances = PDHCG_NOALLOC_MAX_INSTANCES;
constexpr size_t kNoAllocStateBytes = ((sizeof(SolverState) * kNoAllocMaxInstances + 255) / 256) * 256;
constexpr size_t kNoAllocInstBytes =
    ((sizeof(Inst<double, double>) * kNoAllocMaxInstances + 255) / 256) * 256;
constexpr size_t kNoAllocQueueWords = size_t(kNoAllocMaxInstances) + 8;
constexpr size_t kNoAllocScratchBytes = kNoAllocStateBytes + kNoAllocInstBytes + 4 * kNoAllocQueueWords;
static_assert(sizeof(Inst<float, double>) == sizeof(Inst<double, double>) &&
                  sizeof(Inst<float, float>) == sizeof(Inst<double, double>) &&
                  sizeof(Inst<float, dfloat>) == sizeof(Inst<double, double>),
              "one descriptor stride for every precision");

// The scratch itself: about 1.1 MB per device for 1024 instances, laid out as
// [SolverState x max][Inst x max][int32 order x max, cursor, error flag, pad].
static __device__ __align__(256) char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;                     // one call at a time per process
static char* g_noalloc_dev[kNoAllocMaxDevices];     // scratch address per device, set once
// Host-side staging of the same layout (static, so the call touches no heap).
static SolverState g_noalloc_hstate[kNoAllocMaxInstances];
alignas(256) static unsigned char g_noalloc_hinst[kNoAllocInstBytes];
static int32_t g_noalloc_horder[kNoAllocQueueWords];
static int64_t g_noalloc_hwork[kNoAllocMaxInstances];

// Set-up, once per device, with that device current: the device address of the
// scratch symbol.  The first call on each device does this, so that call should
// come before any stream capture the caller runs on that device.
static int noalloc_scratch(int device, char** out) {
  if (device < 0 || device >= kNoAllocMaxDevices) {
    set_error("solve_batch_noalloc: device ordinal beyond the static table");
    return PDHCG_E_INVALID;
  }
  if (!g_noalloc_dev[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "solve_batch_noalloc: cudaGetSymbolAddress");
    g_noalloc_dev[device] = static_cast<char*>(p);
  }
  *out = g_noalloc_dev[device];
  return PDHCG_OK;
}

int solve_batch_noalloc_impl(pdhcg_t* const* probs, int count, pdhcg_result* res,
                             double* const* x_out_dev, double* const* y_out_dev) {
  if (count < 0 || (count > 0 && !probs)) {
    set_error("solve_batch_noalloc: bad arguments");
    return PDHCG_E_INVALID;
  }
  if (count > kNoAllocMaxInstances) {
    set_error("solve_batch_noalloc: count exceeds the static scratch limit of "
              "PDHCG_NOALLOC_MAX_INSTANCES (1024) instances");
    return PDHCG_E_INVALID;
  }
  if (count == 0) return PDHCG_OK;
  const pdhcg_problem* P0 = probs[0];
  for (int i = 0; i < count; ++i) {
    if (!probs[i] || probs[i]->precision != P0->precision || probs[i]->device != P0->device ||
        probs[i]->stream != P0->stream) {
      set_error("solve_batch_noalloc: handles must be non-NULL and share precision, device and stream");
      return PDHCG_E_INVALID;
    }
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  CK(cudaSetDevice(P0->device));
  char* base = nullptr;
  int rc = noalloc_scratch(P0->device, &base);
  if (rc) return rc;
  cudaStream_t s = P0->stream;
  SolverState* d_st = reinterpret_cast<SolverState*>(base);
  char* d_inst = base + kNoAllocStateBytes;
  int32_t* d_i32 = reinterpret_cast<int32_t*>(base + kNoAllocStateBytes + kNoAllocInstBytes);

  // Longest-processing-time-first queue order (ties by index; std::sort needs no buffer).
  for (int i = 0; i < count; ++i) {
    g_noalloc_hstate[i] = initial_state(probs[i]);
    g_noalloc_hwork[i] = (probs[i]->method != PDHCG_INNER_DIAG ? 4 * probs[i]->nnzQ : 0) +
                         2 * probs[i]->nnzA + probs[i]->n + probs[i]->m;
    g_noalloc_horder[i] = i;
  }
  std::sort(g_noalloc_horder, g_noalloc_horder + count, [](int32_t a, int32_t b) {
    return g_noalloc_hwork[a] != g_noalloc_hwork[b] ? g_noalloc_hwork[a] > g_noalloc_hwork[b] : a < b;
  });
  // The words after the order must start at zero on every call: [count] is the
  // queue cursor the CTAs advance atomically, [count + 1] the device error flag.
  for (size_t w = size_t(count); w < kNoAllocQueueWords; ++w) g_noalloc_horder[w] = 0;

  // Once the kernel is enqueued, every exit waits for the stream first, so the
  // scratch is idle whenever the lock is released (also on an error path).
  bool launched = false;
  auto fail = [&](cudaError_t e, const char* where) {
    if (launched) (void)cudaStreamSynchronize(s);
    return cuda_fail(e, where);
  };
  rc = dispatch_precision(P0->precision, [&](auto tag) {
    using M = typename decltype(tag)::Mat;
    using V = typename decltype(tag)::Vec;
    Inst<M, V>* hi = reinterpret_cast<Inst<M, V>*>(g_noalloc_hinst);
    size_t need = 0;
    for (int i = 0; i < count; ++i) {
      new (&hi[i]) Inst<M, V>(make_inst<M, V>(probs[i]));  // placement into the static staging
      hi[i].st = d_st + i;
      hi[i].x_out = x_out_dev ? x_out_dev[i] : nullptr;
      // lifted bound rows: the kernel writes the handle's own y staging, and
      // the original rows' duals are copied out after the launch
      hi[i].y_out = (y_out_dev && probs[i]->m) ? (probs[i]->m_user == probs[i]->m ? y_out_dev[i]
                                                                                  : probs[i]->y_stage)
                                               : nullptr;
      const size_t b = smem_need(probs[i]);
      if (b <= kSmemVecBudget) need = std::max(need, b);
    }
    CK(cudaMemcpyAsync(d_st, g_noalloc_hstate, sizeof(SolverState) * size_t(count), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_inst, hi, sizeof(Inst<M, V>) * size_t(count), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_i32, g_noalloc_horder, sizeof(int32_t) * kNoAllocQueueWords, cudaMemcpyHostToDevice,
                       s));
    LaunchPlan plan;
    plan.diag_only = 1;
    for (int i = 0; i < count; ++i) {
      plan.structured |= probs[i]->k > 0;
      plan.diag_only &= probs[i]->method == PDHCG_INNER_DIAG && probs[i]->k == 0;
    }
    plan.npool = count;
    plan.pool_inst = d_i32;
    plan.pool_next = d_i32 + count;
    plan.err = d_i32 + count + 1;
    plan.iter_budget = 0;
    plan.smem_vec_bytes = int64_t(need);
    plan.pool_bs = pool_width(P0);
    plan.timeout_ns = uint64_t(std::max(P0->prm.device_timeout_ms, 1)) * 1000000ull;
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P0->device));
    const int per_sm = std::max(1, pool_blocks_per_sm<M, V>(need, plan.pool_bs));
    const int grid = std::max(1, std::min(count, per_sm * sms));
    cudaError_t e = launch_solve<M, V>(reinterpret_cast<const Inst<M, V>*>(d_inst), plan, grid, s);
    if (e != cudaSuccess) return cuda_fail(e, "solve_batch_noalloc launch");
    launched = true;
    e = cudaMemcpyAsync(g_noalloc_hstate, d_st, sizeof(SolverState) * size_t(count), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return fail(e, "solve_batch_noalloc: state read-back");
    return PDHCG_OK;
  });
  if (rc) return rc;
  for (int i = 0; i < count; ++i)
    if (y_out_dev && y_out_dev[i] && probs[i]->m_user && probs[i]->m_user != probs[i]->m) {
      const cudaError_t e = cudaMemcpyAsync(y_out_dev[i], probs[i]->y_stage, sizeof(double) * size_t(probs[i]->m_user),
                                            cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return fail(e, "solve_batch_noalloc: dual copy");
    }
  // Returns only after the launch and the state read-back finished, so the next
  // call (which holds the same lock) never overwrites scratch in use.
  {
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "solve_batch_noalloc: stream synchronize");
  }
  bool dev_err = false;
  for (int i = 0; i < count; ++i) {
    if (g_noalloc_hstate[i].device_error) dev_err = true;
    if (res) fill_result(probs[i], g_noalloc_hstate[i], res + i);
  }
  if (dev_err) {
    set_error("solve_batch_noalloc: a bounded device wait gave up");
    return PDHCG_E_DEVICE_TIMEOUT;
  }
  return PDHCG_OK;
}

}  // namespace pdhcg

extern "C" int pdhcg_solve_batch_noalloc(pdhcg_t* const* probs, int count, pdhcg_result* res,
                                         double* const* x_out_dev, double* const* y_out_dev) {
  return pdhcg::solve_batch_noalloc_impl(probs, count, res, x_out_dev, y_out_dev);
}

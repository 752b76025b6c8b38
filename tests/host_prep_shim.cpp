// host_prep_shim.cpp — test-only C entry points over the library's host-side
// preparation (paper_2602_23967_b300/csrc/host_prep.cpp): the SELL-C-sigma
// packing, the balanced split of rows over a group's CTAs and the lifting of
// variable bounds into rows, so that a CPU test can check them.  Built by
// tests/test_host_prep_cpu.py with g++; not part of the library.
#include <cstring>
#include <vector>

#include "host_problem.h"

namespace {
pdhcg::SellHost g_sell;
std::vector<int32_t> g_rp[2], g_ci[2];
}  // namespace

extern "C" {

// Pack a row space of nrows rows from one or two CSR matrices (rp2 == NULL for
// one).  rp*: nrows + 1 row pointers; ci*: column indices.  Returns 0.
int shim_build_sell(int32_t nrows, const int32_t* rp1, const int32_t* ci1, const int32_t* rp2,
                    const int32_t* ci2) {
  const int nmat = rp2 ? 2 : 1;
  const int32_t* rps[2] = {rp1, rp2};
  const int32_t* cis[2] = {ci1, ci2};
  const std::vector<int32_t>* rp[2] = {nullptr, nullptr};
  const std::vector<int32_t>* ci[2] = {nullptr, nullptr};
  for (int k = 0; k < nmat; ++k) {
    g_rp[k].assign(rps[k], rps[k] + nrows + 1);
    g_ci[k].assign(cis[k], cis[k] + rps[k][nrows]);
    rp[k] = &g_rp[k];
    ci[k] = &g_ci[k];
  }
  pdhcg::build_sell(nrows, nmat, rp, ci, &g_sell);
  return 0;
}

// The same with a row layout of its own (sort window, long and huge row lengths).
int shim_build_sell_layout(int32_t nrows, const int32_t* rp1, const int32_t* ci1, const int32_t* rp2,
                           const int32_t* ci2, int32_t sigma, int64_t long_row, int64_t huge_row) {
  const int nmat = rp2 ? 2 : 1;
  const int32_t* rps[2] = {rp1, rp2};
  const int32_t* cis[2] = {ci1, ci2};
  const std::vector<int32_t>* rp[2] = {nullptr, nullptr};
  const std::vector<int32_t>* ci[2] = {nullptr, nullptr};
  for (int k = 0; k < nmat; ++k) {
    g_rp[k].assign(rps[k], rps[k] + nrows + 1);
    g_ci[k].assign(cis[k], cis[k] + rps[k][nrows]);
    rp[k] = &g_rp[k];
    ci[k] = &g_ci[k];
  }
  pdhcg::SellLayout lay;
  lay.sigma = sigma;
  lay.long_row = long_row;
  lay.huge_row = huge_row;
  pdhcg::build_sell(nrows, nmat, rp, ci, &g_sell, lay);
  return 0;
}

// The autotuner's selection rule on given timings.
int shim_pick_fastest(const double* seconds, int32_t n, double margin) {
  return pdhcg::pick_fastest(std::vector<double>(seconds, seconds + n), margin);
}

// sizes[0..5]: nslices, longs, huges, columns of matrix 0, of matrix 1, nmat-1 slots used.
void shim_sizes(int64_t* sizes) {
  sizes[0] = g_sell.nslices;
  sizes[1] = int64_t(g_sell.longs.size());
  sizes[2] = int64_t(g_sell.huges.size());
  sizes[3] = int64_t(g_sell.col[0].size());
  sizes[4] = int64_t(g_sell.col[1].size());
  sizes[5] = int64_t(g_sell.ptr[1].size());
}

// Copy the layout out; buffers sized by shim_sizes (ptr*: nslices + 1).
void shim_copy(int32_t* perm, int32_t* longs, int32_t* huges, int64_t* ptr0, int64_t* ptr1, int32_t* col0,
               int32_t* col1) {
  std::memcpy(perm, g_sell.perm.data(), sizeof(int32_t) * g_sell.perm.size());
  std::memcpy(longs, g_sell.longs.data(), sizeof(int32_t) * g_sell.longs.size());
  std::memcpy(huges, g_sell.huges.data(), sizeof(int32_t) * g_sell.huges.size());
  std::memcpy(ptr0, g_sell.ptr[0].data(), sizeof(int64_t) * g_sell.ptr[0].size());
  std::memcpy(ptr1, g_sell.ptr[1].data(), sizeof(int64_t) * g_sell.ptr[1].size());
  std::memcpy(col0, g_sell.col[0].data(), sizeof(int32_t) * g_sell.col[0].size());
  std::memcpy(col1, g_sell.col[1].data(), sizeof(int32_t) * g_sell.col[1].size());
}

// Balanced contiguous split of n weights into nblk ranges; bounds: nblk + 1.
void shim_split_balanced(const int64_t* w, int32_t n, int32_t nblk, int32_t* bounds) {
  const std::vector<int64_t> wv(w, w + n);
  const std::vector<int32_t> b = pdhcg::split_balanced(wv, nblk);
  std::memcpy(bounds, b.data(), sizeof(int32_t) * b.size());
}

namespace {
pdhcg::HostQP g_qp;
}

// Validate a problem (Q may be NULL) and lift its finite variable bounds into
// rows (the CG_LIFTED reading).  Returns the library's status code.
int shim_lift(const pdhcg_csr* Q, const pdhcg_csr* A, const double* c, const double* lc, const double* uc,
              const double* lv, const double* uv) {
  g_qp = pdhcg::HostQP{};
  const int rc = pdhcg::build_host_qp(Q, A, c, lc, uc, lv, uv, &g_qp);
  if (rc) return rc;
  pdhcg::lift_box_rows(&g_qp);
  return 0;
}

// sizes[0..2]: m after lifting, nnz(A), m_user
void shim_lift_sizes(int64_t* sizes) {
  sizes[0] = g_qp.m;
  sizes[1] = int64_t(g_qp.Ac.size());
  sizes[2] = g_qp.m_user;
}

// Lifted A (CSR) and A^T (CSR), row bounds, variable bounds and types.
void shim_lift_copy(int32_t* Ap, int32_t* Ac, double* Av, int32_t* ATp, int32_t* ATc, double* ATv, double* lc,
                    double* uc, double* lv, double* uv, int8_t* vtype) {
  std::memcpy(Ap, g_qp.Ap.data(), sizeof(int32_t) * g_qp.Ap.size());
  std::memcpy(Ac, g_qp.Ac.data(), sizeof(int32_t) * g_qp.Ac.size());
  std::memcpy(Av, g_qp.Av.data(), sizeof(double) * g_qp.Av.size());
  std::memcpy(ATp, g_qp.ATp.data(), sizeof(int32_t) * g_qp.ATp.size());
  std::memcpy(ATc, g_qp.ATc.data(), sizeof(int32_t) * g_qp.ATc.size());
  std::memcpy(ATv, g_qp.ATv.data(), sizeof(double) * g_qp.ATv.size());
  std::memcpy(lc, g_qp.lc.data(), sizeof(double) * g_qp.lc.size());
  std::memcpy(uc, g_qp.uc.data(), sizeof(double) * g_qp.uc.size());
  std::memcpy(lv, g_qp.lv.data(), sizeof(double) * g_qp.lv.size());
  std::memcpy(uv, g_qp.uv.data(), sizeof(double) * g_qp.uv.size());
  std::memcpy(vtype, g_qp.vtype.data(), g_qp.vtype.size());
}

}  // extern "C"

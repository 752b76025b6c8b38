// host_prep.cpp — validation and canonical CSR layout of a problem on the host.
//
// Integer bookkeeping only (checks, row sorting, the counting-sort transpose
// that builds the explicit A^T, partition tables); every floating-point step
// of the method runs in the CUDA kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <utility>
#include <string>
#include <vector>

#include "host_problem.h"

namespace pdhcg {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error_cstr() { return g_last_error.c_str(); }

namespace {

int invalid(const std::string& msg) {
  set_error(msg);
  return PDHCG_E_INVALID;
}

// Copy a CSR into int32 row pointers with columns sorted inside each row;
// rejects malformed structure, non-finite values and duplicate entries.
int canon_csr(const pdhcg_csr* M, const char* name, int32_t nrows, int32_t ncols,
              std::vector<int32_t>& rp, std::vector<int32_t>& ci, std::vector<double>& v) {
  if (M->nrows != nrows || M->ncols != ncols)
    return invalid(std::string(name) + ": shape does not match the problem");
  if (M->nnz < 0 || M->nnz >= (int64_t(1) << 31))
    return invalid(std::string(name) + ": nnz must be in [0, 2^31)");
  if (nrows > 0 && (M->rowptr == nullptr)) return invalid(std::string(name) + ": rowptr is NULL");
  if (M->nnz > 0 && (M->col == nullptr || M->val == nullptr))
    return invalid(std::string(name) + ": col/val is NULL");
  rp.assign(size_t(nrows) + 1, 0);
  ci.resize(size_t(M->nnz));
  v.resize(size_t(M->nnz));
  if (nrows == 0) {
    if (M->nnz != 0) return invalid(std::string(name) + ": nnz > 0 with no rows");
    return PDHCG_OK;
  }
  if (M->rowptr[0] != 0) return invalid(std::string(name) + ": rowptr[0] != 0");
  if (M->rowptr[nrows] != M->nnz) return invalid(std::string(name) + ": rowptr[nrows] != nnz");
  std::vector<std::pair<int32_t, double>> tmp;
  for (int32_t i = 0; i < nrows; ++i) {
    const int64_t s = M->rowptr[i], e = M->rowptr[i + 1];
    if (e < s) return invalid(std::string(name) + ": rowptr decreases");
    rp[i + 1] = int32_t(e);
    bool sorted = true;
    for (int64_t k = s; k < e; ++k) {
      const int32_t j = M->col[k];
      const double x = M->val[k];
      if (j < 0 || j >= ncols) return invalid(std::string(name) + ": column index out of range");
      if (!std::isfinite(x)) return invalid(std::string(name) + ": non-finite value");
      if (k > s && j <= M->col[k - 1]) sorted = false;
      ci[k] = j;
      v[k] = x;
    }
    if (!sorted) {
      tmp.clear();
      for (int64_t k = s; k < e; ++k) tmp.emplace_back(ci[k], v[k]);
      std::stable_sort(tmp.begin(), tmp.end(),
                       [](const auto& a, const auto& b) { return a.first < b.first; });
      for (int64_t k = s; k < e; ++k) {
        ci[k] = tmp[size_t(k - s)].first;
        v[k] = tmp[size_t(k - s)].second;
        if (k > s && ci[k] == ci[k - 1])
          return invalid(std::string(name) + ": duplicate entry in a row");
      }
    }
  }
  return PDHCG_OK;
}

// Counting-sort transpose (stable in the row index, so every output row is sorted).
void transpose(int32_t nrows, int32_t ncols, const std::vector<int32_t>& rp,
               const std::vector<int32_t>& ci, const std::vector<double>& v,
               std::vector<int32_t>& tp, std::vector<int32_t>& tc, std::vector<double>& tv) {
  tp.assign(size_t(ncols) + 1, 0);
  for (int32_t j : ci) tp[size_t(j) + 1]++;
  for (int32_t j = 0; j < ncols; ++j) tp[j + 1] += tp[j];
  tc.resize(ci.size());
  tv.resize(v.size());
  std::vector<int32_t> cur(tp.begin(), tp.end() - 1);
  for (int32_t i = 0; i < nrows; ++i)
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int32_t dst = cur[ci[k]]++;
      tc[dst] = i;
      tv[dst] = v[k];
    }
}

int check_bounds(const double* lo, const double* hi, int32_t len, const char* what) {
  for (int32_t i = 0; i < len; ++i) {
    const double l = lo[i], u = hi[i];
    if (std::isnan(l) || std::isnan(u)) return invalid(std::string(what) + ": NaN bound");
    if (l > u) return invalid(std::string(what) + ": lower bound above upper bound");
    if (l == INFINITY || u == -INFINITY) return invalid(std::string(what) + ": infeasible infinite bound");
  }
  return PDHCG_OK;
}

int8_t bound_type(double l, double u) {
  return int8_t((std::isfinite(l) ? 1 : 0) | (std::isfinite(u) ? 2 : 0));
}

}  // namespace

int build_host_qp(const pdhcg_csr* Q, const pdhcg_csr* A, const double* c, const double* lc,
                  const double* uc, const double* lv, const double* uv, HostQP* h, const pdhcg_csr* R) {
  if (A == nullptr) return invalid("A must be given (use nrows = 0 for no constraints)");
  const int32_t n = A->ncols, m = A->nrows;
  if (n <= 0) return invalid("n must be positive");
  if (m < 0) return invalid("m must be non-negative");
  if (c == nullptr || lv == nullptr || uv == nullptr) return invalid("c, lv, uv must be given");
  if (m > 0 && (lc == nullptr || uc == nullptr)) return invalid("lc, uc must be given");
  h->n = n;
  h->m = m;
  int rc = canon_csr(A, "A", m, n, h->Ap, h->Ac, h->Av);
  if (rc) return rc;
  h->has_q = Q != nullptr;
  h->diag_q = true;
  if (Q) {
    rc = canon_csr(Q, "Q", n, n, h->Qp, h->Qc, h->Qv);
    if (rc) return rc;
    // symmetry: compare Q with its transpose entry by entry (missing = 0)
    std::vector<int32_t> tp, tc;
    std::vector<double> tv;
    transpose(n, n, h->Qp, h->Qc, h->Qv, tp, tc, tv);
    double qmax = 0.0;
    for (double x : h->Qv) qmax = std::max(qmax, std::fabs(x));
    for (int32_t i = 0; i < n; ++i) {
      int32_t a = h->Qp[i], ae = h->Qp[i + 1], b = tp[i], be = tp[i + 1];
      while (a < ae || b < be) {
        double va = 0.0, vb = 0.0;
        int32_t ja = a < ae ? h->Qc[a] : INT32_MAX, jb = b < be ? tc[b] : INT32_MAX;
        int32_t j = std::min(ja, jb);
        if (ja == j) va = h->Qv[a++];
        if (jb == j) vb = tv[b++];
        if (std::fabs(va - vb) > 1e-12 * (std::fabs(va) + std::fabs(vb)) + 1e-14 * qmax)
          return invalid("Q is not symmetric");
      }
    }
    for (int32_t i = 0; i < n && h->diag_q; ++i)
      for (int32_t k = h->Qp[i]; k < h->Qp[i + 1]; ++k)
        if (h->Qc[k] != i && h->Qv[k] != 0.0) {
          h->diag_q = false;
          break;
        }
  } else {
    h->Qp.assign(size_t(n) + 1, 0);
    h->Qc.clear();
    h->Qv.clear();
  }
  if (R) {
    // Q v = P v + R^T (R v): keep R, and store [P | R^T] in the Q arrays
    if (R->ncols != n || R->nrows <= 0) return invalid("R: must be k x n with k >= 1");
    h->k = R->nrows;
    rc = canon_csr(R, "R", h->k, n, h->Rp, h->Rc, h->Rv);
    if (rc) return rc;
    std::vector<int32_t> tp, tc;
    std::vector<double> tv;
    transpose(h->k, n, h->Rp, h->Rc, h->Rv, tp, tc, tv);
    std::vector<int32_t> qp(size_t(n) + 1, 0), qc;
    std::vector<double> qv;
    qc.reserve(h->Qc.size() + tc.size());
    qv.reserve(h->Qv.size() + tv.size());
    for (int32_t j = 0; j < n; ++j) {
      for (int32_t q = h->Qp[j]; q < h->Qp[j + 1]; ++q) {
        qc.push_back(h->Qc[q]);
        qv.push_back(h->Qv[q]);
      }
      for (int32_t q = tp[j]; q < tp[j + 1]; ++q) {
        qc.push_back(n + tc[q]);
        qv.push_back(tv[q]);
      }
      qp[size_t(j) + 1] = int32_t(qc.size());
    }
    h->Qp.swap(qp);
    h->Qc.swap(qc);
    h->Qv.swap(qv);
    h->has_q = true;
    h->diag_q = false;
  }
  transpose(m, n, h->Ap, h->Ac, h->Av, h->ATp, h->ATc, h->ATv);
  h->c.assign(c, c + n);
  for (int32_t j = 0; j < n; ++j)
    if (!std::isfinite(c[j])) return invalid("c has a non-finite entry");
  rc = check_bounds(lv, uv, n, "variable bounds");
  if (rc) return rc;
  h->lv.assign(lv, lv + n);
  h->uv.assign(uv, uv + n);
  if (m > 0) {
    rc = check_bounds(lc, uc, m, "constraint bounds");
    if (rc) return rc;
    h->lc.assign(lc, lc + m);
    h->uc.assign(uc, uc + m);
  }
  h->vtype.resize(size_t(n));
  h->ctype.resize(size_t(m));
  h->any_box = false;
  for (int32_t j = 0; j < n; ++j) {
    h->vtype[j] = bound_type(lv[j], uv[j]);
    if (h->vtype[j] != kFree) h->any_box = true;
  }
  for (int32_t i = 0; i < m; ++i) h->ctype[i] = bound_type(lc[i], uc[i]);
  h->m_user = m;
  return PDHCG_OK;
}

void lift_box_rows(HostQP* h) {
  const int32_t n = h->n;
  int32_t added = 0;
  for (int32_t j = 0; j < n; ++j) {
    if (h->vtype[size_t(j)] == kFree) continue;
    h->Ap.push_back(h->Ap.back() + 1);
    h->Ac.push_back(j);
    h->Av.push_back(1.0);
    h->lc.push_back(h->lv[size_t(j)]);
    h->uc.push_back(h->uv[size_t(j)]);
    h->ctype.push_back(h->vtype[size_t(j)]);
    h->lv[size_t(j)] = -INFINITY;
    h->uv[size_t(j)] = INFINITY;
    h->vtype[size_t(j)] = kFree;
    ++added;
  }
  h->m += added;
  h->any_box = false;
  transpose(h->m, n, h->Ap, h->Ac, h->Av, h->ATp, h->ATc, h->ATv);
}

SellLayout sell_layout_of(const pdhcg_params& p) {
  SellLayout l;
  if (p.sell_sigma > 0) l.sigma = p.sell_sigma;
  if (p.long_row > 0) l.long_row = p.long_row;
  if (p.huge_row > 0) l.huge_row = p.huge_row;
  return l;
}

int pick_fastest(const std::vector<double>& seconds, double margin) {
  int best = -1;
  for (size_t i = 0; i < seconds.size(); ++i) {
    const double t = seconds[i];
    if (!(t > 0.0) || !std::isfinite(t)) continue;
    if (best < 0 || t < seconds[size_t(best)]) best = int(i);
  }
  if (best <= 0) return best < 0 ? -1 : 0;
  const double t0 = seconds[0];
  if (t0 > 0.0 && std::isfinite(t0) && seconds[size_t(best)] >= t0 * (1.0 - margin)) return 0;
  return best;
}

void build_sell(int32_t nrows, int nmat, const std::vector<int32_t>* rp[2],
                const std::vector<int32_t>* ci[2], SellHost* out, const SellLayout& lay) {
  out->perm.clear();
  out->longs.clear();
  out->huges.clear();
  auto len = [&](int k, int32_t r) -> int64_t { return (*rp[k])[r + 1] - (*rp[k])[r]; };
  std::vector<int32_t> regular;
  regular.reserve(size_t(nrows));
  for (int32_t r = 0; r < nrows; ++r) {
    int64_t mx = 0;
    for (int k = 0; k < nmat; ++k) mx = std::max(mx, len(k, r));
    if (mx >= lay.huge_row) out->huges.push_back(r);
    else if (mx > lay.long_row) out->longs.push_back(r);
    else regular.push_back(r);
  }
  // sort by combined length (descending) inside windows of sigma rows
  std::vector<int64_t> tot(size_t(nrows), 0);
  for (int32_t r : regular)
    for (int k = 0; k < nmat; ++k) tot[size_t(r)] += len(k, r);
  const size_t sigma = size_t(std::max(lay.sigma, 1));
  for (size_t w0 = 0; w0 < regular.size(); w0 += sigma) {
    const size_t w1 = std::min(regular.size(), w0 + sigma);
    std::stable_sort(regular.begin() + long(w0), regular.begin() + long(w1),
                     [&](int32_t a, int32_t b) { return tot[size_t(a)] > tot[size_t(b)]; });
  }
  out->nslices = int32_t((regular.size() + 31) / 32);
  out->perm.assign(size_t(out->nslices) * 32, -1);
  std::copy(regular.begin(), regular.end(), out->perm.begin());
  for (int k = 0; k < 2; ++k) {
    out->ptr[k].assign(size_t(out->nslices) + 1, 0);
    out->col[k].clear();
  }
  for (int k = 0; k < nmat; ++k) {
    std::vector<int64_t>& ptr = out->ptr[k];
    for (int32_t s = 0; s < out->nslices; ++s) {
      int64_t w = 0;
      for (int l = 0; l < 32; ++l) {
        const int32_t r = out->perm[size_t(s) * 32 + size_t(l)];
        if (r >= 0) w = std::max(w, len(k, r));
      }
      ptr[size_t(s) + 1] = ptr[size_t(s)] + 32 * w;
    }
    std::vector<int32_t>& col = out->col[k];
    col.assign(size_t(ptr.back()), 0);
    for (int32_t s = 0; s < out->nslices; ++s) {
      const int64_t w = (ptr[size_t(s) + 1] - ptr[size_t(s)]) / 32;
      for (int l = 0; l < 32; ++l) {
        const int32_t r = out->perm[size_t(s) * 32 + size_t(l)];
        if (r < 0) continue;
        const int64_t b = (*rp[k])[r], lr = len(k, r);
        for (int64_t j = 0; j < w && j < lr; ++j) col[size_t(ptr[size_t(s)] + 32 * j + l)] = (*ci[k])[size_t(b + j)];
      }
    }
  }
}

std::vector<int32_t> split_balanced(const std::vector<int64_t>& w, int nblk) {
  std::vector<int32_t> b(size_t(nblk) + 1, 0);
  const int32_t N = int32_t(w.size());
  int64_t total = 0;
  for (int64_t x : w) total += x;
  int64_t acc = 0;
  int32_t i = 0;
  for (int k = 1; k < nblk; ++k) {
    const double target = double(total) * k / nblk;
    while (i < N && double(acc) + 0.5 * double(w[size_t(i)]) < target) acc += w[size_t(i++)];
    b[size_t(k)] = i;
  }
  b[size_t(nblk)] = N;
  return b;
}

}  // namespace pdhcg

// setup_kernel.cuh — device setup of one instance (off the timed loop).
//
//  1. Ruiz equilibration of K = [Q A^T; A 0] in the infinity norm (reading of the
//     paper's unstated "system scaling"): each pass divides every column of the
//     currently scaled K by the square root of its largest magnitude.  The
//     scaled entries are (Q_ij D_i) D_j and (A_ij E_i) D_j.
//  2. Scaled data in the iteration's types: Q, A, A^T values, c = D c,
//     lv = lv / D, uv = uv / D, lc = E lc, uc = E uc, diag(Q), the Gershgorin
//     bound of Q (BB step range), ||c||, ||finite(lc, uc)|| (initial primal weight).
//  2b. The scaled values in SELL slice order (the solve kernel's layout).
//  3. ||A||_2 of the scaled A (the values the iteration uses) by Lanczos on
//     A^T A in FP64 (Sec. 3.2 fixes eta = 0.998/||A|| but not how ||A|| is
//     obtained): t = A v_k, w = A^T t, alpha_k = ||t||^2,
//     w -= alpha_k v_k + beta_{k-1} v_{k-1}, beta_k = ||w||, v_{k+1} = w / beta_k,
//     from v_1 = ones/sqrt(n), without reorthogonalisation (the largest Ritz
//     value converges from below regardless).  The largest eigenvalue of the
//     tridiagonal T_k is taken at k = 8, 16, 24, 36, 54, ... (k + max(8, k/2))
//     and at the step cap; the estimate stops when two agree to power_tol
//     relative or when beta_k vanishes (invariant Krylov space, T_k exact).
#pragma once
#include "device_common.cuh"

namespace pdhcg {

template <class MatT, class VecT>
struct SetupArgs {
  int32_t n, m, has_q, ruiz_iters, power_max_iter, lanes_var, lanes_con;
  double power_tol, eta_override, omega0_override;
  const int32_t *Qp, *Qc, *Ap, *Ac, *ATp, *ATc;
  const double *Qv_o, *Av_o, *ATv_o;  // original values
  const double *c_o, *lv_o, *uv_o, *lc_o, *uc_o;
  const int32_t *var_part, *con_part;
  double *D, *E, *Dn, *En;            // scaling work (D, E hold the result)
  double *pv, *pu, *pw, *pt;          // Lanczos work: v_k, v_{k-1}, w (n each), t (m)
  MatT *Qs, *As, *ATs;                // scaled values (outputs)
  // SELL form of A^T, Q and A (row spaces, slice pointers, columns) and the
  // scaled values in slice order (outputs, filled from Qs / As / ATs)
  SpaceLayout vsp, csp;
  const int64_t *sATp, *sQp, *sAp;
  const int32_t *sATc, *sQc, *sAc;
  MatT *sATv, *sQv, *sAv;
  // structured objective Q = P + R^T R: the Q arrays hold [P | R^T] (columns
  // >= n address R v); R (k x n) with its scaled copy R D and SELL form
  int32_t k;
  const int32_t *Rp, *Rc;
  const double* Rv_o;
  MatT* Rs;
  SpaceLayout rsp;
  const int64_t* sRp;
  MatT* sRv;
  VecT *c, *lv, *uv, *lc, *uc, *qdiag;
  SolverState* st;
  // FP32 matrix values only (else null): rounding remainders of the scaled
  // values, CSR and SELL order, written beside the values above
  float *Qs_lo, *As_lo, *ATs_lo, *sATv_lo, *sQv_lo, *sAv_lo, *Rs_lo, *sRv_lo;
};

// Remainder of a scaled value after rounding to the matrix type: the FP32
// value plus this float reproduces v to about 2^-48 relative.
__device__ __forceinline__ float round_remainder(double v) {
  const float h = float(v);
  return isfinite(h) ? float(v - double(h)) : 0.f;
}

// max over a CSR row of f(k), by a sub-warp of L lanes; result in every lane.
template <class F>
__device__ __forceinline__ double sub_row_max(const int32_t* rp, int row, bool valid, int sl, int L,
                                              F f) {
  double acc = 0.0;
  if (valid)
    for (int k = rp[row] + sl; k < rp[row + 1]; k += L) acc = fmax(acc, f(k));
  for (int off = L >> 1; off > 0; off >>= 1) acc = fmax(acc, __shfl_xor_sync(kFull, acc, off));
  return acc;
}
template <class F>
__device__ __forceinline__ double sub_row_sum(const int32_t* rp, int row, bool valid, int sl, int L,
                                              F f) {
  double acc = 0.0;
  if (valid)
    for (int k = rp[row] + sl; k < rp[row + 1]; k += L) acc += f(k);
  for (int off = L >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
  return acc;
}

// Setup runs one instance per CTA in the batched path; its row loops are
// latency-bound, so rows are summed by at most 4 lanes each and 4 row groups'
// loads are issued together (measured: batched setup of 13 MPC QPs 18.5 ms ->
// 12.1 ms).
#ifndef PDHCG_SETUP_ROWS_UNROLL
#define PDHCG_SETUP_ROWS_UNROLL 4
#endif
constexpr int kSetupRowsUnroll = PDHCG_SETUP_ROWS_UNROLL;
template <int BS, class F>
__device__ __forceinline__ void rows_loop(int lo, int hi, int L, F f) {
  const int sub = threadIdx.x / L, sl = threadIdx.x & (L - 1), nsub = BS / L;
#pragma unroll kSetupRowsUnroll
  for (int base = lo; base < hi; base += nsub) f(base + sub, base + sub < hi, sl);
}

// Lanczos steps kept per estimate (tridiagonal coefficients in shared memory).
constexpr int kLanczosCap = 1024;

// Number of eigenvalues below x of the symmetric tridiagonal matrix with
// diagonal a[0..k) and off-diagonal b[0..k-1): negative pivots of T - x I.
__device__ __forceinline__ int sturm_below(const double* a, const double* b, int k, double x) {
  int c = 0;
  double d = 1.0;
  for (int i = 0; i < k; ++i) {
    d = (a[i] - x) - (i > 0 ? (b[i - 1] * b[i - 1]) / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++c;
  }
  return c;
}

// Largest eigenvalue of that matrix by 33-way multisection over the lanes of one
// warp (every lane a different shift per round, 5 bits per round), from
// [max diagonal, Gershgorin bound] down to adjacent doubles; returns the upper
// end of the final interval.  Called by all 32 lanes of one warp.
__device__ __forceinline__ double tridiag_max_eig_warp(const double* a, const double* b, int k) {
  const int lane = threadIdx.x & 31;
  double lo = a[0], hi = a[0];
  for (int i = lane; i < k; i += 32) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
    lo = fmax(lo, a[i]);
    hi = fmax(hi, a[i] + r);
  }
  for (int off = 16; off > 0; off >>= 1) {
    lo = fmax(lo, __shfl_xor_sync(kFull, lo, off));
    hi = fmax(hi, __shfl_xor_sync(kFull, hi, off));
  }
  hi = hi + 1e-12 * (fabs(hi) + 1e-300);
  for (int round = 0; round < 24; ++round) {
    const double x = lo + (hi - lo) * (double(lane + 1) * (1.0 / 33.0));
    const bool above = x > lo && x < hi && sturm_below(a, b, k, x) == k;
    const unsigned mask = __ballot_sync(kFull, above);
    const int f = mask ? __ffs(mask) - 1 : 32;
    const double nhi = f < 32 ? __shfl_sync(kFull, x, f & 31) : hi;
    const double nlo = f > 0 ? __shfl_sync(kFull, x, (f - 1) & 31) : lo;
    const bool done = !(nhi - nlo > 0x1p-52 * fabs(nhi)) || (nhi == hi && nlo == lo);
    lo = nlo;
    hi = nhi;
    if (done) break;
  }
  return hi;
}

// Scaled CSR values into SELL slice order: warp w of CTA r takes slices
// r * NW + w, stepping over the whole group; padding slots get 0.
template <int BS, class MatT>
__device__ __forceinline__ void fill_sell_space(const Group<BS>& g, int nslices, const int32_t* perm,
                                                const int64_t* sptr, const int32_t* rowptr, const MatT* csr,
                                                MatT* sell) {
  constexpr int NW = BS / 32;
  const int lane = threadIdx.x & 31;
  for (int s = g.rank * NW + int(threadIdx.x >> 5); s < nslices; s += g.nblk * NW) {
    const int row = perm[s * 32 + lane];
    const int64_t b = sptr[s];
    const int W = int((sptr[s + 1] - b) >> 5);
    const int rb = row >= 0 ? rowptr[row] : 0;
    const int len = row >= 0 ? rowptr[row + 1] - rb : 0;
    for (int j = 0; j < W; ++j) sell[b + 32 * j + lane] = j < len ? csr[rb + j] : MatT(0);
  }
}

template <int BS, class MatT, class VecT>
__device__ void setup_instance(Group<BS>& g, const SetupArgs<MatT, VecT>& a) {
  int vlo, vhi, clo, chi;
  g.range(a.var_part, a.n, vlo, vhi);
  g.range(a.con_part, a.m, clo, chi);
#ifndef PDHCG_SETUP_MAX_LANES
#define PDHCG_SETUP_MAX_LANES 4
#endif
  const int Lv = a.lanes_var < PDHCG_SETUP_MAX_LANES ? a.lanes_var : PDHCG_SETUP_MAX_LANES;
  const int Lc = a.lanes_con < PDHCG_SETUP_MAX_LANES ? a.lanes_con : PDHCG_SETUP_MAX_LANES;
  double* D = a.D;
  double* E = a.E;
  double* Dn = a.Dn;
  double* En = a.En;
  for_elems<BS>(vlo, vhi, [&](int j) { D[j] = 1.0; });
  for_elems<BS>(clo, chi, [&](int i) { E[i] = 1.0; });
  // structured Q = P + R^T R: diag(R^T R) (squared column norms of R, the R^T
  // entries of row j of the stored [P | R^T]) joins the column maxima of Ruiz
  double* rdiag = a.pu;  // free until the Lanczos estimate
  if (a.k > 0)
    for_elems<BS>(vlo, vhi, [&](int j) {
      double t = 0.0;
      for (int q = a.Qp[j]; q < a.Qp[j + 1]; ++q)
        if (a.Qc[q] >= a.n) t += a.Qv_o[q] * a.Qv_o[q];
      rdiag[j] = t;
    });
  if (!group_sync<BS>(g)) return;

  // ---- 1. Ruiz passes ----
  for (int pass = 0; pass < a.ruiz_iters; ++pass) {
    rows_loop<BS>(vlo, vhi, Lv, [&](int j, bool valid, int sl) {
      double cq = 0.0;
      if (a.has_q)  // the P part only (columns < n) in a structured objective
        cq = sub_row_max(a.Qp, j, valid, sl, Lv, [&](int k) {
          return a.Qc[k] < a.n ? fabs((a.Qv_o[k] * D[a.Qc[k]]) * D[j]) : 0.0;
        });
      double ca = sub_row_max(a.ATp, j, valid, sl, Lv,
                              [&](int k) { return fabs((a.ATv_o[k] * E[a.ATc[k]]) * D[j]); });
      if (valid && sl == 0) {
        double cn = fmax(cq, ca);
        if (a.k > 0) cn = fmax(cn, (rdiag[j] * D[j]) * D[j]);
        Dn[j] = D[j] * (cn > 0.0 ? 1.0 / sqrt(cn) : 1.0);
      }
    });
    rows_loop<BS>(clo, chi, Lc, [&](int i, bool valid, int sl) {
      double rn = sub_row_max(a.Ap, i, valid, sl, Lc, [&](int k) { return fabs((a.Av_o[k] * E[i]) * D[a.Ac[k]]); });
      if (valid && sl == 0) En[i] = E[i] * (rn > 0.0 ? 1.0 / sqrt(rn) : 1.0);
    });
    if (!group_sync<BS>(g)) return;
    double* t = D; D = Dn; Dn = t;
    t = E; E = En; En = t;
  }
  // the result must end in a.D / a.E
  if (D != a.D) {
    for_elems<BS>(vlo, vhi, [&](int j) { a.D[j] = D[j]; });
    for_elems<BS>(clo, chi, [&](int i) { a.E[i] = E[i]; });
    if (!group_sync<BS>(g)) return;
    D = a.D;
    E = a.E;
  }

  // ---- 2. scaled data ----
  double red[5];  // ||c~||^2, ||b~||^2, gersh (max), bscale (max), cinf (max)
  {
    double cn2 = 0.0, bn2 = 0.0, gmax = 0.0, bsc = 0.0, cinf = 0.0, rcol = 0.0;
    rows_loop<BS>(vlo, vhi, Lv, [&](int j, bool valid, int sl) {
      double qd = 0.0, gs = 0.0, rs = 0.0;
      if (a.has_q) {
        if (valid)
          for (int k = a.Qp[j] + sl; k < a.Qp[j + 1]; k += Lv) {
            const int col = a.Qc[k];
            if (col < a.n) {
              const double v = (a.Qv_o[k] * D[j]) * D[col];
              a.Qs[k] = MatT(v);
              if (a.Qs_lo) a.Qs_lo[k] = round_remainder(v);
              if (col == j) qd += v;
              gs += fabs(v);
            } else {  // (R^T)_j,(col-n) scaled: R D
              const double v = a.Qv_o[k] * D[j];
              a.Qs[k] = MatT(v);
              if (a.Qs_lo) a.Qs_lo[k] = round_remainder(v);
              rs += fabs(v);
            }
          }
        for (int off = Lv >> 1; off > 0; off >>= 1) {
          qd += __shfl_xor_sync(kFull, qd, off);
          gs += __shfl_xor_sync(kFull, gs, off);
          rs += __shfl_xor_sync(kFull, rs, off);
        }
      }
      if (valid)
        for (int k = a.ATp[j] + sl; k < a.ATp[j + 1]; k += Lv) {
          const double v = (a.ATv_o[k] * E[a.ATc[k]]) * D[j];
          a.ATs[k] = MatT(v);
          if (a.ATs_lo) a.ATs_lo[k] = round_remainder(v);
        }
      if (valid && sl == 0) {
        const double cs = a.c_o[j] * D[j];
        a.c[j] = VecT(cs);
        a.lv[j] = VecT(a.lv_o[j] / D[j]);
        a.uv[j] = VecT(a.uv_o[j] / D[j]);
        a.qdiag[j] = VecT(qd);
        cn2 += cs * cs;
        gmax = fmax(gmax, gs);
        rcol = fmax(rcol, rs);  // ||R D||_1 (largest column sum)
        cinf = fmax(cinf, fabs(a.c_o[j]));
      }
    });
    rows_loop<BS>(clo, chi, Lc, [&](int i, bool valid, int sl) {
      if (valid)
        for (int k = a.Ap[i] + sl; k < a.Ap[i + 1]; k += Lc) {
          const double v = (a.Av_o[k] * E[i]) * D[a.Ac[k]];
          a.As[k] = MatT(v);
          if (a.As_lo) a.As_lo[k] = round_remainder(v);
        }
      if (valid && sl == 0) {
        const double l = a.lc_o[i] * E[i], u = a.uc_o[i] * E[i];
        a.lc[i] = VecT(l);
        a.uc[i] = VecT(u);
        if (isfinite(l)) bn2 += l * l;
        if (isfinite(u)) bn2 += u * u;
        if (isfinite(a.lc_o[i])) bsc = fmax(bsc, fabs(a.lc_o[i]));
        if (isfinite(a.uc_o[i])) bsc = fmax(bsc, fabs(a.uc_o[i]));
      }
    });
    // rows of R: scaled copy R D and ||R D||_inf (largest row sum)
    double rrow = 0.0;
    if (a.k > 0) {
      const int r0 = int(int64_t(a.k) * g.rank / g.nblk), r1 = int(int64_t(a.k) * (g.rank + 1) / g.nblk);
      for (int l = r0 + int(threadIdx.x); l < r1; l += BS) {
        double t = 0.0;
        for (int q = a.Rp[l]; q < a.Rp[l + 1]; ++q) {
          const double v = a.Rv_o[q] * D[a.Rc[q]];
          a.Rs[q] = MatT(v);
          if (a.Rs_lo) a.Rs_lo[q] = round_remainder(v);
          t += fabs(v);
        }
        rrow = fmax(rrow, t);
      }
    }
    double red7[7] = {cn2, bn2, gmax, bsc, cinf, rcol, rrow};
    if (!group_reduce<BS, 7>(g, red7, (1u << 2) | (1u << 3) | (1u << 4) | (1u << 5) | (1u << 6))) return;
    red[0] = red7[0];
    red[1] = red7[1];
    // bound on ||Q||: Gershgorin of the scaled P plus ||R D||_2^2 <= ||R D||_1 ||R D||_inf
    red[2] = red7[2] + red7[5] * red7[6];
    red[3] = red7[3];
    red[4] = red7[4];
  }

  // ---- SELL values of the scaled matrices (the solve kernel's layout) ----
  fill_sell_space(g, a.vsp.nslices, a.vsp.perm, a.sATp, a.ATp, a.ATs, a.sATv);
  if (a.has_q) fill_sell_space(g, a.vsp.nslices, a.vsp.perm, a.sQp, a.Qp, a.Qs, a.sQv);
  fill_sell_space(g, a.csp.nslices, a.csp.perm, a.sAp, a.Ap, a.As, a.sAv);
  if (a.k > 0) fill_sell_space(g, a.rsp.nslices, a.rsp.perm, a.sRp, a.Rp, a.Rs, a.sRv);
  if (a.ATs_lo) {
    const float* cATl = a.ATs_lo;
    const float* cQl = a.Qs_lo;
    const float* cAl = a.As_lo;
    fill_sell_space(g, a.vsp.nslices, a.vsp.perm, a.sATp, a.ATp, cATl, a.sATv_lo);
    if (a.has_q) fill_sell_space(g, a.vsp.nslices, a.vsp.perm, a.sQp, a.Qp, cQl, a.sQv_lo);
    fill_sell_space(g, a.csp.nslices, a.csp.perm, a.sAp, a.Ap, cAl, a.sAv_lo);
    if (a.k > 0) {
      const float* cRl = a.Rs_lo;
      fill_sell_space(g, a.rsp.nslices, a.rsp.perm, a.sRp, a.Rp, cRl, a.sRv_lo);
    }
  }
  if (!group_sync<BS>(g)) return;

  // ---- 3. ||A||_2 by Lanczos on A^T A (FP64 vectors, the scaled values) ----
  double lam = 0.0, lam_prev = -1.0, bprev = 0.0;
  int it = 0;
  const int prank = g.nblk > 1 ? g.rank : -1;
  const Csr<MatT> Acsr{a.m, a.Ap[a.m], a.Ap, a.Ac, a.As};
  const Csr<MatT> ATcsr{a.n, a.ATp[a.n], a.ATp, a.ATc, a.ATs};
  RowCtx rc{g.red};
  if (a.m > 0) {
    const int kmax = a.power_max_iter < kLanczosCap ? a.power_max_iter : kLanczosCap;
    const double v0 = 1.0 / sqrt(double(a.n));
    for_elems<BS>(vlo, vhi, [&](int j) {
      a.pv[j] = v0;
      a.pu[j] = 0.0;
    });
    if (!group_sync<BS>(g)) return;
    int next_check = 8;
    for (it = 1; it <= kmax; ++it) {
      // t = A v and w = A^T t with the solver's SELL row engine (plain loads:
      // the SELL values were written by this launch, which rules out the
      // read-only cache path)
      double tt[1] = {0.0};
      space_rows<BS, Ld::Generic, double>(
          a.csp, prank, src(Sell<MatT>{a.sAp, a.sAc, a.sAv}, Acsr, [&](int j) { return a.pv[j]; }),
          nosrc<MatT>(), rc, [&](int i, const double* sums) {
            a.pt[i] = sums[0];
            tt[0] += sums[0] * sums[0];
          });
      if (!group_reduce<BS, 1>(g, tt, 0u)) return;
      const double alpha = tt[0];
      double ww[1] = {0.0};
      space_rows<BS, Ld::Generic, double>(
          a.vsp, prank, src(Sell<MatT>{a.sATp, a.sATc, a.sATv}, ATcsr, [&](int i) { return a.pt[i]; }),
          nosrc<MatT>(), rc, [&](int j, const double* sums) {
            const double wj = sums[0] - alpha * a.pv[j] - bprev * a.pu[j];
            a.pw[j] = wj;
            ww[0] += wj * wj;
          });
      if (!group_reduce<BS, 1>(g, ww, 0u)) return;
      const double beta = sqrt(ww[0]);
      if (threadIdx.x == 0) {
        g.lz[it - 1] = alpha;
        g.lz[kLanczosCap + it - 1] = beta;
      }
      const bool invariant = !(beta > 1e-13 * sqrt(alpha * alpha + bprev * bprev));
      if (it == next_check || invariant || it == kmax) {
        __syncthreads();
        if ((threadIdx.x >> 5) == 0) {
          const double l = tridiag_max_eig_warp(g.lz, g.lz + kLanczosCap, it);
          if (threadIdx.x == 0) g.lz_out[0] = l;
        }
        __syncthreads();
        lam = g.lz_out[0];
        if (invariant || (lam_prev >= 0.0 && fabs(lam - lam_prev) <= a.power_tol * lam)) break;
        lam_prev = lam;
        next_check += next_check / 2 > 8 ? next_check / 2 : 8;
      }
      const double ib = 1.0 / beta;
      for_elems<BS>(vlo, vhi, [&](int j) {
        a.pu[j] = a.pv[j];
        a.pv[j] = a.pw[j] * ib;
      });
      if (!group_sync<BS>(g)) return;
      bprev = beta;
    }
    if (it > kmax) it = kmax;
  }
  if (g.rank == 0 && threadIdx.x == 0) {
    SolverState& S = *a.st;
    const double normA = a.m > 0 ? sqrt(lam) : 0.0;
    S.norm_A = normA;
    S.eta = normA > 0.0 ? 0.998 / normA : 1.0;
    if (a.eta_override > 0.0) S.eta = a.eta_override;
    S.power_iters = it;
    S.gersh = red[2];
    const double cn = sqrt(red[0]), bn = sqrt(red[1]);
    S.omega0 = (cn > 1e-10 && bn > 1e-10) ? cn / bn : 1.0;
    if (a.omega0_override > 0.0) S.omega0 = a.omega0_override;
    S.bscale = red[3];
    S.cinf = red[4];
  }
}

template <int BS, class MatT, class VecT>
__global__ void __launch_bounds__(BS) setup_kernel(SetupArgs<MatT, VecT> a, unsigned long long* bar,
                                                   double* part, int32_t* err, uint64_t timeout_ns) {
  __shared__ double sm_warp[2 * (BS / 32) * kSlots];
  __shared__ double sm_tot[2 * kSlots];
  __shared__ double sm_lz[2 * kLanczosCap + 1];
  __shared__ double sm_red[(BS / 32) * kRowSums];
  __shared__ int sm_flag;
  Group<BS> g;
  g.lz = sm_lz;
  g.lz_out = sm_lz + 2 * kLanczosCap;
  g.red = sm_red;
  g.nblk = gridDim.x;
  g.rank = blockIdx.x;
  g.bar32 = reinterpret_cast<unsigned*>(bar);
  g.epoch = 0;
  g.part = part;
  g.sm_warp = sm_warp;
  g.sm_tot = sm_tot;
  g.sm_flag = &sm_flag;
  g.err = err;
  g.timeout_ns = timeout_ns;
  g.failed = false;
  if (threadIdx.x == 0) sm_flag = 0;
  __syncthreads();
  setup_instance<BS>(g, a);
}

// Setup of many instances in one launch: each CTA takes the next instance from a
// queue and sets it up alone.  Compiled for PDHCG_SETUP_POOL_MIN_BLOCKS resident
// CTAs per SM: the setup of a small instance is a chain of dependent passes
// (Ruiz, Lanczos), so more instances in flight per SM hide more of its latency.
#ifndef PDHCG_SETUP_POOL_MIN_BLOCKS
#define PDHCG_SETUP_POOL_MIN_BLOCKS 2
#endif
template <int BS, class MatT, class VecT>
__global__ void __launch_bounds__(BS, PDHCG_SETUP_POOL_MIN_BLOCKS) setup_pool_kernel(const SetupArgs<MatT, VecT>* args, int count,
                                                        int* next, int32_t* err, uint64_t timeout_ns) {
  __shared__ double sm_warp[2 * (BS / 32) * kSlots];
  __shared__ double sm_tot[2 * kSlots];
  __shared__ double sm_lz[2 * kLanczosCap + 1];
  __shared__ double sm_red[(BS / 32) * kRowSums];
  __shared__ int sm_flag;
  __shared__ int sm_idx;
  Group<BS> g;
  g.lz = sm_lz;
  g.lz_out = sm_lz + 2 * kLanczosCap;
  g.red = sm_red;
  g.nblk = 1;
  g.rank = 0;
  g.bar32 = nullptr;
  g.part = nullptr;
  g.sm_warp = sm_warp;
  g.sm_tot = sm_tot;
  g.sm_flag = &sm_flag;
  g.err = err;
  g.timeout_ns = timeout_ns;
  g.failed = false;
  if (threadIdx.x == 0) sm_flag = 0;
  __syncthreads();
  while (true) {
    if (threadIdx.x == 0) sm_idx = atomicAdd(next, 1);
    __syncthreads();
    const int idx = sm_idx;
    __syncthreads();
    if (idx >= count) break;
    g.epoch = 0;
    setup_instance<BS>(g, args[idx]);
    __syncthreads();
  }
}

}  // namespace pdhcg

// solve_kernel.cuh — the PDHCG-II outer loop and inner solvers as one persistent kernel.
//
// One call of solve_instance() runs the iteration of one instance on a group of
// CTAs (see device_common.cuh) until it stops (KKT tolerance, infeasibility,
// limits) or its slice (a step count or, for serving, device time) is used up.  Per PDHG step:
//
//   Phase I   (n-space rows)  g = A^T y, b = x/tau - c - g            (Eq. primal_update)
//                             DIAG: x+ = clamp(b / (diag Q + 1/tau))   (Sec. 2.2, closed form)
//                             CG:   r = b - H x       BB: grad = H x - b, H = Q + I/tau
//   inner loop                CG (2 phases/step) or projected BB (2 phases/step)  (Sec. 2.2)
//                             to the adaptive tolerance eps_k                      (Sec. 3.3)
//   Phase II  (m-space rows)  A xbar with xbar = 2x+ - x gathered on the fly,
//                             y+ = sigma (v - proj_S(v)), v = y/sigma + A xbar    (Eq. dual_update)
//                             reflected Halpern on y (and x)                       (Sec. 3.1)
//   every k_eval steps        KKT residuals on the original data (Sec. 4.2), primal and dual
//                             infeasibility tests (Sec. 5.1, 5.2), restart test and PID
//                             update of the primal weight (Sec. 3.2, Eq. pid)
//
// Structured objective Q = P + R^T R (Sec. 2.2): before each Q product an
// R-space phase computes t = R v over the k rows of R, and the Q rows gather
// P v and R^T t as one matrix [P | R^T] whose columns >= n address t.  These
// phases exist only in the kernel variant with kR = true.
//
// Vector updates run in VecT; inner products use DotAcc (FP64, or compensated
// FP32 that is exact to about 2^-48 relative) and are combined across the
// group in FP64; all scalar decisions are FP64 and identical in every CTA.
#pragma once
#include "device_common.cuh"

namespace pdhcg {

// Phase functions are separate device functions by default (smaller code, one
// register allocation per phase); PDHCG_INLINE_PHASES=1 inlines them into the
// control loop.
#ifndef PDHCG_INLINE_PHASES
#define PDHCG_INLINE_PHASES 0
#endif
#if PDHCG_INLINE_PHASES
#define PDHCG_PHASE_ATTR __forceinline__
#else
#define PDHCG_PHASE_ATTR __noinline__
#endif
// The two row phases every PDHG step runs (Phase I, Phase II) may be inlined
// into the control loop on their own (PDHCG_INLINE_HOT=1).
#ifndef PDHCG_INLINE_HOT
#define PDHCG_INLINE_HOT 0
#endif
#if PDHCG_INLINE_PHASES || PDHCG_INLINE_HOT
#define PDHCG_HOT_ATTR __forceinline__
#else
#define PDHCG_HOT_ATTR __noinline__
#endif

template <int NV>
struct Red {
  double v[NV];
};

// Thread-local inner-product accumulator.
template <class T>
struct DotAcc;
template <>
struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double get() const { return s; }
};
// FP32 values accumulated as an unevaluated sum hi + lo with error-free
// transformations (TwoProduct by FMA, Knuth's TwoSum): the result is the
// exact dot product of the FP32 inputs up to about 2^-48 relative, at FP32
// throughput (the FP64 pipe of the B300 is too narrow for per-element use).
template <>
struct DotAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_prod(float a, float b) {
    float p = a * b;
    float pe = fmaf(a, b, -p);
    float s = hi + p;
    float bb = s - hi;
    float e = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += e + pe;
  }
  __device__ __forceinline__ double get() const { return double(hi) + double(lo); }
};

// Double-float values: the products of the leading parts are summed exactly as
// for FP32 (TwoProduct, TwoSum); the cross terms hi*lo enter the low word.
template <>
struct DotAcc<dfloat> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_prod(dfloat a, dfloat b) {
    const float p = a.hi * b.hi;
    float pe = fmaf(a.hi, b.hi, -p);
    pe = fmaf(a.hi, b.lo, pe);
    pe = fmaf(a.lo, b.hi, pe);
    float s, e;
    two_sum(hi, p, s, e);
    hi = s;
    lo += e + pe;
  }
  __device__ __forceinline__ double get() const { return double(hi) + double(lo); }
};

// Thread partials -> values handed to group_reduce.  FP64 / FP32 accumulators
// hand over their thread partials (group_reduce sums them across the warp).
// Double-float partials are summed across the warp here, in double-float on the
// FP32 pipe, and lane j converts total j to FP64, so the warp issues one
// conversion for all NV values; group_reduce then skips its warp stage
// (kWarpTotals below).
template <class T>
struct WarpTotals : std::false_type {};
template <>
struct WarpTotals<dfloat> : std::true_type {};

template <int NV, class T>
__device__ __forceinline__ Red<NV> finish_dots(const DotAcc<T> (&a)[NV]) {
  Red<NV> r;
#pragma unroll
  for (int j = 0; j < NV; ++j) r.v[j] = a[j].get();
  return r;
}
template <int NV>
__device__ __forceinline__ Red<NV> finish_dots(const DotAcc<dfloat> (&a)[NV]) {
  static_assert(NV <= 32, "one lane per value");
  const int ln = threadIdx.x & 31;
  dfloat mine(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    float h, l;
    two_sum(a[j].hi, a[j].lo, h, l);
    dfloat t(h, l);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += shfl_xor(t, off);
    if (ln == j) mine = t;
  }
  const double conv = double(mine);
  Red<NV> r;
#pragma unroll
  for (int j = 0; j < NV; ++j) r.v[j] = __shfl_sync(0xffffffffu, conv, j);
  return r;
}

// PID update of log(omega) at the end of a restarted round (Eq. pid).  Skipped
// when either movement is below 1e-10; omega kept within omega0 * [1/c, c].
__device__ __forceinline__ void pid_update(SolverState& S, const DevParams& P, double dx,
                                           double dy) {
  if (!(dx > 1e-10) || !(dy > 1e-10)) return;
  double omega = exp(S.log_omega);
  double e = log(omega * dx / dy);
  S.e_sum += e;
  double lw = S.log_omega - (P.kp * e + P.ki * S.e_sum + P.kd * (e - S.e_prev));
  S.e_prev = e;
  double lim = log(P.omega_clamp);
  lw = fmin(fmax(lw, S.log_omega0 - lim), S.log_omega0 + lim);
  S.log_omega = lw;
}

// Accumulates device-timer intervals per category (thread 0 of the group's first
// CTA) when built with PDHCG_PHASE_TIMERS=1; otherwise every mark is a no-op.
#ifndef PDHCG_PHASE_TIMERS
#define PDHCG_PHASE_TIMERS 0
#endif
struct PhaseClock {
  bool on;
  uint64_t last;
  __device__ __forceinline__ void mark(double* tm, int cat) {
    if (PDHCG_PHASE_TIMERS && on) {
      const uint64_t t = globaltimer_ns();
      tm[cat] += double(t - last);
      last = t;
    }
  }
};


// Scalars of one PDHG step in the vector arithmetic type.
template <class CT>
struct StepScalars {
  CT itau, isig, sig, wk, ak, th, th1;
};

// The step's scalars 1/tau, 1/sigma, sigma, (k+1)/(k+2), 1/(k+2), theta,
// 1 + theta (k: the Halpern index of the step): lane q computes scalar q as one quotient and converts it to the
// vector type, so the warp issues one FP64 division and one conversion for all
// seven (the FP64 pipe is narrow); the values are the same as computing each on
// its own.  Every lane then takes them by shuffle.  Called by whole warps.
template <class CT>
__device__ __forceinline__ StepScalars<CT> step_scalars(const SolverState& S, const DevParams& P, int64_t k,
                                                       double& inv_tau, double& inv_sigma) {
  StepScalars<CT> sc;
  const int ln = threadIdx.x & 31;
  const double kp2 = double(k + 2);
  const double num = ln == 2 ? S.sigma : ln == 3 ? double(k + 1) : ln == 5 ? P.theta : ln == 6 ? 1.0 + P.theta : 1.0;
  const double den = ln == 0 ? S.tau : ln == 1 ? S.sigma : (ln == 3 || ln == 4) ? kp2 : 1.0;
  const double q = num / den;
  const CT qc = CT(q);
  inv_tau = __shfl_sync(kFull, q, 0);
  inv_sigma = __shfl_sync(kFull, q, 1);
  sc.itau = shfl_idx(qc, 0);
  sc.isig = shfl_idx(qc, 1);
  sc.sig = shfl_idx(qc, 2);
  sc.wk = shfl_idx(qc, 3);
  sc.ak = shfl_idx(qc, 4);
  sc.th = shfl_idx(qc, 5);
  sc.th1 = shfl_idx(qc, 6);
  return sc;
}

// Inner tolerance of this step (Sec. 3.3), updating S.eps_in.  With FP32 or
// double-float vectors the subproblem residual cannot be resolved below the
// rounding error of the gradient H x - b: the inner solve stops there instead
// of running to its step cap (FP64 vectors: the paper's rule unchanged).
// FP32: a few units in the last place of b.  Double-float: 16 units of 2^-48
// times ||H|| ||x|| + ||b||, bounded with ||x|| <= tau ||b|| and
// ||H|| <= gersh + 1/tau by (1 + gersh tau) ||b||.
template <class VecT>
__device__ __forceinline__ double inner_tolerance(SolverState& S, const DevParams& P, int method, double bb2,
                                                  double inv_tau) {
  if (S.K == 0) S.eps_in = P.eps_inner_first * fmax(1.0, sqrt(bb2));
  else S.eps_in = fmin(S.eps_in, fmax(P.gamma_inner * S.omega * S.mv * inv_tau, P.eps_inner_min));
  double floor_abs = 0.0;
  if (method != PDHCG_INNER_DIAG) {
    if (sizeof(VecT) == 4) floor_abs = 0x1p-20 * sqrt(bb2);
    else if (std::is_same<VecT, dfloat>::value) floor_abs = 0x1p-44 * (1.0 + S.gersh * S.tau) * sqrt(bb2);
  }
  return fmax(S.eps_in, floor_abs);
}

// ---- structured objective Q = P + R^T R (Sec. 2.2): out = R v over the k rows
// of R, the k-vector that the Q products of the next phase gather from ----
// With FP32 values R v is taken with the remainders as well (R has few rows),
// so t carries no rounding of R and the defect correction at the checks only
// has to cover [P | R^T].
template <int BS, Ld LM, class MatT, class VecT, class G>
__device__ __forceinline__ void r_rows(const Inst<MatT, VecT>& I, int prank, G gat, VecT* __restrict__ out,
                                       const RowCtx& rc) {
  constexpr bool kLo = std::is_same<MatT, float>::value;
  space_rows<BS, LM, VecT>(I.rsp, prank, src_lo<kLo>(I.Rsl, I.R, gat), nosrc<MatT>(), rc,
                           [&](int l, const VecT* sums) {
                             if constexpr (kLo) out[l] = sums[0] + sums[1];
                             else out[l] = sums[0];
                           });
}
// R x (Phase I and BB steps: Q x, x the given vector)
template <int BS, Ld LM, class MatT, class VecT>
__device__ PDHCG_PHASE_ATTR void r_phase_x(const Inst<MatT, VecT>& I, int prank, const VecT* __restrict__ x,
                                           const RowCtx& rc) {
  r_rows<BS, LM>(I, prank, [&](int j) { return x[j]; }, I.rt1, rc);
}
// R p with p = r + beta p_old formed on the fly as in CG Phase A
template <int BS, Ld LM, class MatT, class VecT>
__device__ PDHCG_PHASE_ATTR void r_phase_p(const Inst<MatT, VecT>& I, int prank, bool first, VecT be,
                                           const VecT* __restrict__ pold, const RowCtx& rc) {
  const VecT* __restrict__ rv = I.r;
  r_rows<BS, LM>(I, prank, [&](int j) { return first ? rv[j] : VecT(fma(be, pold[j], rv[j])); }, I.rt1, rc);
}
// R x+ and R (x+ - x) in FP64 for the checks
template <int BS, Ld LM, class MatT, class VecT>
__device__ PDHCG_PHASE_ATTR void r_phase_check(const Inst<MatT, VecT>& I, int prank, int cur, const RowCtx& rc) {
  const VecT* __restrict__ x = cur ? I.xb1 : I.xb0;
  const VecT* __restrict__ xT = I.xT;
  VecT* __restrict__ o1 = I.rt1;
  VecT* __restrict__ o2 = I.rt2;
  constexpr bool kLo = std::is_same<MatT, float>::value;
  space_rows<BS, LM, double>(
      I.rsp, prank,
      src2_lo<kLo>(I.Rsl, I.R, [&](int j) { return double(xT[j]); },
                   [&](int j) { return double(xT[j]) - double(x[j]); }),
      nosrc<MatT>(), rc, [&](int l, const double* sums) {
        if constexpr (kLo) {
          o1[l] = VecT(sums[0] + sums[2]);
          o2[l] = VecT(sums[1] + sums[3]);
        } else {
          o1[l] = VecT(sums[0]);
          o2[l] = VecT(sums[1]);
        }
      });
}

// ---- Phase I: g = A^T y, b = x/tau - c - g, inner-solver start (Eq. primal_update) ----
// returns {inner start norm^2, ||b||^2, ||x+ - x||^2, ||x_new - x||^2}
template <int BS, Ld LM, bool kR, class MatT, class VecT>
__device__ PDHCG_HOT_ATTR Red<4> phase1(const Inst<MatT, VecT>& I, int prank, int method, int cur,
                                      StepScalars<VecT> sc, const RowCtx& rc) {
  using CT = VecT;
  using Acc = VecT;
  const VecT* __restrict__ x = cur ? I.xb1 : I.xb0;
  VecT* __restrict__ xn = cur ? I.xb0 : I.xb1;
  const VecT* __restrict__ y = cur ? I.yb1 : I.yb0;
  const VecT* __restrict__ c = I.c;
  const VecT* __restrict__ lv = I.lv;
  const VecT* __restrict__ uv = I.uv;
  const VecT* __restrict__ qd = I.qdiag;
  const VecT* __restrict__ xa = I.xa;
  VecT* __restrict__ xT = I.xT;
  VecT* __restrict__ xbar = I.xbar;
  VecT* __restrict__ rv = I.r;
  VecT* __restrict__ grad = I.grad;
  VecT* __restrict__ bvv = I.bv;
  const CT itau = sc.itau, wkc = sc.wk, akc = sc.ak, th = sc.th, th1 = sc.th1;
  const int nv = I.n;                    // Q columns >= n address R x (structured Q)
  const VecT* __restrict__ rt = I.rt1;
  DotAcc<CT> a0, a1, a2, a3;
  space_rows<BS, LM, Acc>(
      I.vsp, prank, src(I.ATs, I.AT, [&](int i) { return y[i]; }),
      src(I.Qs, I.Q, [&](int k) { return kR && k >= nv ? rt[k - nv] : x[k]; }, method != PDHCG_INNER_DIAG && I.has_q != 0),
      rc,
      [&](int j, const Acc* sums) {
        const CT xj = x[j];
        const CT bj = xj * itau - c[j] - CT(sums[0]);
        a1.add_prod(bj, bj);
        if (method == PDHCG_INNER_DIAG) {
          const CT xt = clampv(bj / (qd[j] + itau), lv[j], uv[j]);
          const CT xnj = wkc * (th1 * xt - th * xj) + akc * xa[j];
          xT[j] = xt;
          xbar[j] = CT(2) * xt - xj;
          xn[j] = xnj;
          a2.add_prod(xt - xj, xt - xj);
          a3.add_prod(xnj - xj, xnj - xj);
        } else if (method == PDHCG_INNER_CG) {
          const CT hx = CT(sums[1]) + xj * itau;
          const CT rj = bj - hx;
          rv[j] = rj;
          xT[j] = xj;
          a0.add_prod(rj, rj);
        } else {
          const CT hx = CT(sums[1]) + xj * itau;
          const CT gj = hx - bj;
          grad[j] = gj;
          bvv[j] = bj;
          xT[j] = xj;
          const CT d = xj - clampv(xj - gj, lv[j], uv[j]);
          a0.add_prod(d, d);
        }
      });
  const DotAcc<CT> acc[4] = {a0, a1, a2, a3};
  return finish_dots<4>(acc);
}

// ---- CG Phase A: p = r + beta p_old (gathered on the fly, bit-identical to the
// owner's write), q = H p; returns p^T q ----
template <int BS, Ld LM, bool kR, class MatT, class VecT>
__device__ PDHCG_PHASE_ATTR double cg_phase_a(const Inst<MatT, VecT>& I, int prank, bool first, VecT be,
                                          const VecT* __restrict__ pold, VecT* __restrict__ pnew, VecT itau,
                                          const RowCtx& rc) {
  using CT = VecT;
  using Acc = VecT;
  const VecT* __restrict__ rv = I.r;
  VecT* __restrict__ qv = I.q;
  const int nv = I.n;
  const VecT* __restrict__ rt = I.rt1;
  DotAcc<CT> apq;
  space_rows<BS, LM, Acc>(
      I.vsp, prank,
      src(I.Qs, I.Q,
          [&](int k) { return kR && k >= nv ? rt[k - nv] : (first ? rv[k] : CT(fma(be, pold[k], rv[k]))); },
          I.has_q != 0),
      nosrc<MatT>(), rc, [&](int i, const Acc* sums) {
        const CT pi = first ? rv[i] : CT(fma(be, pold[i], rv[i]));
        pnew[i] = pi;
        const CT qi = CT(sums[0]) + pi * itau;
        qv[i] = qi;
        apq.add_prod(pi, qi);
      });
  const DotAcc<CT> acc[1] = {apq};
  return finish_dots<1>(acc).v[0];
}

// ---- CG Phase B: x += alpha p, r -= alpha q; returns r^T r ----
template <int BS, class MatT, class VecT>
__device__ PDHCG_PHASE_ATTR double cg_phase_b(const Inst<MatT, VecT>& I, int lo, int hi, VecT al,
                                          const VecT* __restrict__ pnew) {
  using CT = VecT;
  VecT* __restrict__ xT = I.xT;
  VecT* __restrict__ rv = I.r;
  const VecT* __restrict__ qv = I.q;
  DotAcc<CT> arr;
  for_elems<BS>(lo, hi, [&](int i) {
    xT[i] = xT[i] + al * pnew[i];
    const CT ri = rv[i] - al * qv[i];
    rv[i] = ri;
    arr.add_prod(ri, ri);
  });
  const DotAcc<CT> acc[1] = {arr};
  return finish_dots<1>(acc).v[0];
}

// ---- xbar = 2 x+ - x, optionally copying x+ from another buffer into xT ----
template <int BS, class MatT, class VecT>
__device__ PDHCG_PHASE_ATTR void write_xbar(const Inst<MatT, VecT>& I, int lo, int hi, const VecT* __restrict__ xp,
                                        const VecT* __restrict__ x, bool copy) {
  VecT* __restrict__ xT = I.xT;
  VecT* __restrict__ xbar = I.xbar;
  for_elems<BS>(lo, hi, [&](int i) {
    const VecT xi = xp[i];
    if (copy) xT[i] = xi;
    xbar[i] = VecT(2) * xi - x[i];
  });
}

// ---- BB Phase B': projected step x_new = proj(x - alpha grad) ----
template <int BS, class MatT, class VecT>
__device__ PDHCG_PHASE_ATTR void bb_phase_b(const Inst<MatT, VecT>& I, int lo, int hi, VecT al,
                                        const VecT* __restrict__ xc, const VecT* __restrict__ gc,
                                        VecT* __restrict__ xo) {
  const VecT* __restrict__ lv = I.lv;
  const VecT* __restrict__ uv = I.uv;
  for_elems<BS>(lo, hi, [&](int i) { xo[i] = clampv(xc[i] - al * gc[i], lv[i], uv[i]); });
}

// ---- BB Phase A': gradient, BB quantities and natural residual at xc ----
// returns {s^T s, s^T (g - g_prev), ||x - proj(x - g)||^2}
template <int BS, Ld LM, bool kR, class MatT, class VecT>
__device__ PDHCG_PHASE_ATTR Red<3> bb_phase_a(const Inst<MatT, VecT>& I, int prank, const VecT* __restrict__ xc,
                                          const VecT* __restrict__ xo, const VecT* __restrict__ gc,
                                          VecT* __restrict__ gn, VecT itau, const RowCtx& rc) {
  using CT = VecT;
  using Acc = VecT;
  const VecT* __restrict__ bvv = I.bv;
  const VecT* __restrict__ lv = I.lv;
  const VecT* __restrict__ uv = I.uv;
  DotAcc<CT> ass, asy, anr;
  const int nv = I.n;
  const VecT* __restrict__ rt = I.rt1;
  space_rows<BS, LM, Acc>(I.vsp, prank,
                          src(I.Qs, I.Q, [&](int k) { return kR && k >= nv ? rt[k - nv] : xc[k]; }, I.has_q != 0),
                          nosrc<MatT>(), rc, [&](int i, const Acc* sums) {
                            const CT xi = xc[i];
                            const CT gi = (CT(sums[0]) + xi * itau) - bvv[i];
                            gn[i] = gi;
                            const CT sv = xi - xo[i];
                            const CT yv = gi - gc[i];
                            ass.add_prod(sv, sv);
                            asy.add_prod(sv, yv);
                            const CT d = xi - clampv(xi - gi, lv[i], uv[i]);
                            anr.add_prod(d, d);
                          });
  const DotAcc<CT> acc[3] = {ass, asy, anr};
  return finish_dots<3>(acc);
}

// ---- Phase II: A xbar, dual step (Eq. dual_update), reflected Halpern (Sec. 3.1) ----
// returns {||y+ - y||^2, ||x+ - x||^2, ||x_new - x||^2} (the x terms only for CG / BB)
template <int BS, Ld LM, class MatT, class VecT>
__device__ PDHCG_HOT_ATTR Red<3> phase2(const Inst<MatT, VecT>& I, int prank, int method, int cur, int vlo,
                                      int vhi, StepScalars<VecT> sc, const RowCtx& rc) {
  using CT = VecT;
  using Acc = VecT;
  const VecT* __restrict__ x = cur ? I.xb1 : I.xb0;
  VecT* __restrict__ xn = cur ? I.xb0 : I.xb1;
  const VecT* __restrict__ y = cur ? I.yb1 : I.yb0;
  VecT* __restrict__ yn = cur ? I.yb0 : I.yb1;
  const VecT* __restrict__ xbar = I.xbar;
  const VecT* __restrict__ xT = I.xT;
  VecT* __restrict__ yT = I.yT;
  const VecT* __restrict__ lc = I.lc;
  const VecT* __restrict__ uc = I.uc;
  const VecT* __restrict__ ya = I.ya;
  const VecT* __restrict__ xa = I.xa;
  const CT isig = sc.isig, sig = sc.sig, wkc = sc.wk, akc = sc.ak, th = sc.th, th1 = sc.th1;
  DotAcc<CT> ady, adx, amv;
  space_rows<BS, LM, Acc>(I.csp, prank, src(I.As, I.A, [&](int j) { return xbar[j]; }), nosrc<MatT>(), rc,
                          [&](int i, const Acc* sums) {
                            const CT yi = y[i];
                            const CT v = yi * isig + CT(sums[0]);
                            const CT yt = sig * (v - clampv(v, lc[i], uc[i]));
                            yT[i] = yt;
                            yn[i] = wkc * (th1 * yt - th * yi) + akc * ya[i];
                            ady.add_prod(yt - yi, yt - yi);
                          });
  if (method != PDHCG_INNER_DIAG) {
    for_elems<BS>(vlo, vhi, [&](int j) {
      const CT xt = xT[j], xj = x[j];
      const CT xnj = wkc * (th1 * xt - th * xj) + akc * xa[j];
      xn[j] = xnj;
      adx.add_prod(xt - xj, xt - xj);
      amv.add_prod(xnj - xj, xnj - xj);
    });
  }
  const DotAcc<CT> acc[3] = {ady, adx, amv};
  return finish_dots<3>(acc);
}

// ---- check phase: KKT residual pieces on the original data (Sec. 4.2) and the
// infeasibility tests' pieces (Sec. 5.1, 5.2), with Delta = T(z) - z ----
//
// Every product here is FP64-accurate: with FP32 matrix values the rounding
// remainders are summed as well (val + lo), so the residuals and certificates
// refer to the problem as given, not to its FP32-rounded copy.
//
// Defect correction (FP32 matrix values only).  The iteration applies the
// FP32-rounded matrices A32 = A - A_lo and Q32 = Q - Q_lo, so its fixed point
// would solve a perturbed problem whose FP64 residuals can stay above the
// tolerance.  At every check the remainder products at the current point
// z^ = T(z) are folded into the data the iteration reads:
//   c_eff  = c + A_lo^T y^ (+ Q_lo x^ unless the closed form, which uses the
//            exact diagonal, solves the subproblem)
//   lc_eff = lc - A_lo x^,  uc_eff = uc - A_lo x^      (scaled space)
// so that A32 x + A_lo x^ in [lc, uc] and Q32 x + Q_lo x^ + A32^T y + A_lo^T y^
// are the FP64 constraint and gradient at x = x^.  The correction lags by one
// check and shrinks as z converges; at the fixed point it is exact.
template <int BS, Ld LM, bool kR, class MatT, class VecT>
__device__ PDHCG_PHASE_ATTR Red<18> check_phase(const Inst<MatT, VecT>& I, int prank, int cur, bool corr_q,
                                                const RowCtx& rc) {
  constexpr bool kLo = std::is_same<MatT, float>::value;
  const VecT* __restrict__ x = cur ? I.xb1 : I.xb0;
  const VecT* __restrict__ y = cur ? I.yb1 : I.yb0;
  const VecT* __restrict__ xT = I.xT;
  const VecT* __restrict__ yT = I.yT;
  const VecT* __restrict__ xa = I.xa;
  const VecT* __restrict__ ya = I.ya;
  const VecT* __restrict__ lv = I.lv;
  const VecT* __restrict__ uv = I.uv;
  const int8_t* __restrict__ ctype = I.ctype;
  const int8_t* __restrict__ vtype = I.vtype;
  const int nv = I.n;
  Red<18> cv;
#pragma unroll
  for (int q = 0; q < 18; ++q) cv.v[q] = 0.0;
  space_rows<BS, LM, double>(
      I.csp, prank,
      src2_lo<kLo>(I.As, I.A, [&](int j) { return double(xT[j]); },
                   [&](int j) { return double(xT[j]) - double(x[j]); }),
      nosrc<MatT>(), rc, [&](int i, const double* sums) {
        double ax = sums[0], ad = sums[1], alo = 0.0;
        if constexpr (kLo) {
          alo = sums[2];
          ax += sums[2];
          ad += sums[3];
        }
        const double Ei = I.E[i];
        const double lcs = I.lc_o[i] * Ei, ucs = I.uc_o[i] * Ei;  // scaled bounds as given
        const double axu = ax / Ei;
        cv.v[0] = fmax(cv.v[0], fabs(axu - clampv(axu, I.lc_o[i], I.uc_o[i])));
        const double yu = double(yT[i]) * Ei;
        cv.v[7] += support_term(yu, I.lc_o[i], I.uc_o[i]);
        const double ytl = proj_Y(double(yT[i]) - double(y[i]), ctype[i]);
        cv.v[9] += support_term(ytl, lcs, ucs);
        cv.v[13] = fmax(cv.v[13], fabs(ad - proj_recc(ad, ctype[i])));
        const double dya = double(yT[i]) - double(ya[i]);
        cv.v[16] += dya * dya;
        if constexpr (kLo) {
          I.lc[i] = VecT(lcs - alo);
          I.uc[i] = VecT(ucs - alo);
        }
      });
  space_rows<BS, LM, double>(
      I.vsp, prank,
      src2_lo<kLo>(I.ATs, I.AT, [&](int i) { return double(yT[i]); },
                   [&](int i) { return proj_Y(double(yT[i]) - double(y[i]), ctype[i]); }),
      src2_lo<kLo>(I.Qs, I.Q, [&](int k) { return kR && k >= nv ? double(I.rt1[k - nv]) : double(xT[k]); },
                   [&](int k) { return kR && k >= nv ? double(I.rt2[k - nv]) : double(xT[k]) - double(x[k]); },
                   I.has_q != 0),
      rc, [&](int j, const double* sums) {
        double aty, atyt, qx, qdd, dc = 0.0;
        if constexpr (kLo) {
          aty = sums[0] + sums[2];
          atyt = sums[1] + sums[3];
          qx = sums[4] + sums[6];
          qdd = sums[5] + sums[7];
          dc = sums[2] + (corr_q ? sums[6] : 0.0);
        } else {
          aty = sums[0];
          atyt = sums[1];
          qx = sums[2];
          qdd = sums[3];
        }
        const double Dj = I.D[j];
        const double cs = I.c_o[j] * Dj;  // scaled c as given
        const double xu = double(xT[j]) * Dj;
        const double qxu = qx / Dj, atyu = aty / Dj;
        const double rj = qxu + I.c_o[j] + atyu;
        const double rh = proj_R(rj, vtype[j]);
        cv.v[1] = fmax(cv.v[1], fabs(rj - rh));
        cv.v[2] = fmax(cv.v[2], fabs(qxu));
        cv.v[3] = fmax(cv.v[3], fabs(atyu));
        cv.v[4] += xu * qxu;
        cv.v[5] += I.c_o[j] * xu;
        cv.v[6] += support_term(-rh, I.lv_o[j], I.uv_o[j]);
        cv.v[8] = fmax(cv.v[8], fabs(atyt - proj_R(atyt, vtype[j])));
        cv.v[9] += support_term(-atyt, double(lv[j]), double(uv[j]));
        const double dx = double(xT[j]) - double(x[j]);
        cv.v[10] = fmax(cv.v[10], fabs(dx));
        cv.v[11] += cs * dx;
        cv.v[12] = fmax(cv.v[12], fabs(dx - proj_recc(dx, vtype[j])));
        cv.v[14] = fmax(cv.v[14], fabs(qdd));
        const double dxa = double(xT[j]) - double(xa[j]);
        cv.v[15] += dxa * dxa;
        if constexpr (kLo) I.c[j] = VecT(cs + dc);
      });
  return cv;
}

// ---- output: unscaled solution (x = D x+, y = E y+) or normalised rays ----
template <int BS, class MatT, class VecT>
__device__ PDHCG_PHASE_ATTR Red<2> ray_norms(const Inst<MatT, VecT>& I, int cur, int vlo, int vhi, int clo, int chi,
                                         double dn) {
  const VecT* __restrict__ x = cur ? I.xb1 : I.xb0;
  const VecT* __restrict__ y = cur ? I.yb1 : I.yb0;
  Red<2> mx{{0.0, 0.0}};
  for_elems<BS>(clo, chi, [&](int i) {
    const double ytl = proj_Y(double(I.yT[i]) - double(y[i]), I.ctype[i]) * I.E[i];
    mx.v[0] = fmax(mx.v[0], fabs(ytl));
  });
  for_elems<BS>(vlo, vhi, [&](int j) {
    const double d = ((double(I.xT[j]) - double(x[j])) / dn) * I.D[j];
    mx.v[1] = fmax(mx.v[1], fabs(d));
  });
  return mx;
}

template <int BS, class MatT, class VecT>
__device__ PDHCG_PHASE_ATTR void write_outputs(const Inst<MatT, VecT>& I, int cur, int vlo, int vhi, int clo, int chi,
                                           int status, double dn, double mxy, double mxx) {
  const VecT* __restrict__ x = cur ? I.xb1 : I.xb0;
  const VecT* __restrict__ y = cur ? I.yb1 : I.yb0;
  if (I.x_out) {
    for_elems<BS>(vlo, vhi, [&](int j) {
      double v = double(I.xT[j]) * I.D[j];
      if (status == PDHCG_DUAL_INFEASIBLE) {
        const double d = ((double(I.xT[j]) - double(x[j])) / dn) * I.D[j];
        v = mxx > 0.0 ? d / mxx : 0.0;
      }
      I.x_out[j] = v;
    });
  }
  if (I.y_out) {
    for_elems<BS>(clo, chi, [&](int i) {
      double v = double(I.yT[i]) * I.E[i];
      if (status == PDHCG_PRIMAL_INFEASIBLE) {
        const double ytl = proj_Y(double(I.yT[i]) - double(y[i]), I.ctype[i]) * I.E[i];
        v = mxy > 0.0 ? ytl / mxy : 0.0;
      }
      I.y_out[i] = v;
    });
  }
}

// ---- restart: new anchor and iterate T(z) ----
template <int BS, class MatT, class VecT>
__device__ PDHCG_PHASE_ATTR void restart_copy(const Inst<MatT, VecT>& I, int cur, int vlo, int vhi, int clo, int chi) {
  VecT* __restrict__ x = cur ? I.xb1 : I.xb0;
  VecT* __restrict__ y = cur ? I.yb1 : I.yb0;
  VecT* __restrict__ xa = I.xa;
  VecT* __restrict__ ya = I.ya;
  const VecT* __restrict__ xT = I.xT;
  const VecT* __restrict__ yT = I.yT;
  for_elems<BS>(vlo, vhi, [&](int j) {
    const VecT v = xT[j];
    x[j] = v;
    xa[j] = v;
  });
  for_elems<BS>(clo, chi, [&](int i) {
    const VecT v = yT[i];
    y[i] = v;
    ya[i] = v;
  });
}

template <int BS, class MatT, class VecT>
__device__ PDHCG_PHASE_ATTR void init_point(const Inst<MatT, VecT>& I, int vlo, int vhi, int clo, int chi) {
  constexpr bool kLo = std::is_same<MatT, float>::value;
  for_elems<BS>(vlo, vhi, [&](int j) {
    double x0 = I.x_init ? I.x_init[j] / I.D[j] : 0.0;
    VecT xv = VecT(clampv(x0, double(I.lv[j]), double(I.uv[j])));
    I.xb0[j] = xv;
    I.xa[j] = xv;
    if constexpr (kLo) I.c[j] = VecT(I.c_o[j] * I.D[j]);  // drop a previous solve's correction
  });
  for_elems<BS>(clo, chi, [&](int i) {
    double y0 = I.y_init ? proj_Y(I.y_init[i] / I.E[i], I.ctype[i]) : 0.0;
    I.yb0[i] = VecT(y0);
    I.ya[i] = VecT(y0);
    if constexpr (kLo) {
      I.lc[i] = VecT(I.lc_o[i] * I.E[i]);
      I.uc[i] = VecT(I.uc_o[i] * I.E[i]);
    }
  });
}

// After the check's reduction (cv as check_phase fills it, cv[17] the device
// time): the residuals of Sec. 4.2, recorded in S, and the status they give:
// OPTIMAL, PRIMAL_INFEASIBLE (Sec. 5.1), DUAL_INFEASIBLE (Sec. 5.2), the limits,
// or 0 to continue.
__device__ __forceinline__ int check_status(SolverState& S, const DevParams& P, double bscale, double cinf,
                                            const double* cv) {
  const double r_primal = cv[0] / (1.0 + bscale);
  const double r_dual = cv[1] / (1.0 + fmax(fmax(cv[2], cv[3]), cinf));
  const double xQx = cv[4], cx = cv[5], pr = cv[6], py = cv[7];
  const double pobj = 0.5 * xQx + cx;
  const double dobj = -pr - 0.5 * xQx - py;
  const double gap = fabs(xQx + cx + pr + py);
  const double r_gap = gap / (1.0 + fmax(fabs(pobj), fabs(0.5 * xQx + pr + py)));
  const double rmax = fmax(r_primal, fmax(r_dual, r_gap));
  S.r_primal = r_primal;
  S.r_dual = r_dual;
  S.r_gap = r_gap;
  S.pobj = pobj;
  S.dobj = dobj;
  int status = 0;
  if (!isfinite(rmax)) status = PDHCG_NUMERICAL_ERROR;
  else if (rmax <= P.eps_tol) status = PDHCG_OPTIMAL;
  if (!status) {
    const double neg = cv[9] < 0.0 ? -cv[9] : 0.0;
    if (neg > 0.0 && cv[8] <= P.eps_inf * neg) status = PDHCG_PRIMAL_INFEASIBLE;
  }
  if (!status) {
    const double dn = cv[10];
    if (dn > 0.0) {
      const double vmax = fmax(cv[12] / dn, fmax(cv[13] / dn, cv[14] / dn));
      if (cv[11] / dn < -P.eps_tol && vmax <= P.eps_inf) status = PDHCG_DUAL_INFEASIBLE;
    }
  }
  if (!status && S.K + 1 >= P.max_iter) status = PDHCG_ITERATION_LIMIT;
  if (!status && cv[17] - S.t_start_ns >= P.time_limit_ns) status = PDHCG_TIME_LIMIT;
  return status;
}

// Restart test on the fixed-point residual (reading of the unstated rule) and,
// at a restart, the PID update of the primal weight (Eq. pid) with the new step
// sizes.  Returns whether to restart.
__device__ __forceinline__ bool restart_decision(SolverState& S, const DevParams& P, double fpr, const double* cv) {
  bool do_restart = false;
  if (S.k >= 1) {
    if (fpr <= P.restart_sufficient * S.fpr_anchor) do_restart = true;
    else if (fpr <= P.restart_necessary * S.fpr_anchor && fpr > S.fpr_last) do_restart = true;
    else if (double(S.k + 1) >= P.restart_artificial * double(S.K + 1)) do_restart = true;
  }
  S.fpr_last = fpr;
  if (do_restart) {
    pid_update(S, P, sqrt(cv[15]), sqrt(cv[16]));
    S.omega = exp(S.log_omega);
    S.tau = S.eta / S.omega;
    S.sigma = S.eta * S.omega;
  }
  return do_restart;
}

// Write back the fields of the state that a launch changes.  The read-only
// ones (eta, ||A||, the Gershgorin bound, omega0, the scales, the Lanczos
// count, the method) are left alone, so the control loop does not keep them
// live for a whole-struct store at its end.
__device__ __forceinline__ void store_state(SolverState* d, const SolverState& S) {
  d->K = S.K;
  d->k = S.k;
  d->inner_total = S.inner_total;
  d->restarts = S.restarts;
  d->omega = S.omega;
  d->log_omega = S.log_omega;
  d->e_sum = S.e_sum;
  d->e_prev = S.e_prev;
  d->tau = S.tau;
  d->sigma = S.sigma;
  d->eps_in = S.eps_in;
  d->mv = S.mv;
  d->fpr_anchor = S.fpr_anchor;
  d->fpr_last = S.fpr_last;
  d->r_primal = S.r_primal;
  d->r_dual = S.r_dual;
  d->r_gap = S.r_gap;
  d->pobj = S.pobj;
  d->dobj = S.dobj;
  d->t_start_ns = S.t_start_ns;
  d->t_end_ns = S.t_end_ns;
#if PDHCG_PHASE_TIMERS
  for (int q = 0; q < 8; ++q) d->tm[q] = S.tm[q];
#endif
  d->status = S.status;
  d->cur = S.cur;
  d->started = S.started;
  d->device_error = S.device_error;
  d->form = S.form;
}

// The control loop: scalar state, decisions and group reductions; the row and
// elementwise work is in the phase functions above.
// kR: the structured-Q variant (instances with a factor R); the plain variant
// compiles without the R phases and the split gathers.
template <int BS, Ld LM, bool kR, class MatT, class VecT, bool kDiag = false>
__device__ PDHCG_PHASE_ATTR void solve_instance(Group<BS>& g, const Inst<MatT, VecT>& I, const LaunchPlan& plan,
                                            const RowCtx& rc) {
  using CT = VecT;
  constexpr bool kWT = WarpTotals<VecT>::value;  // phase dots arrive as warp totals
  SolverState S = *I.st;
  if (S.status != 0) return;
  const DevParams& P = I.prm;
  // kDiag: the kernel variant for launches whose instances all use the closed
  // form (diagonal Q); the inner-solver code is compiled out, which spares the
  // control loop registers and their spills
  const int method = kDiag ? int(PDHCG_INNER_DIAG) : S.method;
  int vlo, vhi, clo, chi;
  g.range(I.var_part, I.n, vlo, vhi);
  g.range(I.con_part, I.m, clo, chi);
  const int prank = g.nblk > 1 ? g.rank : -1;
  bool ok = true;
#if PDHCG_PHASE_TIMERS
  PhaseClock clk{threadIdx.x == 0 && g.rank == 0, globaltimer_ns()};
#define PDHCG_CLK(cat) clk.mark(S.tm, cat)
#else
#define PDHCG_CLK(cat) ((void)0)
#endif

  if (!S.started) {
    init_point<BS>(I, vlo, vhi, clo, chi);
    double t[1] = {double(globaltimer_ns())};
    ok = group_reduce<BS, 1>(g, t, 1u);
    S.t_start_ns = t[0];
    S.started = 1;
    S.cur = 0;
  }
  S.form = g.nblk > 1 ? 1 : 0;
  const int64_t K_first = S.K;
  // the next step count that is a multiple of k_eval (a check period ends there)
  int64_t next_check = (S.K / P.k_eval + 1) * P.k_eval;
  // device-time slice budget (single-CTA solves): thread 0 reads the clock every
  // 16 steps and shares the decision, so the whole CTA pauses together
  __shared__ int sm_pause;
  const uint64_t t_resume = globaltimer_ns();

  // The step's FP64 scalars are computed by warp 0 alone and handed to the CTA
  // through shared memory: every warp computing them would occupy the narrow
  // FP64 pipe eight times over.  Same operations on the same values, so the
  // results are the bits each warp would compute.  A box is rewritten only
  // after the group reductions that follow its reads.
  __shared__ StepScalars<CT> sm_sc;
  __shared__ double sm_scal[5];  // 1/tau, 1/sigma, then the step's three square roots
  // The next step's scalars, computed ahead by the last warp after its share of
  // Phase II (it takes the fewest slices), valid when no check ends the step
  // (only a check can restart, which changes k, tau and sigma otherwise).
  __shared__ StepScalars<CT> sm_sc_next;
  __shared__ double sm_scal_next[2];
  bool next_ready = false;
  // The inner solvers' scalar decisions, taken by thread 0 the same way:
  // [0] stop flag, [1] eps, [2] S.eps_in; the step lengths in the vector type.
  __shared__ double sm_in[3];
  __shared__ CT sm_in_ct[2];  // CG beta / BB alpha, CG alpha

  while (ok) {
    const int cur = S.cur;
    double inv_tau, inv_sigma;
    StepScalars<CT> sc;
    if (next_ready) {  // published before the barriers that ended the last step
      sc = sm_sc_next;
      inv_tau = sm_scal_next[0];
      inv_sigma = sm_scal_next[1];
    } else {
      if (threadIdx.x < 32) {
        sc = step_scalars<CT>(S, P, S.k, inv_tau, inv_sigma);
        if (threadIdx.x == 0) {
          sm_sc = sc;
          sm_scal[0] = inv_tau;
          sm_scal[1] = inv_sigma;
        }
      }
      __syncthreads();
      sc = sm_sc;
      inv_tau = sm_scal[0];
      inv_sigma = sm_scal[1];
    }

    // Phase I (structured Q: R x first)
    if (kR && I.k > 0 && method != PDHCG_INNER_DIAG) {
      r_phase_x<BS, LM>(I, prank, cur ? I.xb1 : I.xb0, rc);
      if (!group_sync<BS>(g)) { ok = false; break; }
    }
    double red1[4];
    {
      const Red<4> r = phase1<BS, LM, kR>(I, prank, method, cur, sc, rc);
#pragma unroll
      for (int q = 0; q < 4; ++q) red1[q] = r.v[q];
    }
    PDHCG_CLK(0);
    if (method == PDHCG_INNER_DIAG) {
      // The closed form uses Phase I's sums (the movement norms, slots 2 and 3)
      // only after Phase II: they ride in Phase II's reduction, and Phase I
      // ends with a plain barrier (xbar must be complete).  Same sums, same order.
      if (!group_sync<BS>(g)) { ok = false; break; }
    } else if (!group_reduce<BS, 4, kWT>(g, red1, 0u)) {
      ok = false;
      break;
    }
    PDHCG_CLK(5);

    // adaptive inner tolerance (Sec. 3.3); the closed form has no inner solve
    double eps = 0.0;
    if (method != PDHCG_INNER_DIAG) {
      if (threadIdx.x == 0) {
        sm_in[1] = inner_tolerance<VecT>(S, P, method, red1[1], inv_tau);
        sm_in[2] = S.eps_in;
      }
      __syncthreads();
      eps = sm_in[1];
      S.eps_in = sm_in[2];
    }

    // inner solve (Sec. 2.2)
    if (method == PDHCG_INNER_CG) {
      // rr, the stop test, alpha and beta: thread 0 (FP64), shared with the CTA
      double rr = red1[0], beta = 0.0;
      int j = 0, pc = 0;
      while (true) {
        if (threadIdx.x == 0) {
          sm_in[0] = (sqrt(rr) <= eps || j >= P.max_inner_iter) ? 1.0 : 0.0;
          sm_in_ct[0] = CT(beta);
        }
        __syncthreads();
        if (sm_in[0] != 0.0) break;
        const CT beta_c = sm_in_ct[0];
        const VecT* pold = pc ? I.p1 : I.p0;
        VecT* pnew = pc ? I.p0 : I.p1;
        if (kR && I.k > 0) {
          r_phase_p<BS, LM>(I, prank, j == 0, beta_c, pold, rc);
          if (!group_sync<BS>(g)) { ok = false; break; }
        }
        double pq[1] = {cg_phase_a<BS, LM, kR>(I, prank, j == 0, beta_c, pold, pnew, sc.itau, rc)};
        PDHCG_CLK(1);
        if (!group_reduce<BS, 1, kWT>(g, pq, 0u)) { ok = false; break; }
        PDHCG_CLK(5);
        if (!(pq[0] > 0.0)) break;
        if (threadIdx.x == 0) sm_in_ct[1] = CT(rr / pq[0]);
        __syncthreads();
        double rn[1] = {cg_phase_b<BS>(I, vlo, vhi, sm_in_ct[1], pnew)};
        PDHCG_CLK(2);
        if (!group_reduce<BS, 1, kWT>(g, rn, 0u)) { ok = false; break; }
        PDHCG_CLK(5);
        if (threadIdx.x == 0) beta = rn[0] / rr;
        rr = rn[0];
        pc ^= 1;
        ++j;
      }
      if (!ok) break;
      S.inner_total += j;
      write_xbar<BS>(I, vlo, vhi, I.xT, cur ? I.xb1 : I.xb0, false);
      if (!group_sync<BS>(g)) { ok = false; break; }
    } else if (method == PDHCG_INNER_BB) {
      // x and grad alternate between two buffers each: (xT, xprev) and (grad, gprev).
      // The stop test and the step length: thread 0 (FP64), shared with the CTA.
      double alpha_min = 0.0, alpha_max = 0.0;
      if (threadIdx.x == 0) {
        alpha_min = 1.0 / (S.gersh + inv_tau);
        alpha_max = 1.0 / inv_tau;
      }
      double nr = red1[0], ss = 0.0, sy = 0.0;
      int j = 0;
      VecT* xc = I.xT;
      VecT* xo = I.xprev;
      VecT* gc = I.grad;
      VecT* go = I.gprev;
      while (true) {
        if (threadIdx.x == 0) {
          sm_in[0] = (sqrt(nr) <= eps || j >= P.max_inner_iter) ? 1.0 : 0.0;
          double alpha = alpha_min;
          if (j > 0) {
            alpha = sy > 0.0 ? ss / sy : alpha_max;
            alpha = fmin(fmax(alpha, alpha_min), alpha_max);
          }
          sm_in_ct[0] = CT(alpha);
        }
        __syncthreads();
        if (sm_in[0] != 0.0) break;
        bb_phase_b<BS>(I, vlo, vhi, sm_in_ct[0], xc, gc, xo);
        { VecT* t = xo; xo = xc; xc = t; }
        PDHCG_CLK(2);
        if (!group_sync<BS>(g)) { ok = false; break; }
        if (kR && I.k > 0) {
          r_phase_x<BS, LM>(I, prank, xc, rc);
          if (!group_sync<BS>(g)) { ok = false; break; }
        }
        PDHCG_CLK(5);
        double v3[3];
        {
          const Red<3> r = bb_phase_a<BS, LM, kR>(I, prank, xc, xo, gc, go, sc.itau, rc);
          v3[0] = r.v[0];
          v3[1] = r.v[1];
          v3[2] = r.v[2];
        }
        PDHCG_CLK(1);
        if (!group_reduce<BS, 3, kWT>(g, v3, 0u)) { ok = false; break; }
        PDHCG_CLK(5);
        { VecT* t = go; go = gc; gc = t; }
        ss = v3[0];
        sy = v3[1];
        nr = v3[2];
        ++j;
      }
      if (!ok) break;
      S.inner_total += j;
      // the result must be in xT for Phase II and the checks; xbar = 2 x+ - x
      write_xbar<BS>(I, vlo, vhi, xc, cur ? I.xb1 : I.xb0, xc != I.xT);
      if (!group_sync<BS>(g)) { ok = false; break; }
    }

    // Phase II.  Slot 3 carries a group's pause decision for time slices: rank
    // 0's clock decides, and the max-reduction hands every CTA the same value.
    // (closed form: slots 4 and 5 carry Phase I's unreduced movement sums)
    double red2[6];
    {
      const Red<3> r = phase2<BS, LM>(I, prank, method, cur, vlo, vhi, sc, rc);
      red2[0] = r.v[0];
      red2[1] = r.v[1];
      red2[2] = r.v[2];
      red2[3] = (plan.slice_ns > 0 && g.nblk > 1 && g.rank == 0 && threadIdx.x == 0 &&
                 globaltimer_ns() - t_resume >= plan.slice_ns)
                    ? 1.0
                    : 0.0;
      red2[4] = method == PDHCG_INNER_DIAG ? red1[2] : 0.0;
      red2[5] = method == PDHCG_INNER_DIAG ? red1[3] : 0.0;
    }
    // the next step's scalars for k + 1 (used if this step ends without a
    // check); the reduction below orders these writes before their reads
    if (threadIdx.x >= BS - 32) {
      double it, is;
      const StepScalars<CT> nx = step_scalars<CT>(S, P, S.k + 1, it, is);
      if (threadIdx.x == BS - 32) {
        sm_sc_next = nx;
        sm_scal_next[0] = it;
        sm_scal_next[1] = is;
      }
    }
    PDHCG_CLK(3);
    if (!group_reduce<BS, 6, kWT>(g, red2, 1u << 3)) { ok = false; break; }
    PDHCG_CLK(5);
    const double dy2 = red2[0];
    const double dx2 = method == PDHCG_INNER_DIAG ? red2[4] : red2[1];
    const double mvh2 = method == PDHCG_INNER_DIAG ? red2[5] : red2[2];
    bool do_restart = false;
    const bool period_end = S.K + 1 == next_check;
    if (period_end) next_check += P.k_eval;
    const bool check = period_end || (S.K + 1 >= P.max_iter);
    next_ready = !check;

    // the step's square roots one lane each, so a warp issues one FP64 sequence
    // for all three: the fixed-point residual (Sec. 3.2) and the primal movement
    // for either outcome of the restart decision.  The closed form needs them
    // only where the restart logic reads them (the first step of a round, a
    // check): the movement feeds the inner tolerance, which it does not have.
    double fpr = 0.0, sq_dx = 0.0, sq_mvh = 0.0;
    if (method != PDHCG_INNER_DIAG || S.k == 0 || check) {
      if (threadIdx.x < 32) {  // warp 0, lane q: root q
        const int ln = threadIdx.x;
        const double sq = sqrt(ln == 0 ? S.omega * dx2 + dy2 / S.omega : ln == 1 ? dx2 : mvh2);
        if (ln < 3) sm_scal[2 + ln] = sq;
      }
      __syncthreads();
      fpr = sm_scal[2];
      sq_dx = sm_scal[3];
      sq_mvh = sm_scal[4];
    }
    if (S.k == 0) {
      S.fpr_anchor = fpr;
      S.fpr_last = fpr;
    }
    if (check) {
      double cv[18];
      if (kR && I.k > 0) {
        r_phase_check<BS, LM>(I, prank, cur, rc);
        if (!group_sync<BS>(g)) { ok = false; break; }
      }
      {
        const Red<18> r = check_phase<BS, LM, kR>(I, prank, cur, method != PDHCG_INNER_DIAG, rc);
#pragma unroll
        for (int q = 0; q < 18; ++q) cv[q] = r.v[q];
      }
      cv[17] = double(globaltimer_ns());
      // max slots: 0 1 2 3 8 10 12 13 14 17
      const unsigned mm = (1u << 0) | (1u << 1) | (1u << 2) | (1u << 3) | (1u << 8) | (1u << 10) |
                          (1u << 12) | (1u << 13) | (1u << 14) | (1u << 17);
      PDHCG_CLK(4);
      if (!group_reduce<BS, 18>(g, cv, mm)) { ok = false; break; }
      PDHCG_CLK(5);

      const int status = check_status(S, P, I.bscale, I.cinf, cv);
      if (status) {
        const double dn = cv[10];
        double mx[2] = {0.0, 0.0};
        if (status == PDHCG_PRIMAL_INFEASIBLE || status == PDHCG_DUAL_INFEASIBLE) {
          const Red<2> r = ray_norms<BS>(I, cur, vlo, vhi, clo, chi, dn);
          mx[0] = r.v[0];
          mx[1] = r.v[1];
          if (!group_reduce<BS, 2>(g, mx, 3u)) { ok = false; break; }
        }
        write_outputs<BS>(I, cur, vlo, vhi, clo, chi, status, dn, mx[0], mx[1]);
        S.status = status;
        S.K += 1;
        S.t_end_ns = cv[17];
        break;
      }

      do_restart = restart_decision(S, P, fpr, cv);
    }

    if (do_restart) {
      restart_copy<BS>(I, cur, vlo, vhi, clo, chi);
      if (!group_sync<BS>(g)) { ok = false; break; }
      PDHCG_CLK(6);
      S.mv = sq_dx;
      S.k = 0;
      S.restarts += 1;
    } else {
      S.cur ^= 1;
      S.mv = sq_mvh;
      S.k += 1;
    }
    S.K += 1;
    if (plan.iter_budget > 0 && S.K - K_first >= plan.iter_budget) break;  // paused
    if (plan.slice_ns > 0 && g.nblk > 1 && red2[3] > 0.0) break;  // paused (group, every step)
    if (plan.slice_ns > 0 && g.nblk == 1 && ((S.K - K_first) & 15) == 0) {
      if (threadIdx.x == 0) sm_pause = globaltimer_ns() - t_resume >= plan.slice_ns;
      __syncthreads();
      const bool pause = sm_pause != 0;
      __syncthreads();  // thread 0 rewrites sm_pause only after every thread has read it
      if (pause) break;  // paused
    }
  }
  if (!ok) S.device_error = 1;
  if (g.rank == 0 && threadIdx.x == 0) store_state(I.st, S);
}

// Copy an instance descriptor into the CTA's shared copy (all threads call).
template <int BS, class MatT, class VecT>
__device__ __forceinline__ void copy_inst(Inst<MatT, VecT>& dst, const Inst<MatT, VecT>& src) {
  constexpr int W4 = int(sizeof(Inst<MatT, VecT>) / 4);
  const uint32_t* s4 = reinterpret_cast<const uint32_t*>(&src);
  uint32_t* d4 = reinterpret_cast<uint32_t*>(&dst);
  __syncthreads();
  for (int i = threadIdx.x; i < W4; i += BS) d4[i] = s4[i];
  __syncthreads();
}

// Solve one pool instance with its vectors in the CTA's shared memory
// (plan.smem_vec_bytes of it).  The vectors are placed in order of how much a
// PDHG step relies on them, each while it still fits: first those the matrix
// products gather at random (y for A^T y; xbar for A xbar; with an inner solver
// also x, T(x) and its work vectors for the Q products), then the iterate and
// anchor entries every step reads, then the problem data it reads (c, bounds,
// diag Q), last T(z), which a step only writes.  A vector that does not fit
// stays in global memory, where the iteration reads and writes it in place, so
// an instance larger than the budget keeps its hottest vectors on chip and more
// CTAs fit on an SM.  Placement changes no arithmetic: the results are the same
// bits as with every vector in global memory.
template <int BS, bool kR, class MatT, class VecT, bool kDiag = false>
__device__ PDHCG_PHASE_ATTR void solve_in_smem(Group<BS>& g, const Inst<MatT, VecT>& Ig, Inst<MatT, VecT>& I,
                                           const LaunchPlan& plan, const RowCtx& rc, char* base,
                                           int method) {
  const int n = Ig.n, m = Ig.m;
  const size_t cap = size_t(plan.smem_vec_bytes);
  size_t off = 0;
  // a shared-memory slot for `count` entries like *p if one is left, else p
  auto place = [&](auto* p, int count) {
    using T = std::remove_const_t<std::remove_pointer_t<decltype(p)>>;
    const size_t bytes = (size_t(count) * sizeof(T) + 15) & ~size_t(15);
    if (off + bytes > cap) return const_cast<T*>(p);
    T* q = reinterpret_cast<T*>(base + off);
    off += bytes;
    return q;
  };
  const bool inner = method == PDHCG_INNER_CG || method == PDHCG_INNER_BB;
  // First the SELL slice offsets of the row spaces: each slice's walk starts
  // with two of them, at the head of its chain of dependent loads.
  auto place_ptr = [&](const int64_t* p, int nslices) -> const int64_t* {
    return p ? place(p, nslices + 1) : p;
  };
  const int64_t* pAT = place_ptr(Ig.ATs.ptr, Ig.vsp.nslices);
  const int64_t* pQ = inner && Ig.has_q ? place_ptr(Ig.Qs.ptr, Ig.vsp.nslices) : Ig.Qs.ptr;
  const int64_t* pA = place_ptr(Ig.As.ptr, Ig.csp.nslices);
  VecT *e0 = nullptr, *e1 = nullptr, *e2 = nullptr, *e3 = nullptr;
  VecT *xT = Ig.xT, *yT = Ig.yT;
  VecT* yb0 = place(Ig.yb0, m);
  VecT* yb1 = place(Ig.yb1, m);
  VecT *xb0, *xb1, *xbar;
  if (inner) {
    xb0 = place(Ig.xb0, n);
    xb1 = place(Ig.xb1, n);
    xT = place(Ig.xT, n);
    e0 = place(method == PDHCG_INNER_CG ? Ig.r : Ig.bv, n);
    e1 = place(method == PDHCG_INNER_CG ? Ig.p0 : Ig.grad, n);
    e2 = place(method == PDHCG_INNER_CG ? Ig.p1 : Ig.gprev, n);
    e3 = place(method == PDHCG_INNER_CG ? Ig.q : Ig.xprev, n);
    xbar = place(Ig.xbar, n);
  } else {
    xbar = place(Ig.xbar, n);
    xb0 = place(Ig.xb0, n);
    xb1 = place(Ig.xb1, n);
  }
  VecT* xa = place(Ig.xa, n);
  VecT* ya = place(Ig.ya, m);
  VecT* c = place(Ig.c, n);
  VecT* qd = place(Ig.qdiag, n);
  VecT* lv = place(Ig.lv, n);
  VecT* uv = place(Ig.uv, n);
  VecT* lc = place(Ig.lc, m);
  VecT* uc = place(Ig.uc, m);
  int8_t* vt = place(Ig.vtype, n);
  int8_t* ct = place(Ig.ctype, m);
  if (!inner) xT = place(Ig.xT, n);
  yT = place(Ig.yT, m);
  const SolverState& S0 = *Ig.st;
  const bool started = S0.started != 0;
  const int cur = S0.cur;
  VecT* xc = cur ? xb1 : xb0;
  const VecT* xcg = cur ? Ig.xb1 : Ig.xb0;
  VecT* yc = cur ? yb1 : yb0;
  const VecT* ycg = cur ? Ig.yb1 : Ig.yb0;
  // copies into the shared-memory slots only (a vector left in global memory
  // is already in place)
  auto copy_ptr = [&](const int64_t* dst, const int64_t* src, int nslices) {
    if (dst != src)
      for (int i = threadIdx.x; i <= nslices; i += BS) const_cast<int64_t*>(dst)[i] = src[i];
  };
  copy_ptr(pAT, Ig.ATs.ptr, Ig.vsp.nslices);
  copy_ptr(pQ, Ig.Qs.ptr, Ig.vsp.nslices);
  copy_ptr(pA, Ig.As.ptr, Ig.csp.nslices);
  for (int i = threadIdx.x; i < n; i += BS) {
    if (c != Ig.c) c[i] = Ig.c[i];
    if (lv != Ig.lv) lv[i] = Ig.lv[i];
    if (uv != Ig.uv) uv[i] = Ig.uv[i];
    if (qd != Ig.qdiag) qd[i] = Ig.qdiag[i];
    if (vt != Ig.vtype) vt[i] = Ig.vtype[i];
    if (started) {
      if (xc != xcg) xc[i] = xcg[i];
      if (xa != Ig.xa) xa[i] = Ig.xa[i];
    }
  }
  for (int i = threadIdx.x; i < m; i += BS) {
    if (lc != Ig.lc) lc[i] = Ig.lc[i];
    if (uc != Ig.uc) uc[i] = Ig.uc[i];
    if (ct != Ig.ctype) ct[i] = Ig.ctype[i];
    if (started) {
      if (yc != ycg) yc[i] = ycg[i];
      if (ya != Ig.ya) ya[i] = Ig.ya[i];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    I.xb0 = xb0; I.xb1 = xb1; I.xT = xT; I.xa = xa; I.xbar = xbar;
    I.c = c; I.lv = lv; I.uv = uv; I.qdiag = qd; I.vtype = vt;
    I.yb0 = yb0; I.yb1 = yb1; I.yT = yT; I.ya = ya; I.lc = lc; I.uc = uc; I.ctype = ct;
    I.ATs.ptr = pAT; I.Qs.ptr = pQ; I.As.ptr = pA;
    if (method == PDHCG_INNER_CG) {
      I.r = e0; I.p0 = e1; I.p1 = e2; I.q = e3;
    } else if (method == PDHCG_INNER_BB) {
      I.bv = e0; I.grad = e1; I.gprev = e2; I.xprev = e3;
    }
  }
  __syncthreads();
  solve_instance<BS, Ld::Cached, kR, MatT, VecT, kDiag>(g, I, plan, rc);
  __syncthreads();
  const int cur2 = Ig.st->cur;
  VecT* xf = cur2 ? xb1 : xb0;
  VecT* xfg = cur2 ? Ig.xb1 : Ig.xb0;
  VecT* yf = cur2 ? yb1 : yb0;
  VecT* yfg = cur2 ? Ig.yb1 : Ig.yb0;
  constexpr bool kLo = std::is_same<MatT, float>::value;
  for (int i = threadIdx.x; i < n; i += BS) {
    if (xf != xfg) xfg[i] = xf[i];
    if (xa != Ig.xa) Ig.xa[i] = xa[i];
    if constexpr (kLo) {
      if (c != Ig.c) Ig.c[i] = c[i];  // the defect-corrected data resumes with the iterate
    }
  }
  for (int i = threadIdx.x; i < m; i += BS) {
    if (yf != yfg) yfg[i] = yf[i];
    if (ya != Ig.ya) Ig.ya[i] = ya[i];
    if constexpr (kLo) {
      if (lc != Ig.lc) Ig.lc[i] = lc[i];
      if (uc != Ig.uc) Ig.uc[i] = uc[i];
    }
  }
}

// Register caps.  The 256-thread kernel (groups, and the default pool width)
// is compiled for 2 resident CTAs per SM: 128 registers.  The narrow 128-thread
// pool kernel is compiled for 4 per SM, also 128 registers; it pays off only
// where four instances' vectors fit on one SM.  Measured on 4,096 MPC QPs:
// with T = 20 (33 KB of vectors each) 4 CTAs per SM ran 43 % more solves per
// second than 2 with 255 registers; with the horizons mixed (up to 88 KB) the
// 256-thread CTAs ran 8 % more than 2 narrow CTAs per SM, and 17 % more with
// T = 50.
#ifndef PDHCG_MIN_BLOCKS
#define PDHCG_MIN_BLOCKS 2
#endif
#ifndef PDHCG_POOL_MIN_BLOCKS
#define PDHCG_POOL_MIN_BLOCKS 4
#endif
template <int BS, class MatT, class VecT, bool kR, bool kDiag = false>
__global__ void __launch_bounds__(BS, BS == kGroupBS ? PDHCG_MIN_BLOCKS : PDHCG_POOL_MIN_BLOCKS) solve_kernel(const Inst<MatT, VecT>* insts, LaunchPlan plan) {
  __shared__ double sm_warp[2 * (BS / 32) * kSlots];
  __shared__ double sm_tot[2 * kSlots];
  __shared__ double sm_red[(BS / 32) * kRowSums];
  extern __shared__ __align__(16) char dsm[];
  __shared__ int sm_flag;
  __shared__ int sm_idx;
  Group<BS> g;
  g.sm_warp = sm_warp;
  g.sm_tot = sm_tot;
  g.sm_flag = &sm_flag;
  g.err = plan.err;
  g.timeout_ns = plan.timeout_ns;
  g.failed = false;
  g.epoch = 0;
  if (threadIdx.x == 0) sm_flag = 0;
  __syncthreads();
  const RowCtx rc{sm_red};
  // the instance descriptor lives in shared memory (one copy per CTA)
  __shared__ __align__(16) char sh_inst_raw[sizeof(Inst<MatT, VecT>)];
  Inst<MatT, VecT>& sh_inst = *reinterpret_cast<Inst<MatT, VecT>*>(sh_inst_raw);
  if ((int)blockIdx.x < plan.group_blocks) {
    int gi = 0;
    while (gi + 1 < plan.ngroups && (int)blockIdx.x >= plan.g_first[gi + 1]) ++gi;
    g.nblk = plan.g_nblk[gi];
    g.rank = (int)blockIdx.x - plan.g_first[gi];
    g.bar32 = reinterpret_cast<unsigned*>(plan.g_bar) + size_t(gi) * kBarWords;
    g.part = plan.g_part + plan.g_part_off[gi];
    copy_inst<BS>(sh_inst, insts[plan.g_inst[gi]]);
    solve_instance<BS, Ld::Stream, kR>(g, sh_inst, plan, rc);
    return;
  }
  g.nblk = 1;
  g.rank = 0;
  g.bar32 = nullptr;
  g.part = nullptr;
  if (plan.npool <= 0) return;  // a launch of groups only
  while (true) {
    if (threadIdx.x == 0) sm_idx = atomicAdd(plan.pool_next, 1);
    __syncthreads();
    const int idx = sm_idx;
    __syncthreads();
    if (idx >= plan.npool) break;
    g.epoch = 0;
    const Inst<MatT, VecT>& Ig = insts[plan.pool_inst[idx]];
    const int method = Ig.st->method;
    copy_inst<BS>(sh_inst, Ig);
    if (plan.smem_vec_bytes > 0 && Ig.st->status == 0) {
      solve_in_smem<BS, kR, MatT, VecT, kDiag>(g, Ig, sh_inst, plan, rc, dsm, method);
    } else {
      solve_instance<BS, Ld::Cached, kR, MatT, VecT, kDiag>(g, sh_inst, plan, rc);
    }
    __syncthreads();
  }
}

}  // namespace pdhcg

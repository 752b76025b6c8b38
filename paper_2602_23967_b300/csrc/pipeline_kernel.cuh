// pipeline_kernel.cuh — one large instance as a CUDA graph of ordinary kernels.
//
// The persistent group kernel holds every phase of the iteration in one
// launch, so its register allocation is the largest phase's and only two CTAs
// of 256 threads fit on an SM: 16 warps to hide the dependent loads of the
// row phases (column index -> gather).  Here each phase is a kernel of its
// own, compiled for four resident CTAs per SM, and a graph with device-driven
// conditional nodes runs the method:
//
//   init
//   while (outer):                                 one PDHG step per pass
//     phase1                                       A^T y, prox RHS, inner start
//     while (inner): cg_a, cg_b  |  bb_b, bb_a     the inner solver (Sec. 2.2)
//     xbar                                         x+ into place, xbar = 2 x+ - x
//     phase2                                       A xbar, dual step, Halpern
//     if (check): check                            KKT, infeasibility, restart
//                 if (restart): restart
//                 if (out): rays, write
//
// The phase functions are the persistent kernel's (solve_kernel.cuh).  Each
// kernel's CTAs write their partial sums to global memory; the last CTA to
// finish (an atomic ticket after a fence) sums them in the fixed order that
// group_reduce uses, takes the scalar decisions of solve_instance() on the
// state in global memory, and sets the graph's conditions.  With the same
// number of CTAs and the same row partition, results equal the persistent
// group kernel's bit for bit.
#pragma once
#include "launch.h"
#include "solve_kernel.cuh"

namespace pdhcg {

constexpr int kPipeBS = 256;
#ifndef PDHCG_PIPE_MIN_BLOCKS
#define PDHCG_PIPE_MIN_BLOCKS 4
#endif

// Conditions of the graph, set from the device.
struct PipeHandles {
  cudaGraphConditionalHandle outer, inner, check, restart, out;
};

// Scalars handed from one kernel of the pipeline to the next.
struct PipeState {
  // device-timer profile of the kernels when built with PDHCG_PIPE_TIMERS=1
  // (kind k: first CTA start to last CTA end summed in ns_busy[k], launches in
  // count[k]; ns_gap: time between one kernel's end and the next one's start;
  // neg_first[k]: bitwise complement of the earliest start, so zero is empty)
  unsigned long long neg_first[12], ns_busy[12], count[12], t_last_end, ns_gap;
  unsigned timer_ticket[12];
  double red1[4];
  double eps;                  // inner tolerance of this step
  double rr, beta, alpha;      // CG
  double ss, sy, nr;           // BB
  double dx2, mvh2, fpr;       // from Phase II
  double cv[18];               // check totals
  double mx[2];                // ray norms
  int32_t j, pc, bsel, brk, status, pad;
  unsigned ticket[8];          // last-CTA counters, one per kernel kind (reset by the last CTA)
  // Scalars of the current step (PipeScalar slots), each set once by the one
  // thread that takes the decisions and read by every CTA of the next kernels:
  // the FP64 value and its double-float split (hi also being the FP32 value).
  double sd[12];
  float shi[12], slo[12];
};

static_assert(sizeof(PipeState) <= kPipeStateBytes, "pipeline state buffer too small");

// The step scalars of the persistent kernel's step_scalars() (the first seven,
// in its order), the inner solvers' step lengths, and 1/tau, 1/sigma in FP64.
// Computing them once instead of in every thread of every CTA keeps the
// kernels' prologues off the narrow FP64 pipe.
enum PipeScalar : int { kPsItau, kPsIsig, kPsSig, kPsWk, kPsAk, kPsTh, kPsTh1, kPsAlpha, kPsBeta, kPsInvTau, kPsInvSigma };

__device__ __forceinline__ void pipe_set(PipeState& P, int k, double v) {
  const dfloat d(v);  // the conversion VecT(v) makes for double-float and FP32 vectors
  P.sd[k] = v;
  P.shi[k] = d.hi;
  P.slo[k] = d.lo;
}
template <class VecT>
__device__ __forceinline__ VecT pipe_get(const PipeState& P, int k) {
  if constexpr (std::is_same<VecT, dfloat>::value) return dfloat(P.shi[k], P.slo[k]);
  else if constexpr (std::is_same<VecT, float>::value) return P.shi[k];
  else return P.sd[k];
}
template <class VecT>
__device__ __forceinline__ StepScalars<VecT> pipe_step_scalars(const PipeState& P) {
  StepScalars<VecT> sc;
  sc.itau = pipe_get<VecT>(P, kPsItau);
  sc.isig = pipe_get<VecT>(P, kPsIsig);
  sc.sig = pipe_get<VecT>(P, kPsSig);
  sc.wk = pipe_get<VecT>(P, kPsWk);
  sc.ak = pipe_get<VecT>(P, kPsAk);
  sc.th = pipe_get<VecT>(P, kPsTh);
  sc.th1 = pipe_get<VecT>(P, kPsTh1);
  return sc;
}
// The quotients step_scalars() takes, one by one (the same IEEE results).
__device__ __forceinline__ void pipe_set_step(PipeState& P, const SolverState& S, const DevParams& prm) {
  const double kp2 = double(S.k + 2);
  pipe_set(P, kPsItau, 1.0 / S.tau);
  pipe_set(P, kPsIsig, 1.0 / S.sigma);
  pipe_set(P, kPsSig, S.sigma / 1.0);
  pipe_set(P, kPsWk, double(S.k + 1) / kp2);
  pipe_set(P, kPsAk, 1.0 / kp2);
  pipe_set(P, kPsTh, prm.theta / 1.0);
  pipe_set(P, kPsTh1, (1.0 + prm.theta) / 1.0);
  P.sd[kPsInvTau] = P.sd[kPsItau];
  P.sd[kPsInvSigma] = P.sd[kPsIsig];
}
// The BB step length of inner step j (j = 0: the lower bound of its range).
__device__ __forceinline__ void pipe_set_bb_alpha(PipeState& P, const SolverState& S, int j, double ss, double sy) {
  const double inv_tau = 1.0 / S.tau;
  const double alpha_min = 1.0 / (S.gersh + inv_tau), alpha_max = 1.0 / inv_tau;
  double alpha = alpha_min;
  if (j > 0) {
    alpha = sy > 0.0 ? ss / sy : alpha_max;
    alpha = fmin(fmax(alpha, alpha_min), alpha_max);
  }
  pipe_set(P, kPsAlpha, alpha);
}

struct PipeArgs {
  const void* inst;  // the instance descriptor, Inst<MatT, VecT> (device)
  PipeState* ps;
  double* part;      // partial sums: slot j of CTA b at part[j * G + b]
  PipeHandles h;
};

// Shared memory of a pipeline kernel.
template <class MatT, class VecT>
struct PipeShared {
  alignas(16) char inst[sizeof(Inst<MatT, VecT>)];
  double warp[(kPipeBS / 32) * kSlots];
  double tot[kSlots];
  double red[(kPipeBS / 32) * kRowSums];
  int last;
};

template <class MatT, class VecT>
__device__ __forceinline__ const Inst<MatT, VecT>& pipe_inst(const PipeArgs& a, PipeShared<MatT, VecT>& sh) {
  Inst<MatT, VecT>& I = *reinterpret_cast<Inst<MatT, VecT>*>(sh.inst);
  copy_inst<kPipeBS>(I, *static_cast<const Inst<MatT, VecT>*>(a.inst));
  return I;
}

// This CTA's partial of NV values (bit j of maxmask: max instead of sum) to
// part; returns true in every thread of the last CTA to get here, which then
// holds the totals in v (fixed order: CTAs lane-strided, lanes, warps).
template <int NV, bool kWT, class Sh>
__device__ __forceinline__ bool pipe_reduce(double (&v)[NV], unsigned maxmask, double* part, unsigned* ticket,
                                            Sh& sh) {
  constexpr int W = kPipeBS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = int(gridDim.x), b = int(blockIdx.x);
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double t = v[j];
    if constexpr (!kWT) {
      const bool mx = (maxmask >> j) & 1u;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double o = __shfl_xor_sync(kFull, t, off);
        t = mx ? fmax(t, o) : t + o;
      }
    }
    if (lane == 0) sh.warp[warp * kSlots + j] = t;
  }
  __syncthreads();
  if (warp == 0 && lane < NV) {
    const bool mx = (maxmask >> lane) & 1u;
    double bp = 0.0;
    for (int w = 0; w < W; ++w) {
      const double o = sh.warp[w * kSlots + lane];
      bp = mx ? fmax(bp, o) : bp + o;
    }
    part[size_t(lane) * G + b] = bp;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) sh.last = atomicAdd(ticket, 1u) == unsigned(G - 1);
  __syncthreads();
  if (!sh.last) return false;
  __threadfence();
  double t[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) t[j] = 0.0;
  for (int c = threadIdx.x; c < G; c += kPipeBS) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      const double o = __ldcg(part + size_t(j) * G + c);
      t[j] = ((maxmask >> j) & 1u) ? fmax(t[j], o) : t[j] + o;
    }
  }
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const bool mx = (maxmask >> j) & 1u;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_xor_sync(kFull, t[j], off);
      t[j] = mx ? fmax(t[j], o) : t[j] + o;
    }
  }
  __syncthreads();  // sh.warp is reused
#pragma unroll
  for (int j = 0; j < NV; ++j)
    if (lane == 0) sh.warp[warp * kSlots + j] = t[j];
  __syncthreads();
  if (warp == 0 && lane < NV) {
    const bool mx = (maxmask >> lane) & 1u;
    double a = 0.0;
    for (int w = 0; w < W; ++w) {
      const double o = sh.warp[w * kSlots + lane];
      a = mx ? fmax(a, o) : a + o;
    }
    sh.tot[lane] = a;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = sh.tot[j];
  if (threadIdx.x == 0) *ticket = 0u;  // the next launch of this kernel starts again at 0
  return true;
}

// Element ranges of this CTA in the even splits of [0, n) and [0, m).
template <class MatT, class VecT>
__device__ __forceinline__ void pipe_ranges(const Inst<MatT, VecT>& I, int& vlo, int& vhi, int& clo, int& chi) {
  const int r = int(blockIdx.x);
  vlo = I.var_part[r];
  vhi = I.var_part[r + 1];
  clo = I.con_part[r];
  chi = I.con_part[r + 1];
}

#ifndef PDHCG_PIPE_TIMERS
#define PDHCG_PIPE_TIMERS 0
#endif
// Kernel timing (PDHCG_PIPE_TIMERS=1 only): every CTA marks its start; the
// last CTA to finish closes the interval of this launch.
struct PipeTimer {
  PipeState* ps;
  int kind;
  __device__ __forceinline__ PipeTimer(PipeState* p, int k) : ps(p), kind(k) {
    if (PDHCG_PIPE_TIMERS && threadIdx.x == 0) atomicMax(&ps->neg_first[kind], ~globaltimer_ns());
  }
  __device__ __forceinline__ ~PipeTimer() {
    if (PDHCG_PIPE_TIMERS && threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(&ps->timer_ticket[kind], 1u) == gridDim.x - 1) {
        const unsigned long long t = globaltimer_ns(), t0 = ~atomicAdd(&ps->neg_first[kind], 0ull);
        ps->ns_busy[kind] += t - t0;
        ps->count[kind] += 1;
        if (ps->t_last_end) ps->ns_gap += t0 > ps->t_last_end ? t0 - ps->t_last_end : 0ull;
        ps->t_last_end = t;
        ps->neg_first[kind] = 0ull;
        ps->timer_ticket[kind] = 0u;
      }
    }
  }
};

#define PDHCG_PIPE_KERNEL template <class MatT, class VecT> __global__ void __launch_bounds__(kPipeBS, PDHCG_PIPE_MIN_BLOCKS)

// ---- init: the starting point (warm start or proj_X(0), 0) and the clock ----
PDHCG_PIPE_KERNEL pipe_init(PipeArgs a) {
  const PipeTimer timer(a.ps, 0);
  __shared__ PipeShared<MatT, VecT> sh;
  const Inst<MatT, VecT>& I = pipe_inst(a, sh);
  int vlo, vhi, clo, chi;
  pipe_ranges(I, vlo, vhi, clo, chi);
  init_point<kPipeBS>(I, vlo, vhi, clo, chi);
  double t[1] = {double(globaltimer_ns())};
  if (pipe_reduce<1, false>(t, 1u, a.part, &a.ps->ticket[0], sh) && threadIdx.x == 0) {
    SolverState& S = *I.st;
    S.t_start_ns = t[0];
    S.started = 1;
    S.cur = 0;
    S.form = 2;
    pipe_set_step(*a.ps, S, I.prm);
  }
}

// ---- Phase I and the start of the inner solve ----
PDHCG_PIPE_KERNEL pipe_phase1(PipeArgs a) {
  const PipeTimer timer(a.ps, 1);
  __shared__ PipeShared<MatT, VecT> sh;
  constexpr bool kWT = WarpTotals<VecT>::value;
  const Inst<MatT, VecT>& I = pipe_inst(a, sh);
  const RowCtx rc{sh.red};
  const SolverState& Sg = *I.st;  // read here; written only by the last CTA below
  const int method = Sg.method;
  const StepScalars<VecT> sc = pipe_step_scalars<VecT>(*a.ps);
  double v[4];
  {
    const Red<4> r = phase1<kPipeBS, Ld::Stream, false>(I, int(blockIdx.x), method, Sg.cur, sc, rc);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = r.v[q];
  }
  if (!pipe_reduce<4, kWT>(v, 0u, a.part, &a.ps->ticket[1], sh) || threadIdx.x != 0) return;
  PipeState& P = *a.ps;
  SolverState S = *I.st;
  const double eps = inner_tolerance<VecT>(S, I.prm, method, v[1], P.sd[kPsInvTau]);
  I.st->eps_in = S.eps_in;
#pragma unroll
  for (int q = 0; q < 4; ++q) P.red1[q] = v[q];
  P.eps = eps;
  P.j = 0;
  P.pc = 0;
  P.bsel = 0;
  P.brk = 0;
  P.beta = 0.0;
  pipe_set(P, kPsBeta, 0.0);
  pipe_set_bb_alpha(P, S, 0, 0.0, 0.0);
  P.rr = v[0];
  P.nr = v[0];
  P.ss = P.sy = 0.0;
  const bool go = method != PDHCG_INNER_DIAG && !(sqrt(v[0]) <= eps || 0 >= I.prm.max_inner_iter);
  cudaGraphSetConditional(a.h.inner, go ? 1u : 0u);
}

// ---- CG Phase A: p = r + beta p_old, q = H p, p^T q ----
PDHCG_PIPE_KERNEL pipe_cg_a(PipeArgs a) {
  const PipeTimer timer(a.ps, 2);
  __shared__ PipeShared<MatT, VecT> sh;
  constexpr bool kWT = WarpTotals<VecT>::value;
  const Inst<MatT, VecT>& I = pipe_inst(a, sh);
  const RowCtx rc{sh.red};
  const PipeState& P = *a.ps;
  const int j = P.j, pc = P.pc;
  const VecT* pold = pc ? I.p1 : I.p0;
  VecT* pnew = pc ? I.p0 : I.p1;
  const VecT itau = pipe_get<VecT>(P, kPsItau);
  const VecT beta = pipe_get<VecT>(P, kPsBeta);
  double v[1] = {cg_phase_a<kPipeBS, Ld::Stream, false>(I, int(blockIdx.x), j == 0, beta, pold, pnew, itau, rc)};
  if (!pipe_reduce<1, kWT>(v, 0u, a.part, &a.ps->ticket[2], sh) || threadIdx.x != 0) return;
  PipeState& Pw = *a.ps;
  if (!(v[0] > 0.0)) {
    Pw.brk = 1;
    cudaGraphSetConditional(a.h.inner, 0u);
  } else {
    Pw.alpha = Pw.rr / v[0];
    pipe_set(Pw, kPsAlpha, Pw.alpha);
  }
}

// ---- CG Phase B: x += alpha p, r -= alpha q, r^T r, next beta ----
PDHCG_PIPE_KERNEL pipe_cg_b(PipeArgs a) {
  const PipeTimer timer(a.ps, 3);
  __shared__ PipeShared<MatT, VecT> sh;
  constexpr bool kWT = WarpTotals<VecT>::value;
  const PipeState& P = *a.ps;
  if (P.brk) return;
  const Inst<MatT, VecT>& I = pipe_inst(a, sh);
  int vlo, vhi, clo, chi;
  pipe_ranges(I, vlo, vhi, clo, chi);
  const VecT* pnew = P.pc ? I.p0 : I.p1;
  double v[1] = {cg_phase_b<kPipeBS>(I, vlo, vhi, pipe_get<VecT>(P, kPsAlpha), pnew)};
  if (!pipe_reduce<1, kWT>(v, 0u, a.part, &a.ps->ticket[3], sh) || threadIdx.x != 0) return;
  PipeState& Pw = *a.ps;
  Pw.beta = v[0] / Pw.rr;
  pipe_set(Pw, kPsBeta, Pw.beta);
  Pw.rr = v[0];
  Pw.pc ^= 1;
  Pw.j += 1;
  const bool go = !(sqrt(Pw.rr) <= Pw.eps || Pw.j >= I.prm.max_inner_iter);
  cudaGraphSetConditional(a.h.inner, go ? 1u : 0u);
}

// BB buffers of the current inner step: x and gradient alternate between two
// buffers each, (xT, xprev) and (grad, gprev), in step with bsel.
template <class MatT, class VecT>
struct BBBufs {
  VecT *xc, *xo, *gc, *go;
};
template <class MatT, class VecT>
__device__ __forceinline__ BBBufs<MatT, VecT> bb_bufs(const Inst<MatT, VecT>& I, int bsel) {
  return bsel ? BBBufs<MatT, VecT>{I.xprev, I.xT, I.gprev, I.grad} : BBBufs<MatT, VecT>{I.xT, I.xprev, I.grad, I.gprev};
}

// ---- BB Phase B': projected step x_o = proj(x_c - alpha g_c) ----
PDHCG_PIPE_KERNEL pipe_bb_b(PipeArgs a) {
  const PipeTimer timer(a.ps, 4);
  __shared__ PipeShared<MatT, VecT> sh;
  const Inst<MatT, VecT>& I = pipe_inst(a, sh);
  int vlo, vhi, clo, chi;
  pipe_ranges(I, vlo, vhi, clo, chi);
  const PipeState& P = *a.ps;
  const BBBufs<MatT, VecT> b = bb_bufs(I, P.bsel);
  bb_phase_b<kPipeBS>(I, vlo, vhi, pipe_get<VecT>(P, kPsAlpha), b.xc, b.gc, b.xo);
}

// ---- BB Phase A': gradient at the new x, BB quantities, natural residual ----
PDHCG_PIPE_KERNEL pipe_bb_a(PipeArgs a) {
  const PipeTimer timer(a.ps, 5);
  __shared__ PipeShared<MatT, VecT> sh;
  constexpr bool kWT = WarpTotals<VecT>::value;
  const Inst<MatT, VecT>& I = pipe_inst(a, sh);
  const RowCtx rc{sh.red};
  const PipeState& P = *a.ps;
  const BBBufs<MatT, VecT> b = bb_bufs(I, P.bsel);
  const VecT itau = pipe_get<VecT>(P, kPsItau);
  double v[3];
  {
    // the new x is in b.xo (written by pipe_bb_b), the old one in b.xc
    const Red<3> r = bb_phase_a<kPipeBS, Ld::Stream, false>(I, int(blockIdx.x), b.xo, b.xc, b.gc, b.go, itau, rc);
    v[0] = r.v[0];
    v[1] = r.v[1];
    v[2] = r.v[2];
  }
  if (!pipe_reduce<3, kWT>(v, 0u, a.part, &a.ps->ticket[4], sh) || threadIdx.x != 0) return;
  PipeState& Pw = *a.ps;
  Pw.ss = v[0];
  Pw.sy = v[1];
  Pw.nr = v[2];
  Pw.bsel ^= 1;
  Pw.j += 1;
  pipe_set_bb_alpha(Pw, *I.st, Pw.j, Pw.ss, Pw.sy);
  const bool go = !(sqrt(Pw.nr) <= Pw.eps || Pw.j >= I.prm.max_inner_iter);
  cudaGraphSetConditional(a.h.inner, go ? 1u : 0u);
}

// ---- x+ into xT, xbar = 2 x+ - x (after CG / BB; the closed form wrote both) ----
PDHCG_PIPE_KERNEL pipe_xbar(PipeArgs a) {
  const PipeTimer timer(a.ps, 6);
  __shared__ PipeShared<MatT, VecT> sh;
  const Inst<MatT, VecT>& I = pipe_inst(a, sh);
  int vlo, vhi, clo, chi;
  pipe_ranges(I, vlo, vhi, clo, chi);
  const PipeState& P = *a.ps;
  SolverState* St = I.st;
  const int method = St->method, cur = St->cur;
  const VecT* x = cur ? I.xb1 : I.xb0;
  if (method == PDHCG_INNER_CG) {
    write_xbar<kPipeBS>(I, vlo, vhi, I.xT, x, false);
  } else if (method == PDHCG_INNER_BB) {
    const VecT* xc = bb_bufs(I, P.bsel).xc;
    write_xbar<kPipeBS>(I, vlo, vhi, xc, x, xc != I.xT);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) St->inner_total += P.j;
}

// ---- Phase II and the step's bookkeeping when no check follows ----
PDHCG_PIPE_KERNEL pipe_phase2(PipeArgs a) {
  const PipeTimer timer(a.ps, 7);
  __shared__ PipeShared<MatT, VecT> sh;
  constexpr bool kWT = WarpTotals<VecT>::value;
  const Inst<MatT, VecT>& I = pipe_inst(a, sh);
  const RowCtx rc{sh.red};
  int vlo, vhi, clo, chi;
  pipe_ranges(I, vlo, vhi, clo, chi);
  const SolverState& Sg = *I.st;  // read here; written only by the last CTA below
  const int method = Sg.method;
  const StepScalars<VecT> sc = pipe_step_scalars<VecT>(*a.ps);
  double v[3];
  {
    const Red<3> r = phase2<kPipeBS, Ld::Stream>(I, int(blockIdx.x), method, Sg.cur, vlo, vhi, sc, rc);
    v[0] = r.v[0];
    v[1] = r.v[1];
    v[2] = r.v[2];
  }
  if (!pipe_reduce<3, kWT>(v, 0u, a.part, &a.ps->ticket[5], sh) || threadIdx.x != 0) return;
  PipeState& P = *a.ps;
  SolverState S = *I.st;
  const DevParams& Pr = I.prm;
  const double dy2 = v[0];
  const double dx2 = method == PDHCG_INNER_DIAG ? P.red1[2] : v[1];
  const double mvh2 = method == PDHCG_INNER_DIAG ? P.red1[3] : v[2];
  const double fpr = sqrt(S.omega * dx2 + dy2 / S.omega);
  if (S.k == 0) {
    S.fpr_anchor = fpr;
    S.fpr_last = fpr;
  }
  P.dx2 = dx2;
  P.mvh2 = mvh2;
  P.fpr = fpr;
  const bool check = ((S.K + 1) % Pr.k_eval == 0) || (S.K + 1 >= Pr.max_iter);
  if (!check) {
    S.cur ^= 1;
    S.mv = sqrt(mvh2);
    S.k += 1;
    S.K += 1;
    pipe_set_step(P, S, Pr);
  }
  *I.st = S;
  cudaGraphSetConditional(a.h.check, check ? 1u : 0u);
  cudaGraphSetConditional(a.h.restart, 0u);
  cudaGraphSetConditional(a.h.out, 0u);
}

// ---- the check: KKT (Sec. 4.2), infeasibility (Sec. 5), restart and PID ----
PDHCG_PIPE_KERNEL pipe_check(PipeArgs a) {
  const PipeTimer timer(a.ps, 8);
  __shared__ PipeShared<MatT, VecT> sh;
  const Inst<MatT, VecT>& I = pipe_inst(a, sh);
  const RowCtx rc{sh.red};
  const SolverState& S0 = *I.st;
  const int method = S0.method, cur = S0.cur;
  double cv[18];
  {
    const Red<18> r = check_phase<kPipeBS, Ld::Stream, false>(I, int(blockIdx.x), cur, method != PDHCG_INNER_DIAG, rc);
#pragma unroll
    for (int q = 0; q < 18; ++q) cv[q] = r.v[q];
  }
  cv[17] = double(globaltimer_ns());
  const unsigned mm = (1u << 0) | (1u << 1) | (1u << 2) | (1u << 3) | (1u << 8) | (1u << 10) | (1u << 12) |
                      (1u << 13) | (1u << 14) | (1u << 17);
  if (!pipe_reduce<18, false>(cv, mm, a.part, &a.ps->ticket[6], sh) || threadIdx.x != 0) return;
  PipeState& P = *a.ps;
  SolverState S = *I.st;
#pragma unroll
  for (int q = 0; q < 18; ++q) P.cv[q] = cv[q];
  const int status = check_status(S, I.prm, I.bscale, I.cinf, cv);
  P.status = status;
  bool restart = false;
  if (!status) {
    restart = restart_decision(S, I.prm, P.fpr, cv);
    if (restart) {
      S.mv = sqrt(P.dx2);
      S.k = 0;
      S.restarts += 1;
    } else {
      S.cur ^= 1;
      S.mv = sqrt(P.mvh2);
      S.k += 1;
    }
    S.K += 1;
    pipe_set_step(P, S, I.prm);
  }
  *I.st = S;
  cudaGraphSetConditional(a.h.restart, restart ? 1u : 0u);
  cudaGraphSetConditional(a.h.out, status ? 1u : 0u);
  cudaGraphSetConditional(a.h.outer, status ? 0u : 1u);
}

// ---- restart: new anchor and iterate T(z) (the current buffer, S.cur unchanged) ----
PDHCG_PIPE_KERNEL pipe_restart(PipeArgs a) {
  const PipeTimer timer(a.ps, 9);
  __shared__ PipeShared<MatT, VecT> sh;
  const Inst<MatT, VecT>& I = pipe_inst(a, sh);
  int vlo, vhi, clo, chi;
  pipe_ranges(I, vlo, vhi, clo, chi);
  restart_copy<kPipeBS>(I, I.st->cur, vlo, vhi, clo, chi);
}

// ---- output: norms of the infeasibility rays ----
PDHCG_PIPE_KERNEL pipe_rays(PipeArgs a) {
  const PipeTimer timer(a.ps, 10);
  __shared__ PipeShared<MatT, VecT> sh;
  const Inst<MatT, VecT>& I = pipe_inst(a, sh);
  int vlo, vhi, clo, chi;
  pipe_ranges(I, vlo, vhi, clo, chi);
  const PipeState& P = *a.ps;
  const int status = P.status;
  double mx[2] = {0.0, 0.0};
  if (status == PDHCG_PRIMAL_INFEASIBLE || status == PDHCG_DUAL_INFEASIBLE) {
    const Red<2> r = ray_norms<kPipeBS>(I, I.st->cur, vlo, vhi, clo, chi, P.cv[10]);
    mx[0] = r.v[0];
    mx[1] = r.v[1];
  }
  if (pipe_reduce<2, false>(mx, 3u, a.part, &a.ps->ticket[7], sh) && threadIdx.x == 0) {
    a.ps->mx[0] = mx[0];
    a.ps->mx[1] = mx[1];
  }
}

// ---- output: unscaled solution or normalised rays, and the final state ----
PDHCG_PIPE_KERNEL pipe_write(PipeArgs a) {
  const PipeTimer timer(a.ps, 11);
  __shared__ PipeShared<MatT, VecT> sh;
  const Inst<MatT, VecT>& I = pipe_inst(a, sh);
  int vlo, vhi, clo, chi;
  pipe_ranges(I, vlo, vhi, clo, chi);
  const PipeState& P = *a.ps;
  write_outputs<kPipeBS>(I, I.st->cur, vlo, vhi, clo, chi, P.status, P.cv[10], P.mx[0], P.mx[1]);
  // every CTA has read the state above before the launch's last CTA changes it
  double z[1] = {0.0};
  if (pipe_reduce<1, false>(z, 0u, a.part, &a.ps->ticket[0], sh) && threadIdx.x == 0) {
    SolverState& S = *I.st;
    S.status = P.status;
    S.K += 1;
    S.t_end_ns = P.cv[17];
  }
}

#undef PDHCG_PIPE_KERNEL

}  // namespace pdhcg

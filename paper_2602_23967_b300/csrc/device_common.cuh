// device_common.cuh — CTA-group machinery shared by the setup and solve kernels.
//
// A "group" is the set of CTAs that work on one instance: either one CTA
// (batched small instances) or several co-resident CTAs of a cooperative
// launch (one large instance).  The same phase code runs on both: rows of a
// phase are split over the group's CTAs, and every phase ends in
// group_reduce(), which is both the group barrier and a deterministic
// reduction of up to kSlots FP64 values.  Every CTA sums the per-CTA partials
// in the same fixed order, so every CTA holds bitwise identical totals and
// takes identical scalar decisions without further communication.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "dfloat.cuh"
#include "pdhcg_internal.h"

namespace pdhcg {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bulk prefetch of [src, src + bytes) into L2 (no completion to wait for).
// src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Streaming loads of matrix data that is read-only for the whole kernel: keep it
// out of L1 and mark it evict-first in L2 so the (re-read) vectors stay resident.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ int ld_stream(const int* p) {
  int v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;"
               : "=r"(v) : "l"(p), "l"(l2_evict_first_policy()));
  return v;
}
__device__ __forceinline__ float ld_stream(const float* p) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;"
               : "=f"(v) : "l"(p), "l"(l2_evict_first_policy()));
  return v;
}
__device__ __forceinline__ double ld_stream(const double* p) {
  double v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;"
               : "=d"(v) : "l"(p), "l"(l2_evict_first_policy()));
  return v;
}

// Read-only loads through L1 (small instances solved by one CTA re-read their
// whole matrix every step; it stays in L1).
template <bool kStream, class T>
__device__ __forceinline__ T ld_mat(const T* p) {
  if constexpr (kStream) return ld_stream(p);
  else return __ldg(p);
}

template <class T>
__device__ __forceinline__ T clampv(T v, T lo, T hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// Sign cone Y_i of the dual (Sec. 2): {0} free row, R+ upper-only, R- lower-only, R boxed.
__device__ __forceinline__ double proj_Y(double v, int8_t t) {
  switch (t) {
    case kFree: return 0.0;
    case kUpOnly: return fmax(v, 0.0);
    case kLowOnly: return fmin(v, 0.0);
    default: return v;
  }
}
// Sign cone R_j of the reduced cost (Sec. 2): {0} free, R- upper-only, R+ lower-only, R boxed.
__device__ __forceinline__ double proj_R(double v, int8_t t) {
  switch (t) {
    case kFree: return 0.0;
    case kUpOnly: return fmin(v, 0.0);
    case kLowOnly: return fmax(v, 0.0);
    default: return v;
  }
}
// Recession cone of a box (Sec. 5.2): {0} boxed, R+ lower-only, R- upper-only, R free.
__device__ __forceinline__ double proj_recc(double d, int8_t t) {
  switch (t) {
    case kBoxed: return 0.0;
    case kLowOnly: return fmax(d, 0.0);
    case kUpOnly: return fmin(d, 0.0);
    default: return d;
  }
}
// One term of p(z; l, u) = u^T z^+ - l^T z^- (Sec. 2); zero z contributes 0.
__device__ __forceinline__ double support_term(double z, double lo, double hi) {
  if (z > 0.0) return hi * z;
  if (z < 0.0) return lo * z;
  return 0.0;
}

template <int BS>
struct Group {
  static constexpr int kWarps = BS / 32;
  int nblk;                     // CTAs in the group
  int rank;                     // this CTA's rank
  unsigned* bar32;              // hierarchical barrier block (multi-CTA only, kBarWords)
  unsigned long long epoch;     // barriers passed
  double* part;                 // 2 * kSlots * nblk partials (multi-CTA only)
  double* sm_warp;              // shared [2][kWarps][kSlots]
  double* sm_tot;               // shared [2][kSlots]
  int* sm_flag;                 // shared
  int* err;
  uint64_t timeout_ns;
  bool failed;
  double* lz = nullptr;         // shared Lanczos coefficients (setup kernels only)
  double* red = nullptr;        // shared BS/32 * 4 doubles for the row engine (setup kernels only)
  double* lz_out = nullptr;     // shared: the warp-computed eigenvalue

  // Row range of this CTA in a space whose partition table is `part`
  // (nblk+1 offsets), or the whole space for a single-CTA group.
  __device__ __forceinline__ void range(const int32_t* part_tab, int nrows, int& lo,
                                        int& hi) const {
    if (nblk == 1 || part_tab == nullptr) {
      lo = 0;
      hi = nrows;
    } else {
      lo = part_tab[rank];
      hi = part_tab[rank + 1];
    }
  }
};

// Bounded spin until *addr >= target.  Returns false after timeout_ns or when
// another CTA reported an error.
__device__ __forceinline__ bool spin_geq(const unsigned long long* addr, unsigned long long target,
                                         uint64_t timeout_ns, const int* err) {
  uint64_t t0 = 0;
  unsigned it = 0;
  while (ld_acquire_u64(addr) < target) {
    if ((++it & 255u) == 0u) {
      uint64_t t = globaltimer_ns();
      if (t0 == 0) t0 = t;
      if (t - t0 > timeout_ns) return false;
      if (ld_relaxed_s32(err) != 0) return false;
    }
  }
  return true;
}

// ---- hierarchical group barrier ----
// Layout of a group's barrier block (zeroed before the launch), 128-byte lines:
// line k < kBarSub: arrival counter of sub-group k (CTAs with rank % nsub == k);
// line kBarSub: top-level counter; line kBarSub + 1: generation (epochs completed).
constexpr int kBarSub = 32;
constexpr int kBarLineWords = 32;  // 128 bytes of unsigned
constexpr int kBarWords = (kBarSub + 2) * kBarLineWords;

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Arrive (thread 0 of each CTA) and wait until all nblk CTAs arrived at epoch
// `epoch` (0-based).  acq_rel atomics chain every CTA's prior writes to the last
// arriver, whose release of the generation word publishes them to all waiters.
__device__ __forceinline__ bool group_arrive_wait(unsigned* bar, int rank, int nblk,
                                                  unsigned long long epoch, uint64_t timeout_ns,
                                                  const int* err) {
  const int nsub = nblk < kBarSub ? nblk : kBarSub;
  const int sub = rank % nsub;
  const unsigned sub_size = unsigned((nblk - sub + nsub - 1) / nsub);
  unsigned* cnt = bar + sub * kBarLineWords;
  unsigned* top = bar + kBarSub * kBarLineWords;
  unsigned* gen = bar + (kBarSub + 1) * kBarLineWords;
  const unsigned target = unsigned(epoch + 1ull);
  if (atom_add_acq_rel(cnt, 1u) == sub_size - 1u) {
    *cnt = 0u;  // ordered before the release below; reused only after the next generation
    if (atom_add_acq_rel(top, 1u) == unsigned(nsub) - 1u) {
      *top = 0u;
      st_release_u32(gen, target);
      return true;
    }
  }
  uint64_t t0 = 0;
  unsigned ns = 32;
  for (unsigned it = 0;; ++it) {
    if (int(ld_acquire_u32(gen) - target) >= 0) return true;
    if ((it & 15u) == 15u) {
      const uint64_t t = globaltimer_ns();
      if (t0 == 0) t0 = t;
      else if (t - t0 > timeout_ns) return false;
      if (ld_relaxed_s32(err) != 0) return false;
    }
    __nanosleep(ns);
    if (ns < 256) ns <<= 1;
  }
}

// End of a phase: barrier over the group plus a reduction of NV values.  Bit j
// of maxmask selects max (values must be >= 0) instead of sum for v[j].
// On return every thread of every CTA of the group holds the totals in v.
// Returns false if a bounded wait gave up (the caller must leave the solve).
//
// Per-warp partials go to shared memory (double-buffered by barrier parity).  A
// single CTA then reduces them in every warp after one __syncthreads.  With
// several CTAs, warp 0 publishes the CTA partial and thread 0 passes the
// hierarchical barrier; warp 0 then sums all CTAs' partials in a fixed order and
// shares the totals through shared memory.
// kWarpTotals: v already holds this warp's totals (the same in every lane).
template <int BS, int NV, bool kWarpTotals = false>
__device__ __forceinline__ bool group_reduce(Group<BS>& g, double (&v)[NV], unsigned maxmask) {
  static_assert(NV <= kSlots, "too many reduction slots");
  constexpr int W = BS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* sw = g.sm_warp + (g.epoch & 1ull) * (W * kSlots);
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double t = v[j];
    if constexpr (!kWarpTotals) {
      const bool mx = (maxmask >> j) & 1u;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        double o = __shfl_xor_sync(kFull, t, off);
        t = mx ? fmax(t, o) : t + o;
      }
    }
    if (lane == 0) sw[warp * kSlots + j] = t;
  }
  __syncthreads();
  if (*g.sm_flag) {
    g.failed = true;
    return false;
  }
  if (g.nblk == 1) {
    // warp 0 reduces the warp partials in a fixed order (lane j <-> slot j) and
    // shares the totals through shared memory: the FP64 adds run once, not in
    // every warp (the FP64 pipe is narrow)
    double* tot1 = g.sm_tot + (g.epoch & 1ull) * kSlots;
    if (warp == 0 && lane < NV) {
      const bool mx = (maxmask >> lane) & 1u;
      double tot = 0.0;
      for (int w = 0; w < W; ++w) {
        const double o = sw[w * kSlots + lane];
        tot = mx ? fmax(tot, o) : tot + o;
      }
      tot1[lane] = tot;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = tot1[j];
    g.epoch++;
    return true;
  }
  double* buf = g.part + (size_t)(g.epoch & 1ull) * kSlots * g.nblk;
  double* tot_sm = g.sm_tot + (g.epoch & 1ull) * kSlots;
  if (warp == 0) {
    if (lane < NV) {
      const bool mx = (maxmask >> lane) & 1u;
      double bp = 0.0;
      for (int w = 0; w < W; ++w) {
        const double o = sw[w * kSlots + lane];
        bp = mx ? fmax(bp, o) : bp + o;
      }
      buf[lane * g.nblk + g.rank] = bp;
    }
    __syncwarp();
    if (lane == 0) {
      if (!group_arrive_wait(g.bar32, g.rank, g.nblk, g.epoch, g.timeout_ns, g.err)) {
        atomicExch(g.err, 1);
        *g.sm_flag = 1;
      }
    }
  }
  __syncthreads();
  if (*g.sm_flag) {
    g.failed = true;
    return false;
  }
  // Every thread loads its CTAs' partials of all slots at once (one round trip
  // to L2), then a fixed-order tree: lanes, warps.  The same in every CTA.
  // A warp with no CTA to load (warp * 32 >= nblk) hands in zeros, which is
  // what its tree would produce, without running the FP64 tree.
  {
    double* sw2 = g.sm_warp + ((g.epoch + 1ull) & 1ull) * (W * kSlots);  // free half until the next epoch
    if (warp * 32 < g.nblk) {
      double t[NV];
#pragma unroll
      for (int j = 0; j < NV; ++j) t[j] = 0.0;
      for (int b = threadIdx.x; b < g.nblk; b += BS) {
        double o[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) o[j] = __ldcg(buf + (size_t)j * g.nblk + b);
#pragma unroll
        for (int j = 0; j < NV; ++j) t[j] = ((maxmask >> j) & 1u) ? fmax(t[j], o[j]) : t[j] + o[j];
      }
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        const bool mx = (maxmask >> j) & 1u;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const double o = __shfl_xor_sync(kFull, t[j], off);
          t[j] = mx ? fmax(t[j], o) : t[j] + o;
        }
        if (lane == 0) sw2[warp * kSlots + j] = t[j];
      }
    } else if (lane < NV) {
      sw2[warp * kSlots + lane] = 0.0;
    }
    __syncthreads();
    if (warp == 0 && lane < NV) {
      const bool mx = (maxmask >> lane) & 1u;
      double a = 0.0;
      for (int w = 0; w < W; ++w) {
        const double o = sw2[w * kSlots + lane];
        a = mx ? fmax(a, o) : a + o;
      }
      tot_sm[lane] = a;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = tot_sm[j];
  g.epoch++;
  return true;
}

// Plain group barrier (no values).
template <int BS>
__device__ __forceinline__ bool group_sync(Group<BS>& g) {
  if (g.nblk == 1) {  // one CTA: a block barrier (the epoch still advances)
    __syncthreads();
    g.epoch++;
    return true;
  }
  double v[1] = {0.0};
  return group_reduce<BS, 1>(g, v, 0u);
}

// ---------------------------------------------------------------------------
// Row engine over a SELL-C-sigma row space.
//
// Regular rows live in 32-row slices; warp w of a CTA takes slices w, w+NW, ...
// of the CTA's range and lane l sums the row in slot l sequentially in column
// order (coalesced 128-byte loads of column indices and values, independent
// gathers).  Long rows are summed by one warp each (CSR, lane-strided, then a
// shuffle tree), huge rows by the whole CTA.  The phase epilogue runs once per
// row with the row sums.  Warps never wait for each other inside a phase, and
// every sum is taken in a fixed order.
// ---------------------------------------------------------------------------
enum class Ld { Stream, Cached, Generic };

template <Ld LM, class T>
__device__ __forceinline__ T ldm(const T* p) {
  if constexpr (LM == Ld::Stream) return ld_stream(p);
  else if constexpr (LM == Ld::Cached) return __ldg(p);
  else return *p;
}
template <Ld LM>
__device__ __forceinline__ int64_t ldm64(const int64_t* p) {
  if constexpr (LM == Ld::Generic) return *p;
  else return __ldg(reinterpret_cast<const long long*>(p));
}

// Shared context of the row engine for one CTA.
constexpr int kRowSums = 8;  // most row sums one space_rows call produces
struct RowCtx {
  double* red;  // BS/32 * kRowSums doubles of shared scratch (huge-row reductions)
};

// A product source: matrix in SELL form (regular rows) and CSR form (long and
// huge rows), with NG gathers (0, 1 or 2) of the column index.  With LO the
// source also sums the products of the values' rounding remainders (Sell::lo,
// Csr::lo) with the same gathers: it then yields 2 NG sums, the NG products
// with the values first, then the NG products with the remainders.
struct NoGather {
  __device__ __forceinline__ float operator()(int) const { return 0.f; }
};
template <class MatT, int NGv, class G1, class G2, bool LOv = false>
struct RowSrc {
  static constexpr int NG = NGv;
  static constexpr bool LO = LOv;
  static constexpr int NSUM = NGv * (LOv ? 2 : 1);
  using mat_type = MatT;
  Sell<MatT> S;
  Csr<MatT> M;
  G1 g1;
  G2 g2;
  bool on;
};
template <class MatT, class G1>
__device__ __forceinline__ RowSrc<MatT, 1, G1, NoGather> src(const Sell<MatT>& S, const Csr<MatT>& M,
                                                             G1 g1, bool on = true) {
  return RowSrc<MatT, 1, G1, NoGather>{S, M, g1, NoGather{}, on};
}
template <class MatT, class G1, class G2>
__device__ __forceinline__ RowSrc<MatT, 2, G1, G2> src2(const Sell<MatT>& S, const Csr<MatT>& M, G1 g1,
                                                        G2 g2, bool on = true) {
  return RowSrc<MatT, 2, G1, G2>{S, M, g1, g2, on};
}
// The same with the remainder products (LO); the caller ensures S.lo and M.lo are set.
template <bool LO, class MatT, class G1>
__device__ __forceinline__ RowSrc<MatT, 1, G1, NoGather, LO> src_lo(const Sell<MatT>& S, const Csr<MatT>& M,
                                                                   G1 g1, bool on = true) {
  return RowSrc<MatT, 1, G1, NoGather, LO>{S, M, g1, NoGather{}, on};
}
template <bool LO, class MatT, class G1, class G2>
__device__ __forceinline__ RowSrc<MatT, 2, G1, G2, LO> src2_lo(const Sell<MatT>& S, const Csr<MatT>& M, G1 g1,
                                                              G2 g2, bool on = true) {
  return RowSrc<MatT, 2, G1, G2, LO>{S, M, g1, g2, on};
}
template <class MatT>
__device__ __forceinline__ RowSrc<MatT, 0, NoGather, NoGather> nosrc() {
  return RowSrc<MatT, 0, NoGather, NoGather>{Sell<MatT>{}, Csr<MatT>{}, NoGather{}, NoGather{}, false};
}

// Columns of a slice whose loads are issued together (memory-level parallelism).
#ifndef PDHCG_SLICE_UNROLL
#define PDHCG_SLICE_UNROLL 4
#endif
#ifndef PDHCG_GROUP_SLICE_UNROLL
#define PDHCG_GROUP_SLICE_UNROLL PDHCG_SLICE_UNROLL
#endif
// multi-CTA groups (streamed matrices, global vectors) / single-CTA solves
template <Ld LM>
__host__ __device__ constexpr int slice_unroll() { return LM == Ld::Stream ? PDHCG_GROUP_SLICE_UNROLL : PDHCG_SLICE_UNROLL; }

// Accumulate slot `lane` of slice s of source X into sums[0..NSUM) in column order.
template <Ld LM, class Acc, class X>
__device__ __forceinline__ void slice_dot(const X& x, int s, int lane, Acc* sums) {
  if constexpr (X::NG > 0) {
    if (!x.on) return;
    // pool CTAs may hold the slice offsets in shared memory: a generic load
    constexpr Ld LP = LM == Ld::Cached ? Ld::Generic : LM;
    const int64_t b = ldm64<LP>(x.S.ptr + s), e = ldm64<LP>(x.S.ptr + s + 1);
    const int W = int((e - b) >> 5);
    const int* cp = x.S.col + b + lane;
    const auto* vp = x.S.val + b + lane;
    if constexpr (X::LO) {
      const float* lp = x.S.lo + b + lane;
#pragma unroll slice_unroll<LM>()
      for (int j = 0; j < W; ++j) {
        const int c = ldm<LM>(cp + 32 * j);
        const auto v = ldm<LM>(vp + 32 * j);
        const float l = ldm<LM>(lp + 32 * j);
        const Acc a1 = Acc(x.g1(c));
        madd(sums[0], v, a1);
        madd(sums[X::NG], l, a1);
        if constexpr (X::NG == 2) {
          const Acc a2 = Acc(x.g2(c));
          madd(sums[1], v, a2);
          madd(sums[3], l, a2);
        }
      }
    } else {
#pragma unroll slice_unroll<LM>()
      for (int j = 0; j < W; ++j) {
        const int c = ldm<LM>(cp + 32 * j);
        const auto v = ldm<LM>(vp + 32 * j);
        madd(sums[0], v, Acc(x.g1(c)));
        if constexpr (X::NG == 2) madd(sums[1], v, Acc(x.g2(c)));
      }
    }
  }
}

template <class X>
struct SrcMat {
  using type = typename X::mat_type;
};

// Prefetch distance, in slices of the same warp, of the bulk L2 prefetch of
// streamed SELL slices (0 = off).
#ifndef PDHCG_L2_PREFETCH
#define PDHCG_L2_PREFETCH 1
#endif
// Element span [b, e) of slice s of source X (empty when s >= s_end or X is off).
template <Ld LM, class X>
__device__ __forceinline__ void slice_span(const X& x, int s, int s_end, int64_t& b, int64_t& e) {
  b = 0;
  e = 0;
  if constexpr (X::NG > 0)
    if (x.on && s < s_end) {
      b = ldm64<LM>(x.S.ptr + s);
      e = ldm64<LM>(x.S.ptr + s + 1);
    }
}
// Bulk L2 prefetch of the column indices and values of span [b, e).  Slices
// start on multiples of 32 elements of 16-byte-aligned arrays, so both copies
// are 16-byte aligned with sizes that are multiples of 16 (checked anyway).
template <class X>
__device__ __forceinline__ void slice_prefetch_l2(const X& x, int64_t b, int64_t e) {
  if constexpr (X::NG > 0) {
    using MatT = typename SrcMat<X>::type;
    if (e <= b) return;
    const int* c = x.S.col + b;
    const MatT* v = x.S.val + b;
    const unsigned cb = unsigned(e - b) * 4u, vb = unsigned(e - b) * unsigned(sizeof(MatT));
    if (((reinterpret_cast<uintptr_t>(c) | cb) & 15u) == 0) bulk_prefetch_l2(c, cb);
    if (((reinterpret_cast<uintptr_t>(v) | vb) & 15u) == 0) bulk_prefetch_l2(v, vb);
  }
}

// Lane-strided partial of CSR row `row` of source X, start offset `first`,
// stride `step`; 8 elements per lane in flight.
template <Ld LM, class Acc, class X>
__device__ __forceinline__ void csr_part(const X& x, int row, int first, int step, Acc* sums) {
  if constexpr (X::NG > 0) {
    if (!x.on) return;
    using MatT = typename SrcMat<X>::type;
    constexpr int U = 8;
    const int b = __ldg(x.M.rowptr + row), e = __ldg(x.M.rowptr + row + 1);
    for (int k0 = b + first; k0 < e; k0 += U * step) {
      int c[U];
      MatT v[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (k0 + u * step < e) {
          c[u] = ldm<LM>(x.M.col + k0 + u * step);
          v[u] = ldm<LM>(x.M.val + k0 + u * step);
        }
      Acc g1v[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (k0 + u * step < e) g1v[u] = Acc(x.g1(c[u]));
      if constexpr (X::NG == 2) {
        Acc g2v[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (k0 + u * step < e) g2v[u] = Acc(x.g2(c[u]));
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (k0 + u * step < e) madd(sums[1], v[u], g2v[u]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (k0 + u * step < e) madd(sums[0], v[u], g1v[u]);
      if constexpr (X::LO) {
        // remainder products, same order (the gathers are reloaded: long rows are few)
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (k0 + u * step < e) {
            const float l = ldm<LM>(x.M.lo + k0 + u * step);
            madd(sums[X::NG], l, g1v[u]);
            if constexpr (X::NG == 2) madd(sums[3], l, Acc(x.g2(c[u])));
          }
      }
    }
  }
}

// Walk this CTA's share of a row space and call epi(row, const Acc* sums) once
// per row; sums holds the A sums then the B sums.  part_rank < 0: the
// whole space (single-CTA group).  red: BS/32 * kRowSums doubles of shared scratch.
template <int BS, Ld LM, class Acc, class SA, class SB, class Epi>
__device__ __forceinline__ void space_rows(const SpaceLayout& sp, int part_rank, const SA& A,
                                        const SB& B, const RowCtx& rc, Epi epi) {
  double* red = rc.red;
  constexpr int NA = SA::NSUM, NB = SB::NSUM, NS = NA + NB;
  static_assert(NS >= 1 && NS <= kRowSums, "1..kRowSums sums per row");
  constexpr int NW = BS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int s0 = 0, s1 = sp.nslices, l0 = 0, l1 = sp.nlong, h0 = 0, h1 = sp.nhuge;
  if (part_rank >= 0 && sp.slice_part) {
    s0 = sp.slice_part[part_rank];
    s1 = sp.slice_part[part_rank + 1];
    l0 = sp.long_part[part_rank];
    l1 = sp.long_part[part_rank + 1];
    h0 = sp.huge_part[part_rank];
    h1 = sp.huge_part[part_rank + 1];
  }
  // regular rows: one slice per warp at a time, lane l summing the row in slot l.
  // Streamed matrices: lane 0 also prefetches into L2 the slice this warp takes
  // PDHCG_L2_PREFETCH turns later (issued after the current slice, whose work
  // covers the latency of the two pointer loads).
  constexpr bool kPf = LM == Ld::Stream && PDHCG_L2_PREFETCH > 0;
  if constexpr (kPf) {
    if (lane == 0)
      for (int d = 0; d < PDHCG_L2_PREFETCH; ++d) {
        int64_t b, e;
        slice_span<LM>(A, s0 + warp + d * NW, s1, b, e);
        slice_prefetch_l2(A, b, e);
        slice_span<LM>(B, s0 + warp + d * NW, s1, b, e);
        slice_prefetch_l2(B, b, e);
      }
  }
  for (int s = s0 + warp; s < s1; s += NW) {
    const int row = ldm<LM>(sp.perm + s * 32 + lane);
    int64_t pab = 0, pae = 0, pbb = 0, pbe = 0;
    if constexpr (kPf) {
      if (lane == 0) {
        slice_span<LM>(A, s + PDHCG_L2_PREFETCH * NW, s1, pab, pae);
        slice_span<LM>(B, s + PDHCG_L2_PREFETCH * NW, s1, pbb, pbe);
      }
    }
    Acc sums[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) sums[q] = Acc(0);
    slice_dot<LM, Acc>(A, s, lane, sums);
    slice_dot<LM, Acc>(B, s, lane, sums + NA);
    if constexpr (kPf) {
      if (lane == 0) {
        slice_prefetch_l2(A, pab, pae);
        slice_prefetch_l2(B, pbb, pbe);
      }
    }
#pragma unroll
    for (int q = 0; q < NS; ++q) acc_finish(sums[q]);
    if (row >= 0) epi(row, sums);
  }
  // long rows: one warp per row
  for (int li = l0 + warp; li < l1; li += NW) {
    const int row = __ldg(sp.longs + li);
    Acc sums[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) sums[q] = Acc(0);
    csr_part<LM, Acc>(A, row, lane, 32, sums);
    csr_part<LM, Acc>(B, row, lane, 32, sums + NA);
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      acc_finish(sums[q]);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) sums[q] += shfl_xor(sums[q], off);
    }
    if (lane == 0) epi(row, sums);
  }
  // huge rows: the whole CTA per row
  for (int hi = h0; hi < h1; ++hi) {
    const int row = __ldg(sp.huges + hi);
    Acc sums[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) sums[q] = Acc(0);
    csr_part<LM, Acc>(A, row, threadIdx.x, BS, sums);
    csr_part<LM, Acc>(B, row, threadIdx.x, BS, sums + NA);
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      acc_finish(sums[q]);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) sums[q] += shfl_xor(sums[q], off);
      if (lane == 0) red[warp * kRowSums + q] = double(sums[q]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      Acc tot[NS];
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        tot[q] = Acc(0);
        for (int w = 0; w < NW; ++w) tot[q] += Acc(red[w * kRowSums + q]);
      }
      epi(row, tot);
    }
    __syncthreads();
  }
}

// Elementwise walk of [lo, hi) (no CSR work), one element per thread.
template <int BS, class Body>
__device__ __forceinline__ void for_elems(int lo, int hi, Body body) {
#pragma unroll 4
  for (int i = lo + (int)threadIdx.x; i < hi; i += BS) body(i);
}

}  // namespace pdhcg

// dfloat.cuh — "double-float" numbers: an unevaluated sum hi + lo of two FP32
// values (|lo| <= ulp(hi) / 2 after normalisation), about 48 significant bits,
// computed entirely on the FP32 pipe.
//
// Why: a B300 SM retires FP64 at 1/64 of its FP32 rate, so per-element FP64
// vector arithmetic saturates the FP64 pipe long before memory.  The vector
// state of the iteration needs more than FP32's 24 bits to reach a relative KKT
// residual of 1e-6, but not FP64's full 53; double-float covers that range at
// FP32 throughput.
//
// Arithmetic from the error-free transformations of the literature:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly, any order of |a|, |b|;
//   FastTwoSum (Dekker 1971): the same when |a| >= |b|;
//   TwoProd via FMA: p + e = a * b exactly;
// combined into double-float add / multiply / divide as in Dekker (1971),
// "A floating-point technique for extending the available precision", with the
// renormalisation after each operation.  Infinite values (absent bounds) only
// flow through comparisons and clamps; their lo part is kept at zero.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

namespace pdhcg {

// The dfloat overloads below must not hide the built-in ones for float / double.
using ::fma;
using ::fmaf;

// 8-byte aligned, so that an entry moves as one 64-bit load or store (a gather
// is one memory request, a shared-memory access one 64-bit word); every array of
// them starts on a 16-byte (shared memory) or 256-byte (device arena) boundary.
struct __align__(8) dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ __forceinline__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ explicit dfloat(int v) : hi(float(v)), lo(0.f) {}
  __host__ __device__ __forceinline__ explicit dfloat(float v) : hi(v), lo(0.f) {}
  // Nearest float, then the float nearest to the remainder.
  __host__ __device__ __forceinline__ explicit dfloat(double v) {
    hi = float(v);
    lo = std::isfinite(hi) ? float(v - double(hi)) : 0.f;
  }
  __host__ __device__ __forceinline__ explicit operator double() const { return double(hi) + double(lo); }
};

// s + e == a + b exactly (six FP32 operations).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// s + e == a + b exactly, given |a| >= |b| or a == 0 (three operations).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
__device__ __forceinline__ dfloat df_norm(float s, float e) {
  float h, l;
  fast_two_sum(s, e, h, l);
  return dfloat(h, l);
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  return std::isfinite(s) ? df_norm(s, e) : dfloat(s, 0.f);
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return std::isfinite(p) ? df_norm(p, e) : dfloat(p, 0.f);
}
// Long division: one FP32 quotient, its remainder in double-float, one correction.
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b) {
  const float q1 = a.hi / b.hi;
  if (!std::isfinite(q1)) return dfloat(q1, 0.f);
  const dfloat r = a - b * dfloat(q1);
  const float q2 = r.hi / b.hi;
  return df_norm(q1, q2);
}
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }
__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) { return a * b + c; }

__device__ __forceinline__ bool operator<(dfloat a, dfloat b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool operator>(dfloat a, dfloat b) { return b < a; }

// SpMV accumulation s += v * x with v an FP32 matrix value.  The rounding error
// of each step is kept in s.lo without renormalising; acc_finish() renormalises
// once per row.
__device__ __forceinline__ void madd(dfloat& s, float v, dfloat x) {
  const float p = v * x.hi;
  float pe = fmaf(v, x.hi, -p);
  pe = fmaf(v, x.lo, pe);
  float t, e;
  two_sum(s.hi, p, t, e);
  s.hi = t;
  s.lo += e + pe;
}
__device__ __forceinline__ void madd(double& s, double v, double x) { s = fma(v, x, s); }
__device__ __forceinline__ void madd(double& s, float v, double x) { s = fma(double(v), x, s); }
__device__ __forceinline__ void madd(float& s, float v, float x) { s = fmaf(v, x, s); }

__device__ __forceinline__ void acc_finish(dfloat& s) {
  float h, l;
  two_sum(s.hi, s.lo, h, l);
  s = dfloat(h, l);
}
__device__ __forceinline__ void acc_finish(double&) {}
__device__ __forceinline__ void acc_finish(float&) {}

__device__ __forceinline__ dfloat shfl_xor(dfloat v, int off) {
  return dfloat(__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off));
}
__device__ __forceinline__ double shfl_xor(double v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
__device__ __forceinline__ dfloat shfl_idx(dfloat v, int src) {
  return dfloat(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}
__device__ __forceinline__ double shfl_idx(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float shfl_idx(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float shfl_xor(float v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }

}  // namespace pdhcg

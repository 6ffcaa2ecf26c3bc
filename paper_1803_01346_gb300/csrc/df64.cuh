// df64.cuh - double-float ("double-word") arithmetic for the FP64-equivalent FFT passes.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, which
// carries a 48-bit significand (unit roundoff 2^-48, about 3.6e-15) on the FP32 pipes: on
// GB300 the FP64 pipe issues at a small fraction of the FP32 rate, so FFT butterflies built
// from a few FP32 operations per double-float operation run several times faster than the
// same butterflies in FP64.  The exponent range is FP32's.
//
// Building blocks (error-free transformations, all in round-to-nearest):
//   two_sum(a, b)      = (s, e) with s = fl(a + b), s + e = a + b exactly   (Knuth; 6 flops)
//   fast_two_sum(a, b) = the same when |a| >= |b| or a = 0                   (Dekker; 3 flops)
//   two_prod(a, b)     = (p, e) with p = fl(a b), p + e = a b exactly, e = fma(a, b, -p)
// Sum: two_sum of the high parts, the low parts added to the error term, renormalised by
// fast_two_sum (the "sloppy" double-word sum of Joldes, Muller and Popescu, ACM TOMS 44
// (2017)).  Under cancellation its relative error is not bounded, but its absolute error is
// below a small multiple of u^2 (|x| + |y|), u = 2^-24, which is the bound an FFT's error
// analysis needs (errors relative to the operands' magnitudes).
// Product: two_prod of the high parts, the cross terms added by fma, renormalised (error
// below about 7 u^2 |x y|; Joldes, Muller and Popescu, ACM TOMS 44 (2017), "DWTimesDW").
// Every step is an explicit _rn intrinsic, so the compiler neither contracts nor reorders
// them.
#pragma once
#include <cuda_runtime.h>

namespace scfft {

struct __align__(8) dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  // nearest double-float of a double (exact when d has at most 48 significant bits); folds at
  // compile time for constants
  __host__ __device__ constexpr dfloat(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

struct __align__(16) dfloat2 {
  dfloat x, y;
};

__device__ __forceinline__ dfloat fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfloat two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  return dfloat(s, __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv)));
}

__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) {
  const dfloat s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dfloat operator-(dfloat x) { return dfloat(-x.hi, -x.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x, dfloat y) { return x + (-y); }
__device__ __forceinline__ dfloat operator*(dfloat x, dfloat y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dfloat& operator+=(dfloat& x, dfloat y) { return x = x + y; }
__device__ __forceinline__ dfloat& operator*=(dfloat& x, dfloat y) { return x = x * y; }

// ---------------------------------------------------------------- two lanes at once
// The sum on two double-floats held lane-wise in float2 pairs (hi lanes, lo lanes), as the
// two-lane FP32 instructions of sm_100 and later: each lane rounds exactly as the scalar step
// does (b * -1 + a rounds as a - b), so a lane gives the scalar result bit for bit and the pair
// costs one instruction per step instead of two.
struct dfpair {
  float2 hi, lo;
};
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ dfpair fast_two_sum2(float2 a, float2 b) {
  const float2 s = __fadd2_rn(a, b);
  dfpair r;
  r.hi = s;
  r.lo = sub2(b, sub2(s, a));
  return r;
}
// lane-wise x + y (the scalar operator+ above in each lane)
__device__ __forceinline__ dfpair add2(dfpair x, dfpair y) {
  const float2 s = __fadd2_rn(x.hi, y.hi);
  const float2 bv = sub2(s, x.hi);
  const float2 av = sub2(s, bv);
  const float2 e = __fadd2_rn(sub2(x.hi, av), sub2(y.hi, bv));
  return fast_two_sum2(s, __fadd2_rn(e, __fadd2_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dfpair pr(dfloat a, dfloat b) {  // lanes (a, b)
  dfpair r;
  r.hi = make_float2(a.hi, b.hi);
  r.lo = make_float2(a.lo, b.lo);
  return r;
}
__device__ __forceinline__ dfloat lane0(dfpair p) { return dfloat(p.hi.x, p.lo.x); }
__device__ __forceinline__ dfloat lane1(dfpair p) { return dfloat(p.hi.y, p.lo.y); }

// complex double-float: sums and differences run the real and imaginary parts as the two lanes
// (products stay scalar: their two-lane forms need the operands' lanes rearranged, which cost
// more than the lanes saved)
__device__ __forceinline__ dfloat2 mk(dfloat a, dfloat b) { dfloat2 r; r.x = a; r.y = b; return r; }
__device__ __forceinline__ dfloat2 mk(dfpair p) { return mk(lane0(p), lane1(p)); }
__device__ __forceinline__ dfloat2 operator+(dfloat2 a, dfloat2 b) { return mk(add2(pr(a.x, a.y), pr(b.x, b.y))); }
__device__ __forceinline__ dfloat2 operator-(dfloat2 a, dfloat2 b) {
  return mk(add2(pr(a.x, a.y), pr(-b.x, -b.y)));
}
__device__ __forceinline__ dfloat2 scl(dfloat2 a, dfloat s) { return mk(a.x * s, a.y * s); }

// Precision of the node-wise arithmetic in the passes (power law, material laws, reverse-mode
// Jacobians): the FFT's own precision, except that the double-float passes evaluate those
// few operations per node in FP64 (pow, sqrt and division have no double-float form here).
template <typename T> struct acc_of { typedef T type; };
template <> struct acc_of<dfloat> { typedef double type; };
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ double to_acc(dfloat v) { return (double)v; }
template <typename T> __device__ __forceinline__ T from_acc(typename acc_of<T>::type v) { return (T)v; }

}  // namespace scfft

// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi)/2), about 48 significant bits, computed with FP32
// instructions only.  GB300 issues FP32 64 times faster than FP64, so the
// defect of the mixed-precision refinement runs in this type.
//
// The error-free transformations are Knuth's TwoSum and Dekker's
// Fast2Sum / FMA-based TwoProduct (Dekker 1971; Knuth, TAOCP vol. 2;
// Hida, Li & Bailey 2001).  The rounded primitives __fadd_rn / __fsub_rn /
// __fmul_rn are used wherever a compiler contraction into an FMA would break
// an exact error term.
#pragma once

#include <cuda_runtime.h>

namespace mgwr {

struct dd {
  float hi, lo;
  dd() = default;
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  // exact for constants; at run time only used on the host or in setup
  __host__ __device__ constexpr dd(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ constexpr dd(int x) : dd((double)x) {}
  __device__ __forceinline__ explicit operator float() const { return __fadd_rn(hi, lo); }
};

// x as a double-float pair with two FP64-pipe operations instead of four: hi =
// x with its last 29 significand bits cleared, built as a float by integer
// operations (exact when x lies in float's normal range), lo = x - hi (exact
// in FP64) rounded to FP32; x - (hi + lo) is below 2^-48 |x|.  Outside that
// range: zero or tiny x gives (0, x rounded), huge, inf or NaN (x rounded, 0).
// hi is truncated, not rounded, so |lo| < ulp(hi) (the pair is not
// renormalised; the sums below accept that).
__device__ __forceinline__ dd dd_split_fast(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e >= 897 && e <= 1150) {
    const double hd = __longlong_as_double((long long)(b & ~0x1FFFFFFFull));
    const unsigned hb = ((unsigned)(b >> 32) & 0x80000000u) | ((unsigned)(e - 896) << 23) |
                        ((unsigned)(b >> 29) & 0x7FFFFFu);
    return dd(__uint_as_float(hb), __double2float_rn(x - hd));
  }
  if (e < 897) return dd(0.f, __double2float_rn(x));
  return dd(__double2float_rn(x), 0.f);
}

// The same pair with no FP64 arithmetic at all, for 2^-74 <= |x| < 2^128: hi as
// in dd_split_fast, lo = the 29 cleared bits as an integer, converted to FP32
// (rounded to 24 bits) and scaled by the exact power of two 2^(e - 1075), with
// x's sign: x - (hi + lo) below 2^-48 |x| as there.  Other x take
// dd_split_fast.
__device__ __forceinline__ dd dd_split_int(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e >= 949 && e <= 1150) {
    const unsigned hb = ((unsigned)(b >> 32) & 0x80000000u) | ((unsigned)(e - 896) << 23) |
                        ((unsigned)(b >> 29) & 0x7FFFFFu);
    const float scale = __int_as_float((e - 1075 + 127) << 23);  // 2^(e - 1075), normal
    const float mag = __fmul_rn(__uint2float_rn((unsigned)(b & 0x1FFFFFFFull)), scale);
    return dd(__uint_as_float(hb), (b >> 63) ? -mag : mag);
  }
  return dd_split_fast(x);
}

// The pair (RN32(x), RN32(x - RN32(x))) that FP64 arithmetic forms ((float)x,
// then the exact FP64 difference rounded), here from integer and FP32
// operations alone for 2^-74 <= |x| < 2^126 and for x = +-0; other x take the
// FP64 forms.  Bitwise the same pair: hi is x's top 24 significand bits rounded
// to nearest (ties to even) on the bits, the increment carrying into the
// exponent; x - hi is the cleared 29-bit remainder, less 2^29 when hi rounded
// up, times the power of two 2^(e - 1075), converted by one FP32 rounding and
// an exact scaling.  GB300 runs the FP64 conversions and subtraction at 1/64
// of the FP32 rate.
__device__ __forceinline__ dd dd_split_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  if (e >= 949 && e <= 1148) {
    const unsigned r29 = (unsigned)(b & 0x1FFFFFFFull);
    unsigned hb = sign | ((unsigned)(e - 896) << 23) | ((unsigned)(b >> 29) & 0x7FFFFFu);
    const bool up = r29 > 0x10000000u || (r29 == 0x10000000u && (hb & 1u));
    hb += up ? 1u : 0u;
    const float scale = __int_as_float((e - 1075 + 127) << 23);  // 2^(e - 1075), normal
    const float mag = __fmul_rn(__int2float_rn((int)r29 - (up ? 0x20000000 : 0)), scale);
    return dd(__uint_as_float(hb), sign ? -mag : mag);
  }
  if ((b << 1) == 0) return dd(__uint_as_float(sign), 0.f);
  const float hi = __double2float_rn(x);
  return dd(hi, __double2float_rn(x - (double)hi));
}

// s + e = a + b exactly (TwoSum, any a, b)
__device__ __forceinline__ dd dd_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dd(s, e);
}

// s + e = a + b exactly when |a| >= |b| (Fast2Sum)
__device__ __forceinline__ dd dd_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dd(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// Sum with one renormalisation: error below about 2^-44 (|a| + |b|); the
// form used inside FFT butterflies, whose error is bounded in norm anyway.
__device__ __forceinline__ dd operator+(dd a, dd b) {
  dd s = dd_two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return dd_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd& operator+=(dd& a, dd b) {
  a = a + b;
  return a;
}

// Sum accurate also under cancellation: error below about 2^-47 |a + b|
// (both pairs summed exactly, two renormalisations).  Used for the stencil
// differences of the defect.
__device__ __forceinline__ dd dd_add_accurate(dd a, dd b) {
  dd s = dd_two_sum(a.hi, b.hi);
  const dd t = dd_two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = dd_fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return dd_fast_two_sum(s.hi, s.lo);
}

// Product: hi*hi split exactly by an FMA, cross terms added once.
__device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dd_fast_two_sum(p, e);
}

__device__ __forceinline__ dd dd_add_float(dd a, float b) {
  dd s = dd_two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return dd_fast_two_sum(s.hi, s.lo);
}

// Sum without the closing renormalisation (8 FP32 operations): hi is the
// rounded sum of the leading words, lo their exact error plus the trailing
// words.  The pair still stands for the sum to about 2^-46 of the operands'
// magnitudes; the FFT butterflies chain these, and every product or accurate
// sum that follows renormalises.
__device__ __forceinline__ dd dd_add_lazy(dd a, dd b) {
  dd s = dd_two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return s;
}
__device__ __forceinline__ dd dd_sub_lazy(dd a, dd b) {
  dd s = dd_two_sum(a.hi, -b.hi);
  s.lo = __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo));
  return s;
}

// a*b + c*e with one TwoSum (19 FP32 operations instead of two products and a
// sum): the leading products p1, p2 with their exact errors from FMAs, the four
// cross terms and both errors gathered in one FP32 sum, TwoSum(p1, p2) and one
// Fast2Sum.  Error about 2^-46 (|a b| + |c e|), as for the separate operations.
__device__ __forceinline__ dd dd_dot2(dd a, dd b, dd c, dd e) {
  const float p1 = __fmul_rn(a.hi, b.hi);
  const float p2 = __fmul_rn(c.hi, e.hi);
  float t = __fmaf_rn(a.hi, b.hi, -p1);
  t = __fadd_rn(t, __fmaf_rn(c.hi, e.hi, -p2));
  t = __fmaf_rn(a.hi, b.lo, t);
  t = __fmaf_rn(a.lo, b.hi, t);
  t = __fmaf_rn(c.hi, e.lo, t);
  t = __fmaf_rn(c.lo, e.hi, t);
  const dd s = dd_two_sum(p1, p2);
  return dd_fast_two_sum(s.hi, __fadd_rn(s.lo, t));
}

// magnitude used for norms: |hi| (relative error below 2^-23)
__device__ __forceinline__ float dd_abs_hi(dd a) { return fabsf(a.hi); }

}  // namespace mgwr

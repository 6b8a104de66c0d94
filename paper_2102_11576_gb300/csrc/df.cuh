// df.cuh -- "double-FP32" arithmetic: a value is the unevaluated sum hi + lo
// of two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.
//
// GB300 runs FP32 at 58x its FP64 rate, so an FFT whose every real operation
// costs ~10 FP32 operations is still several times faster than the same FFT
// in FP64.  The operations are the classical error-free transforms:
//   two_sum (Knuth): s = a + b and the exact rounding error of that sum,
//   two_prod (with FMA, Dekker's product): p = a * b and its exact error,
// combined as in double-double arithmetic (Dekker 1971; Hida, Li & Bailey's
// QD library describes the same building blocks).  Additions use the
// "sloppy" form, whose error is bounded by a few units of 2^-48 times
// |a| + |b| -- the normwise bound an FFT error analysis needs.
#pragma once

namespace rsfde {

struct __align__(8) df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df operator+(df a, df b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s, e);
}

__device__ __forceinline__ df operator-(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__device__ __forceinline__ df& operator*=(df& a, df b) { return a = a * b; }

// acc + a * b: the product's error term is carried into the sum without its
// own renormalisation (a fused form of the two operators above).
__device__ __forceinline__ df df_fma(df acc, df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(acc.hi, p);
  const float bb = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  return df_fast_two_sum(s, __fadd_rn(err, __fadd_rn(acc.lo, e)));
}

// Conversions between the storage and arithmetic types (float, double, df);
// float -> df is exact and needs no FP64 instruction.
template <typename To, typename From>
__device__ __forceinline__ To cvt(From x) {
  return static_cast<To>(x);
}
template <>
__device__ __forceinline__ df cvt<df, float>(float x) {
  return df(x, 0.0f);
}
template <>
__device__ __forceinline__ df cvt<df, double>(double x) {
  return df(x);
}
template <>
__device__ __forceinline__ df cvt<df, df>(df x) {
  return x;
}
template <>
__device__ __forceinline__ double cvt<double, df>(df x) {
  return double(x);
}
template <>
__device__ __forceinline__ float cvt<float, df>(df x) {
  return __fadd_rn(x.hi, x.lo);
}

}  // namespace rsfde

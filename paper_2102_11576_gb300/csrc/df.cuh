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

// Conversions between FP64 and FP32 on the integer pipe.  GB300's FP64 pipe
// runs a double <-> float conversion at a small fraction of its FMA rate (a
// conversion per element cost an FP64-bound Gram-Schmidt update as much as
// ten FMAs), so the hot paths move the fields of the IEEE encodings instead.
// f32_trunc: the float whose significand is the double's leading 24 bits
// (rounded toward zero; |error| < 2^-23 |x|); values below the float range
// become signed zero, above it infinity.
__device__ __forceinline__ float f32_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hi = (unsigned int)(b >> 32);
  const int e = (int)((hi >> 20) & 0x7FF) - 896;  // float biased exponent
  const unsigned int sign = hi & 0x80000000u;
  const unsigned int man = (unsigned int)(b >> 29) & 0x7FFFFFu;
  unsigned int f = sign;
  if (e == 1151 && (b & 0xFFFFFFFFFFFFFull)) f |= 0x7FC00000u;  // NaN stays NaN
  else if (e >= 255) f |= 0x7F800000u;
  else if (e > 0) f |= ((unsigned int)e << 23) | man;
  return __uint_as_float(f);
}
// f64_exact: the double equal to a float (every float is a double); normal
// numbers, zeros, infinities and NaNs by their fields, subnormal floats (below
// 2^-126) through the conversion instruction.
__device__ __forceinline__ double f64_exact(float x) {
  const unsigned int f = __float_as_uint(x);
  const unsigned int e = (f >> 23) & 0xFF;
  const unsigned int man = f & 0x7FFFFFu;
  if (e == 0 && man != 0) return (double)x;
  const unsigned long long sign = (unsigned long long)(f & 0x80000000u) << 32;
  unsigned long long ed = 0;
  if (e == 255) ed = 0x7FFull;
  else if (e != 0) ed = e + 896;
  return __longlong_as_double((long long)(sign | (ed << 52) | ((unsigned long long)man << 29)));
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
  return f64_exact(x.hi) + f64_exact(x.lo);
}
template <>
__device__ __forceinline__ double cvt<double, float>(float x) {
  return f64_exact(x);
}
template <>
__device__ __forceinline__ float cvt<float, df>(df x) {
  return __fadd_rn(x.hi, x.lo);
}

}  // namespace rsfde

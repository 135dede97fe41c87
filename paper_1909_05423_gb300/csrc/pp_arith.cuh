// pp_arith.cuh -- arithmetic types of the GPU path.
//
// GB300 runs FP64 at about 1/67 of its FP32 rate, and FP32<->FP64 conversion
// instructions at the FP64 rate.  The FP64-accurate path therefore computes in
// "double-float" arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers (Dekker 1971, "A floating-point technique for extending the available
// precision"; Knuth's TwoSum), giving a ~47-bit significand.  FP64 grid values
// are split into (hi, lo) with integer bit operations and re-assembled with one
// FP64 add of the two exactly converted parts.  The mixed-precision path uses
// plain FP32 for the transforms and the same double-float arithmetic in the
// tridiagonal solve.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pp {

// ---------------------------------------------------------------- double-float
struct __align__(8) df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float h) { return df{h, 0.0f}; }

// Knuth TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// Dekker FastTwoSum (|a| >= |b|): s + e == a + b exactly.
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df operator+(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  df r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ df operator-(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
// product with FMA-based TwoProd; the lo*lo term (2^-48 relative) is dropped.
__device__ __forceinline__ df operator*(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  df r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}
// a*b - c*d with one renormalisation (used by the complex product).
__device__ __forceinline__ df dot2_sub(df a, df b, df c, df d) {
  float p1 = __fmul_rn(a.hi, b.hi);
  float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  float p2 = __fmul_rn(c.hi, d.hi);
  float e2 = __fmaf_rn(c.hi, d.hi, -p2);
  float s, e;
  two_sum(p1, -p2, s, e);
  e = __fadd_rn(e, __fsub_rn(e1, e2));
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  e = __fmaf_rn(-c.hi, d.lo, e);
  e = __fmaf_rn(-c.lo, d.hi, e);
  df r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
// a*b + c*d
__device__ __forceinline__ df dot2_add(df a, df b, df c, df d) { return dot2_sub(a, b, -c, d); }
__device__ __forceinline__ df df_half(df a) { return df{0.5f * a.hi, 0.5f * a.lo}; }

// Unnormalised forms for the line transforms.  The leading parts are still summed (TwoSum) or
// multiplied (TwoProd) exactly and the trailing part still collects every error term, but the
// final FastTwoSum that makes |lo| <= ulp(hi)/2 is skipped (3 of 11 instructions of a sum, 3 of
// 7 of a product).  hi + lo keeps its value; lo only grows by about ulp(hi) per operation, so
// after the ~15 operations a transform applies to a value the rounding error of lo stays near
// 2^-48 of the magnitudes the value was computed from, the norm-wise accuracy of the FFT.
// Products and sums read unnormalised pairs correctly: TwoSum and TwoProd need no ordering of
// their operands, and lo enters only through FP32 adds and FMAs.
__device__ __forceinline__ df add_u(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return df{s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}
__device__ __forceinline__ df mul_u(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df{p, e};
}
__device__ __forceinline__ df dot2_sub_u(df a, df b, df c, df d) {
  const float p1 = __fmul_rn(a.hi, b.hi);
  const float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  const float p2 = __fmul_rn(c.hi, d.hi);
  const float e2 = __fmaf_rn(c.hi, d.hi, -p2);
  float s, e;
  two_sum(p1, -p2, s, e);
  e = __fadd_rn(e, __fsub_rn(e1, e2));
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  e = __fmaf_rn(-c.hi, d.lo, e);
  e = __fmaf_rn(-c.lo, d.hi, e);
  return df{s, e};
}

// df reciprocal: one Newton step on the FP32 reciprocal.
__device__ __forceinline__ df df_rcp(df a) {
  float r = __frcp_rn(a.hi);
  df one = df{1.0f, 0.0f};
  df ra = df{r, 0.0f};
  df err = one - a * ra;     // 1 - a r
  return ra + ra * err;      // r (1 + (1 - a r))
}

// ------------------------------------------------ FP64 <-> double-float (integer)
// Integer instructions run at half the FP32 rate on this GPU, so each conversion has a short
// path for the normal range (one range test) and falls back to the general code otherwise.
// t = |high word| - (896 << 20) re-biases the FP64 exponent to FP32: for 1 <= e_f <= 254,
// t = e_f 2^20 + (top 20 mantissa bits), and (t << 3) | (low word >> 29) is the FP32 magnitude
// truncated to 23 mantissa bits.

// General-case split (every exponent, inf, nan); see df_from_double.
static __device__ __noinline__ df df_from_double_slow(double d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(d);
  unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  unsigned sign = h32 & 0x80000000u;
  int e = (int)((h32 >> 20) & 0x7ffu);
  int ef = e - 896;  // float biased exponent
  unsigned mh = ((h32 & 0xfffffu) << 3) | (l32 >> 29);
  df r;
  if (ef >= 255) {  // overflow / inf / nan
    r.hi = __uint_as_float(sign | 0x7f800000u | (e == 0x7ff && ((h32 & 0xfffffu) | l32) ? 0x400000u : 0u));
    r.lo = 0.0f;
    return r;
  }
  if (ef < 1) {
    // below FP32's normal range: the nearest FP32 value (subnormal, or zero below ~1.4e-45), so
    // that a source of tiny magnitude stays visible to the z solve's range report
    r.hi = __double2float_rn(d);
    r.lo = 0.0f;
    return r;
  }
  r.hi = __uint_as_float(sign | ((unsigned)ef << 23) | mh);
  if (ef >= 24) {
    unsigned base = sign | ((unsigned)(ef - 23) << 23);
    r.lo = __fsub_rn(__uint_as_float(base | ((l32 & 0x1fffffffu) >> 6)), __uint_as_float(base));
  } else {
    r.lo = 0.0f;
  }
  return r;
}

// Split an FP64 value into hi + lo (hi = truncated 24-bit significand, lo = the next 23 bits),
// using integer operations only.  |d| < 2^-103 keeps only hi; |d| < 2^-126 becomes the nearest
// FP32 subnormal (zero below 2^-150).
__device__ __forceinline__ df df_from_double(double d) {
  const unsigned h32 = (unsigned)__double2hiint(d), l32 = (unsigned)__double2loint(d);
  const unsigned sign = h32 & 0x80000000u;
  const unsigned t = (h32 & 0x7fffffffu) - (896u << 20);
  if (t - (24u << 20) >= (231u << 20)) return df_from_double_slow(d);  // e_f outside [24, 254]
  df r;
  r.hi = __uint_as_float(sign | __funnelshift_l(l32, t, 3));
  // lo: the 23 bits below hi's last place, as (2^(e_f-23) (1 + m/2^23)) - 2^(e_f-23)
  const unsigned base = sign | ((t - (23u << 20)) >> 20 << 23);
  r.lo = __fsub_rn(__uint_as_float(base | ((l32 & 0x1fffffffu) >> 6)), __uint_as_float(base));
  return r;
}

// FP32 -> FP64, exact, integer operations only.
__device__ __forceinline__ double double_from_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned a = u & 0x7fffffffu;
  if (a - 0x00800000u < 0x7f000000u)  // normal: 1 <= e_f <= 254
    return __hiloint2double((int)((u & 0x80000000u) | ((a >> 3) + (896u << 20))), (int)(u << 29));
  unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (a == 0) return __longlong_as_double((long long)sign);
  if (a < 0x00800000u) {
    // subnormal a 2^-149: shift the leading one to bit 23; the exponent drops by the shift
    const int sh = __clz((int)a) - 8;
    const unsigned m = (a << sh) & 0x7fffffu;
    return __longlong_as_double((long long)(sign | ((unsigned long long)(897 - sh) << 52) | ((unsigned long long)m << 29)));
  }
  return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull | ((u & 0x7fffffu) ? 0x8000000000000ull : 0ull)));
}

// hi + lo as the nearest FP64 value: both parts are exact in FP64, one FP64 add.  hi is widened
// with integer bit operations, lo by the FP64 unit's conversion: the FP64 unit runs beside the
// FP32 and integer pipes, and in the issue-bound kernels that write FP64 (measured: x-inverse
// 8.06 -> 7.77 ms at 1024^3) moving one conversion onto it is cheaper than issuing its integer ops.
__device__ __forceinline__ double df_to_double(df v) {
  return __dadd_rn(double_from_f32(v.hi), (double)v.lo);
}

// General-case FP64 -> FP32 (zeros, subnormal results, overflow, inf, nan): the hardware
// conversion, round to nearest even (the FP64-rate unit; this path is rare).
static __device__ __noinline__ float f32_from_double_slow(double d) { return __double2float_rn(d); }

// FP64 -> FP32 rounded to nearest, integer operations only.  Ties round away from zero on the
// normal-range path (a tie needs the 29 discarded bits to be exactly 1000...0; both neighbours are
// half an ulp away).
__device__ __forceinline__ float f32_from_double(double d) {
  const unsigned h32 = (unsigned)__double2hiint(d), l32 = (unsigned)__double2loint(d);
  const unsigned t = (h32 & 0x7fffffffu) - (896u << 20);
  if (t - (1u << 20) >= (254u << 20)) return f32_from_double_slow(d);  // e_f outside [1, 254]
  // rounding carries propagate into the exponent (254 with all ones rounds to inf, as it should)
  const unsigned mag = __funnelshift_l(l32, t, 3) + ((l32 >> 28) & 1u);
  return __uint_as_float((h32 & 0x80000000u) | mag);
}

__device__ __forceinline__ float df_to_f32(df v) { return __fadd_rn(v.hi, v.lo); }

// ------------------------------------------------------------- scalar traits
template <class R> struct Ar;
template <> struct Ar<float> {
  __device__ static __forceinline__ float add(float a, float b) { return a + b; }
  __device__ static __forceinline__ float sub(float a, float b) { return a - b; }
  __device__ static __forceinline__ float mul(float a, float b) { return a * b; }
  __device__ static __forceinline__ float neg(float a) { return -a; }
  __device__ static __forceinline__ float half(float a) { return 0.5f * a; }
  __device__ static __forceinline__ float zero() { return 0.0f; }
  __device__ static __forceinline__ float sqrt1_2() { return 0.70710678118654752f; }
  __device__ static __forceinline__ float sqrt3_2() { return 0.86602540378443865f; }
  __device__ static __forceinline__ float sqrt2() { return 1.41421356237309505f; }
  // complex product parts: a*b - c*d and a*b + c*d
  __device__ static __forceinline__ float dsub(float a, float b, float c, float d) { return fmaf(a, b, -c * d); }
  __device__ static __forceinline__ float dadd(float a, float b, float c, float d) { return fmaf(a, b, c * d); }
};
// The line transforms compute with the unnormalised forms (above); the z solve's recurrences
// use the normalised operators.
template <> struct Ar<df> {
  __device__ static __forceinline__ df add(df a, df b) { return add_u(a, b); }
  __device__ static __forceinline__ df sub(df a, df b) { return add_u(a, -b); }
  __device__ static __forceinline__ df mul(df a, df b) { return mul_u(a, b); }
  __device__ static __forceinline__ df neg(df a) { return -a; }
  __device__ static __forceinline__ df half(df a) { return df_half(a); }
  __device__ static __forceinline__ df zero() { return df{0.0f, 0.0f}; }
  // hi/lo splits of 1/sqrt(2), sqrt(3)/2 and sqrt(2)
  __device__ static __forceinline__ df sqrt1_2() { return df{0x1.6a09e6p-1f, 0x1.9fcef4p-27f}; }
  __device__ static __forceinline__ df sqrt3_2() { return df{0x1.bb67aep-1f, 0x1.0b0996p-26f}; }
  __device__ static __forceinline__ df sqrt2() { return df{0x1.6a09e6p+0f, 0x1.9fcef4p-26f}; }
  __device__ static __forceinline__ df dsub(df a, df b, df c, df d) { return dot2_sub_u(a, b, c, d); }
  __device__ static __forceinline__ df dadd(df a, df b, df c, df d) { return dot2_sub_u(a, b, -c, d); }
};

// ------------------------------------------------------------------ complex
template <class R> struct alignas(2 * sizeof(R)) cx {
  R re, im;
};
template <class R> __device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) {
  return {Ar<R>::add(a.re, b.re), Ar<R>::add(a.im, b.im)};
}
template <class R> __device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) {
  return {Ar<R>::sub(a.re, b.re), Ar<R>::sub(a.im, b.im)};
}
template <class R> __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return {Ar<R>::dsub(a.re, b.re, a.im, b.im), Ar<R>::dadd(a.re, b.im, a.im, b.re)};
}
// a * conj(b)
template <class R> __device__ __forceinline__ cx<R> cmulc(cx<R> a, cx<R> b) {
  return {Ar<R>::dadd(a.re, b.re, a.im, b.im), Ar<R>::dsub(a.im, b.re, a.re, b.im)};
}
template <class R> __device__ __forceinline__ cx<R> cconj(cx<R> a) { return {a.re, Ar<R>::neg(a.im)}; }
// multiply by -i (forward) or +i (inverse)
template <class R, bool INV> __device__ __forceinline__ cx<R> cmul_mi(cx<R> a) {
  if (INV) return {Ar<R>::neg(a.im), a.re};
  return {a.im, Ar<R>::neg(a.re)};
}
template <class R> __device__ __forceinline__ cx<R> chalf(cx<R> a) { return {Ar<R>::half(a.re), Ar<R>::half(a.im)}; }
template <class R> __device__ __forceinline__ cx<R> cscale(cx<R> a, R s) { return {Ar<R>::mul(a.re, s), Ar<R>::mul(a.im, s)}; }

// --------------------------------------------------------- storage <-> R
// Storage kinds: IO_F64 (double), IO_F32 (float), SP_DF (float2 hi/lo pair), SP_F32 (float).
template <class R, class S> struct Io;
// ld = cv(raw): raw() issues the load, cv() converts its bits.
template <> struct Io<df, double> {
  __device__ static __forceinline__ double raw(const double* p, long long i) { return __ldg(p + i); }
  __device__ static __forceinline__ df cv(double v) { return df_from_double(v); }
  __device__ static __forceinline__ df ld(const double* p, long long i) { return df_from_double(__ldg(p + i)); }
  __device__ static __forceinline__ void st(double* p, long long i, df v) { p[i] = df_to_double(v); }
};
template <> struct Io<df, float2> {
  __device__ static __forceinline__ float2 raw(const float2* p, long long i) { return __ldg(p + i); }
  __device__ static __forceinline__ df cv(float2 v) { return df{v.x, v.y}; }
  __device__ static __forceinline__ df ld(const float2* p, long long i) { float2 v = p[i]; return df{v.x, v.y}; }
  __device__ static __forceinline__ void st(float2* p, long long i, df v) { p[i] = make_float2(v.hi, v.lo); }
};
template <> struct Io<df, float> {
  __device__ static __forceinline__ float raw(const float* p, long long i) { return __ldg(p + i); }
  __device__ static __forceinline__ df cv(float v) { return df{v, 0.0f}; }
  __device__ static __forceinline__ df ld(const float* p, long long i) { return df{p[i], 0.0f}; }
  __device__ static __forceinline__ void st(float* p, long long i, df v) { p[i] = df_to_f32(v); }
};
template <> struct Io<float, double> {
  __device__ static __forceinline__ double raw(const double* p, long long i) { return __ldg(p + i); }
  __device__ static __forceinline__ float cv(double v) { return f32_from_double(v); }
  __device__ static __forceinline__ float ld(const double* p, long long i) { return f32_from_double(__ldg(p + i)); }
  // FP32 -> FP64 by the FP64 unit's exact conversion (measured faster than the integer widening here)
  __device__ static __forceinline__ void st(double* p, long long i, float v) { p[i] = (double)v; }
};
template <> struct Io<float, float> {
  __device__ static __forceinline__ float raw(const float* p, long long i) { return __ldg(p + i); }
  __device__ static __forceinline__ float cv(float v) { return v; }
  __device__ static __forceinline__ float ld(const float* p, long long i) { return p[i]; }
  __device__ static __forceinline__ void st(float* p, long long i, float v) { p[i] = v; }
};

}  // namespace pp

// df64.cuh — double-float ("float-float") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi) / 2, which carries a 48-bit significand in FP32's
// exponent range. GB300 issues 128 FP32 lanes per SM and clock against 2 FP64 lanes, so a
// double-float operation of 3-15 FP32 instructions is 4-20x cheaper than the native FP64 one.
//
// Error-free transformations (all with explicit round-to-nearest intrinsics, so the compiler
// cannot contract or reassociate them):
//   two_sum       s + e = a + b exactly                  (Knuth, TAOCP vol. 2, Sec. 4.2.2)
//   fast_two_sum  s + e = a + b exactly for |a| >= |b|   (Dekker 1971)
//   two_prod      p + e = a * b exactly, e from one FMA  (Dekker 1971, with a fused multiply-add)
// and from them the double-float add, multiply, multiply-add, reciprocal and square root in the
// form of Dekker (1971) and of Thall, "Extended-precision floating-point numbers for GPU
// computation" (2006). The add is Dekker's: its absolute error is a few units of 2^-48 (|x| + |y|),
// the same order as the inputs' own rounding, which is what differences of neighbour values in a
// stencil need. Reciprocal and square root take the FP32 result as seed and one Newton step
// r + r (1 - x r) (resp. s + (x - s^2) / (2 s)) with the residual evaluated exactly.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace pt {

struct __align__(8) df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // nearest double-float to a double: hi = fl32(x), lo = fl32(x - hi)
  __host__ __device__ constexpr explicit df64(double x)
      : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

namespace dfd {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ df64 renorm(float s, float e) {
  float h, l;
  fast_two_sum(s, e, h, l);
  return df64(h, l);
}

}  // namespace dfd

__device__ __forceinline__ df64 operator-(df64 x) { return df64(-x.hi, -x.lo); }

__device__ __forceinline__ df64 operator+(df64 x, df64 y) {
  float s, e;
  dfd::two_sum(x.hi, y.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
  return dfd::renorm(s, e);
}
__device__ __forceinline__ df64 operator-(df64 x, df64 y) { return x + (-y); }

__device__ __forceinline__ df64 operator*(df64 x, df64 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return dfd::renorm(p, e);
}
// a * b + c with one renormalisation (the FP64 / FP32 fma stay visible next to it)
using ::fma;
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  dfd::two_sum(p, c.hi, s, t);
  t = __fadd_rn(t, __fadd_rn(e, c.lo));
  return dfd::renorm(s, t);
}
__device__ __forceinline__ df64& operator+=(df64& x, df64 y) { return x = x + y; }
__device__ __forceinline__ df64& operator-=(df64& x, df64 y) { return x = x - y; }

// Comparisons of normalised values (|lo| <= ulp(hi) / 2): lexicographic on (hi, lo).
__device__ __forceinline__ bool operator<(df64 x, df64 y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }
__device__ __forceinline__ bool operator>(df64 x, df64 y) { return y < x; }
__device__ __forceinline__ bool operator==(df64 x, df64 y) { return x.hi == y.hi && x.lo == y.lo; }

// x * 2^k for a power of two given as a float (exact, both parts scaled)
__device__ __forceinline__ df64 scale2(df64 x, float pow2) { return df64(x.hi * pow2, x.lo * pow2); }

// 1 / x: FP32 correctly rounded seed r, then r + r d with d = 1 - x r from the exact product
// x.hi r = p + q (|d| <= 2^-24, relative error ~2^-46).
__device__ __forceinline__ df64 df_rcp(df64 x) {
  const float r = __frcp_rn(x.hi);
  const float p = __fmul_rn(x.hi, r);
  float q = __fmaf_rn(x.hi, r, -p);
  q = __fmaf_rn(x.lo, r, q);
  const float d = __fsub_rn(__fsub_rn(1.0f, p), q);   // 1 - p is exact (p within an ulp of 1)
  return dfd::renorm(r, __fmul_rn(r, d));
}

// sqrt(x), x >= 0: FP32 correctly rounded seed s, then s + (x - s^2) / (2 s) with s^2 exact.
__device__ __forceinline__ df64 df_sqrt(df64 x) {
  if (!(x.hi > 0.0f)) return df64(sqrtf(x.hi), 0.0f);   // 0 stays 0, a negative gives NaN
  const float s = __fsqrt_rn(x.hi);
  const float p = __fmul_rn(s, s);
  const float q = __fmaf_rn(s, s, -p);
  const float d = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), q), x.lo);   // x - s^2
  return dfd::renorm(s, __fmul_rn(d, __fdividef(0.5f, s)));
}

// x^(1/m) for an integer m >= 2, x > 0: Newton's iteration y <- y + y (x - y^m) / (m y^m) on
// y^m = x from an FP32 seed, twice (the seed's ~2^-21 error becomes ~m (2^-21)^2 and then
// falls below the double-float rounding).
__device__ __forceinline__ df64 df_pow_m(df64 y, int m) {
  df64 r(1.0f, 0.0f), b = y;
  for (int e = m; e > 0; e >>= 1) {          // square and multiply
    if (e & 1) r = r * b;
    if (e > 1) b = b * b;
  }
  return r;
}
__device__ __forceinline__ df64 df_root(df64 x, int m) {
  df64 y(exp2f(log2f(x.hi) / (float)m), 0.0f);
  for (int s = 0; s < 2; ++s) {
    const df64 ym = df_pow_m(y, m);
    const df64 d = x - ym;                      // small: evaluated in double-float
    const float corr = __fdividef(__fmul_rn(d.hi, y.hi), __fmul_rn((float)m, ym.hi));
    y = y + df64(corr, 0.0f);
  }
  return y;
}

}  // namespace pt

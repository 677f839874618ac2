// Double-float arithmetic on the FP32 pipe: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits (relative
// precision ~2^-47 per operation) and FP32's exponent range. GB300 issues FP32 at 64
// times its FP64 rate, so an algorithm that needs more than FP32's 24 bits but not
// FP64's 53 runs several times faster here than in FP64, even at 10-20 FP32
// instructions per operation.
//
// Building blocks (error-free transformations): Knuth's TwoSum (s + e = a + b exactly),
// Dekker's FastTwoSum (the same for |a| >= |b|) and the FMA-based TwoProd
// (p + e = a b exactly). The operations are the double-word algorithms analysed by
// Joldes, Muller and Popescu (ACM TOMS 44, 2017): the accurate sum of two double words
// (relative error <= 3u^2, u = 2^-24), the product of a double word by a word or by a
// double word (<= 2u^2 / 5u^2), and division and square root by one Newton correction
// of an FP32 estimate. Every product that feeds an error-free transformation is
// written with __fmul_rn or fmaf so that the compiler cannot contract it into a
// neighbouring addition.
#pragma once

namespace mem {

struct df {
  float hi, lo;
  __host__ __device__ df() : hi(0.f), lo(0.f) {}
  __host__ __device__ df(float h) : hi(h), lo(0.f) {}
  __host__ __device__ df(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df(s, e);
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df(p, fmaf(a, b, -p));
}

// nearest double word to an FP64 value (inputs of the FP64 test entry point)
__host__ __device__ inline df df_from_double(double d) {
  const float h = (float)d;
  return df(h, (float)(d - (double)h));
}
__host__ __device__ inline double to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }

// Out of line: the sum is the most frequent operation (20 instructions), and inlined at
// every use it made the solver's code outgrow the instruction cache (warps stalled on
// instruction fetch); one call per sum measured 1.4x faster in the dilepton integrand.
static __device__ __noinline__ df operator+(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator+(df a, float b) {
  const df s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ df operator+(float a, df b) { return b + a; }
__device__ __forceinline__ df operator-(df a, float b) { return a + (-b); }
__device__ __forceinline__ df operator-(float a, df b) { return (-b) + a; }

__device__ __forceinline__ df operator*(df a, float b) {
  const df p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}
__device__ __forceinline__ df operator*(float a, df b) { return b * a; }

__device__ __forceinline__ df operator*(df a, df b) {
  const df p = two_prod(a.hi, b.hi);
  const float t = fmaf(a.lo, b.hi, __fmul_rn(a.hi, b.lo));
  return fast_two_sum(p.hi, __fadd_rn(p.lo, t));
}

// a b + c
__device__ __forceinline__ df df_fma(df a, df b, df c) { return a * b + c; }

// quotient: an FP32 estimate q1 = a / b, the remainder a - q1 b in double-word
// arithmetic (it cancels to ~u |a|), and one correction
__device__ __forceinline__ df operator/(df a, df b) {
  const float r = __frcp_rn(b.hi);
  const float q1 = __fmul_rn(a.hi, r);
  const df rem = a - b * q1;
  return fast_two_sum(q1, __fmul_rn(rem.hi, r));
}
__device__ __forceinline__ df operator/(float a, df b) { return df(a) / b; }
__device__ __forceinline__ df operator/(df a, float b) { return a / df(b); }

// square root (0 for a <= 0): an FP32 estimate s and one Newton correction from the
// double-word residual a - s^2
__device__ __forceinline__ df df_sqrt(df a) {
  if (!(a.hi > 0.f)) return df(0.f);
  const float s = __fsqrt_rn(a.hi);
  const df res = a - two_prod(s, s);
  return fast_two_sum(s, __fdiv_rn(res.hi, __fmul_rn(2.f, s)));
}

// multiplication by a power of two is exact
__device__ __forceinline__ df df_ldexp(df a, float pow2) { return df(a.hi * pow2, a.lo * pow2); }

__device__ __forceinline__ df df_abs(df a) { return a.hi < 0.f ? -a : a; }

// ordering of normalised double words: by hi, then by lo
__device__ __forceinline__ bool operator<(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df a, df b) { return b < a; }
__device__ __forceinline__ bool operator<=(df a, df b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(df a, df b) { return !(a < b); }

}  // namespace mem

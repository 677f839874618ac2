// Range-restricted angle functions of the Breit-Wigner maps: atan2(y, x) for
// y > 0 and sin(a) for a in [0, pi], the only ranges the maps produce. Own
// polynomial approximations: atan(t) = t P(t^2) on [0, 1] (odd terms to t^19)
// and sin(x) = x Q(x^2) on [0, pi/2] (odd terms to x^9), coefficients from a
// relative least-squares fit on Chebyshev nodes in float64
// (paper_1407_7595_gb300/fit_poly.py; fit errors 2.6e-9 and 6.1e-9, below FP32
// rounding). Both keep full relative precision near their zeros, where the maps
// need it.
#pragma once
#include <cmath>

namespace mem {

constexpr float F_PI_HI = 3.14159274101257324f;      // float(pi)
constexpr float F_PI_LO = -8.74227766e-08f;          // pi - float(pi)
constexpr float F_HALF_PI = 1.57079637050628662f;

// atan(t), t in [0, 1]
__host__ __device__ __forceinline__ float atan_unit(float t) {
  const float t2 = t * t;
  float p = -1.770786066e-03f;
  p = fmaf(p, t2, +1.081130988e-02f);
  p = fmaf(p, t2, -3.098250514e-02f);
  p = fmaf(p, t2, +5.775726431e-02f);
  p = fmaf(p, t2, -8.391357443e-02f);
  p = fmaf(p, t2, +1.094781763e-01f);
  p = fmaf(p, t2, -1.426332178e-01f);
  p = fmaf(p, t2, +1.999844292e-01f);
  p = fmaf(p, t2, -3.333329336e-01f);
  p = fmaf(p, t2, +9.999999989e-01f);
  return t * p;
}

// atan2(y, x) for y > 0: the angle of (x, y) in (0, pi).
__host__ __device__ __forceinline__ float atan2_ypos(float y, float x) {
  const float ax = fabsf(x);
  const bool steep = y > ax;
  const float r = atan_unit((steep ? ax : y) / (steep ? y : ax));
  const float a = steep ? F_HALF_PI - r : r;   // angle of (|x|, y)
  return x >= 0.f ? a : (F_PI_HI - a) + F_PI_LO;
}

// sin(a), a in [0, pi]: sin(a) = sin(pi - a) folds the upper half onto [0, pi/2].
__host__ __device__ __forceinline__ float sin_0pi(float a) {
  const float b = a > F_HALF_PI ? (F_PI_HI - a) + F_PI_LO : a;
  const float b2 = b * b;
  float q = 2.605090005e-06f;
  q = fmaf(q, b2, -1.980914983e-04f);
  q = fmaf(q, b2, +8.333055963e-03f);
  q = fmaf(q, b2, -1.666665863e-01f);
  q = fmaf(q, b2, +9.999999976e-01f);
  return b * q;
}

// tanh(x) to ~1e-6 relative (the bounded scale of the learned sampler's
// couplings): below |x| = 1/4 the odd Taylor polynomial to x^7 (truncation
// 62 x^9 / 2835 < 1e-7 |x| there); above it (1 - e) / (1 + e) with
// e = exp(-2|x|) <= exp(-1/2), which has no cancellation in 1 - e.
__host__ __device__ __forceinline__ float tanh_coupling(float x) {
  const float a = fabsf(x);
  const float x2 = x * x;
  const float poly = x * fmaf(x2, fmaf(x2, fmaf(x2, -17.f / 315.f, 2.f / 15.f), -1.f / 3.f), 1.f);
#ifdef __CUDA_ARCH__
  const float e = __expf(-2.f * a);
#else
  const float e = expf(-2.f * a);
#endif
  const float big = copysignf((1.f - e) / (1.f + e), x);
  return a < 0.25f ? poly : big;
}

}  // namespace mem

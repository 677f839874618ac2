// Device building blocks of the integrand kernels: counter-based generator,
// VEGAS map, compensated sums and numerically stable FP32 change-of-variable
// primitives. Part of libmem.so (GB300, sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mem_fastmath.cuh"

namespace mem {

constexpr int NG = 128;          // VEGAS bins per dimension
constexpr int MAXD = 8;          // maximum integration dimensions
constexpr int REC = 32;          // floats per event record
constexpr float PI_F = 3.14159265358979f;
constexpr double PI_D = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): random points of the
// Monte Carlo sum (Sec. 2, Eq. "sum"). Counter = (point index, draw block << 8
// | stream tag, event id, permutation), key = (seed lo, seed hi).
// ---------------------------------------------------------------------------
struct u32x4 { uint32_t a, b, c, d; };

// The key schedule of all 10 rounds (key + r x the Weyl constants), built once
// on the host and passed to the kernels as a __grid_constant__ parameter, so
// that each round's key is a constant-bank operand of its XOR.
struct PhiloxKey {
  uint32_t k0[10], k1[10];
};

__host__ __device__ inline PhiloxKey philox_key(uint64_t seed) {
  PhiloxKey k;
  uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    k.k0[r] = a;
    k.k1[r] = b;
    a += 0x9E3779B9u;
    b += 0xBB67AE85u;
  }
  return k;
}

__device__ __forceinline__ u32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                               uint32_t c3, const PhiloxKey& key) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    c0 = hi1 ^ c1 ^ key.k0[r];
    c1 = lo1;
    c2 = hi0 ^ c3 ^ key.k1[r];
    c3 = lo0;
  }
  return {c0, c1, c2, c3};
}

// Uniform in (0,1) from 23 random bits: ((x >> 9) + 0.5) 2^-23 = (2k+1) 2^-24,
// exactly representable in FP32 on all of (0,1).
__device__ __forceinline__ float u01(uint32_t x) {
  return __uint2float_rn((x >> 9) * 2u + 1u) * 5.9604644775390625e-08f;
}

// Stream tags (low byte of counter word 1): 0 = points on the VEGAS grid,
// 2 = base draws of the learned sampler.
constexpr uint32_t TAG_VEGAS = 0, TAG_FLOW = 2;

template <int D>
__device__ __forceinline__ void point_uniforms(const PhiloxKey& key, uint32_t event_id,
                                               uint32_t perm, uint32_t idx, float (&u)[D],
                                               uint32_t tag = TAG_VEGAS) {
#pragma unroll
  for (int b = 0; b < (D + 3) / 4; ++b) {
    u32x4 o = philox4x32_10(idx, ((uint32_t)b << 8) | tag, event_id, perm, key);
    if (4 * b + 0 < D) u[4 * b + 0] = u01(o.a);
    if (4 * b + 1 < D) u[4 * b + 1] = u01(o.b);
    if (4 * b + 2 < D) u[4 * b + 2] = u01(o.c);
    if (4 * b + 3 < D) u[4 * b + 3] = u01(o.d);
  }
}

// ---------------------------------------------------------------------------
// VEGAS map (Sec. 2; Lepage 1978). The FP32 device copy stores, per bin, the
// left edge, the width and the complement of the right edge, each rounded once
// from the FP64 master: narrow bins keep full relative precision in the
// Jacobian NG * width, and both x and 1 - x come out with full relative
// precision (maps that are steep near x = 1 use the complement).
// ---------------------------------------------------------------------------
struct __align__(16) GridBin { float x0, w, xc, pad; };

template <int D>
__device__ __forceinline__ float vegas_map(const GridBin* __restrict__ g, const float (&u)[D],
                                           float (&x)[D], float (&xc)[D], int (&bin)[D]) {
  float J = 1.f;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const float t = u[j] * (float)NG;  // exact: u = (2k+1) 2^-24, NG a power of two
    int i = (int)t;
    i = i > NG - 1 ? NG - 1 : i;
    const GridBin b = g[j * NG + i];
    x[j] = fmaf(t - (float)i, b.w, b.x0);
    xc[j] = fmaf((float)(i + 1) - t, b.w, b.xc);  // (i+1) - t is exact
    J *= (float)NG * b.w;
    bin[j] = i;
  }
  return J;
}

// ---------------------------------------------------------------------------
// Compensated accumulation: Kahan (1965) per thread in FP32; the 32 lanes of a
// warp are merged as double-float pairs (Knuth's TwoSum in FP32, error-free in
// the high parts; ~2^-44 relative), the warps of a CTA with TwoSum in FP64.
// (FP64 runs at a small fraction of the FP32 rate on this part: a warp-level
// FP64 butterfly cost ~60 FP64 operations per thread per CTA.)
// ---------------------------------------------------------------------------
struct Kahan32 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

struct DD { double hi, lo; };

__device__ __forceinline__ DD two_sum_merge(DD a, DD b) {
  const double s = a.hi + b.hi;
  const double bb = s - a.hi;
  const double err = (a.hi - (s - bb)) + (b.hi - bb);
  return {s, err + a.lo + b.lo};
}

struct FF { float hi, lo; };  // unevaluated sum hi + lo

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);  // s + e = a.hi + b.hi exactly
  const float t = e + (a.lo + b.lo);
  const float h = s + t;
  return {h, t - (h - s)};
}

// Warp sum of the lanes' Kahan states (s - c), valid in every lane, as an FP64
// double-word for the CTA merge.
__device__ __forceinline__ DD warp_reduce_kahan(const Kahan32& k) {
  FF v = {k.s, -k.c};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    FF w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = ff_add(v, w);
  }
  return {(double)v.hi, (double)v.lo};
}

// ---------------------------------------------------------------------------
// Stable FP32 primitives
// ---------------------------------------------------------------------------
// exp(a) - 1 for |a| <= 0.35 by its Taylor series (11 terms, truncation
// below 1e-12 relative); used where a difference of exponentials would cancel.
__device__ __forceinline__ float expm1_small(float a) {
  float p = 1.f / 39916800.f;
  p = fmaf(p, a, 1.f / 3628800.f);
  p = fmaf(p, a, 1.f / 362880.f);
  p = fmaf(p, a, 1.f / 40320.f);
  p = fmaf(p, a, 1.f / 5040.f);
  p = fmaf(p, a, 1.f / 720.f);
  p = fmaf(p, a, 1.f / 120.f);
  p = fmaf(p, a, 1.f / 24.f);
  p = fmaf(p, a, 1.f / 6.f);
  p = fmaf(p, a, 0.5f);
  p = fmaf(p, a, 1.f);
  return p * a;
}

// Breit-Wigner change of variables q^2 = m^2 + m G tan(theta), theta uniform
// over [theta_lo, theta_hi] <-> q^2 in [lo, hi] (Sec. 3: propagator
// virtualities as integration variables). Written with the complements
// psi_lo = pi/2 + theta_lo, psi_hi = pi/2 - theta_hi so that q^2 - lo, cos(theta)
// and the Jacobian keep full FP32 relative precision from the resonance peak
// to the far tails:
//   q^2 - lo = m G sin(R v) / (sin(psi_lo + R v) sin(psi_lo)),  R = theta_hi - theta_lo
//   dq^2/dv = R m G / cos^2(theta)   and   (dq^2/dv) / |q^2 - m^2 + i m G|^2 = R / (m G).
struct BW {
  float q2;      // mapped virtuality
  float d_lo;    // q^2 - lo (no cancellation)
  float R;       // theta range
  float inv_c2;  // 1 / cos^2(theta)
};

// psi_hi = atan2(m G, hi - m^2) is passed in (it is a constant when hi is).
__device__ __forceinline__ BW bw_map(float lo, float hi_minus_lo, float m2, float mg, float v,
                                     float w /* = 1 - v, exact */, float psi_hi) {
  const float hi = lo + hi_minus_lo;
  const float psi_lo = atan2_ypos(mg, m2 - lo);
  const float R = atan2_ypos(hi_minus_lo * mg, fmaf(hi - m2, lo - m2, mg * mg));
  const float a_lo = fmaf(R, v, psi_lo);  // pi/2 + theta
  const float a_hi = fmaf(R, w, psi_hi);  // pi/2 - theta
  const float c = sin_0pi(a_lo <= a_hi ? a_lo : a_hi);  // cos(theta)
  const float s_lo = mg * rsqrtf(fmaf(m2 - lo, m2 - lo, mg * mg));  // sin(psi_lo)
  BW r;
  r.d_lo = mg * sin_0pi(R * v) / (c * s_lo);
  r.q2 = lo + r.d_lo;
  r.R = R;
  r.inv_c2 = 1.f / (c * c);
  return r;
}

// Double-word FP64 partials stored per (item, chunk) slot.
struct Slot {
  double s1, c1, s2, c2;  // sum w (hi, lo), sum w^2 (hi, lo)
  uint32_t n_bad;         // non-finite weights skipped
  uint32_t pad;
};

}  // namespace mem

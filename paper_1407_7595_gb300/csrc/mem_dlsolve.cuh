// The two-neutrino solution of the dilepton final states (Sec. 3, Eq. "dilepsolv"),
// shared by the dilepton ttbar, ttH and ttbb integrands and the solver's test entry
// point: given the massless b, bbar, l+, mu- momenta, the missing transverse momentum
// and the four virtualities q^2(W+), q^2(W-), q^2(t), q^2(tbar), every real neutrino
// pair (nu, nubar) with those invariants, and the Jacobian
// 1 / |det d(q^2_W+, q^2_t, q^2_W-, q^2_tbar) / d(nu_x, nu_y, nu_z, nubar_z)|.
//
// Method: l.nu and b.nu fix the neutrino's energy and p_z as affine functions of
// (p_x, p_y) (likewise for the antineutrino in its own transverse momentum, which is
// the missing pT minus the neutrino's); the two mass shells are then conics in the
// neutrino's (p_x, p_y), and their common points are the real roots x of the
// resultant quartic in x, with y from the two conics' common linear combination.
//
// Precision: double-float (mem_df.cuh, ~48 bits on the FP32 pipe). The resultant's
// coefficients are products of four conic coefficients and cancel by several orders
// of magnitude, beyond FP32's 24 bits; 48 bits keep them to ~1e-9 or better where
// FP64 would keep ~1e-11, far below the FP32 rounding (~1e-7) of the virtualities
// and energies the integrand feeds in. Search steps that only bracket or start a root
// (the derivative chain's critical points, the root locations) run in FP32. Momenta
// are in units of DL_UNIT = 128 GeV (a power of two: scaling is exact).
//
// Real roots of the quartic: every real root of a polynomial lies between two
// consecutive real roots of its derivative (Rolle), so the roots of the linear,
// quadratic and cubic derivatives bracket those of the quartic, whose signs at the
// bracket ends are taken in double-float; each root is located in FP32 and finished by
// double-float Newton steps, then polished on the two conics (Newton in 2D).
#pragma once
#include "mem_df.cuh"
#include "mem_ttbar.cuh"   // LCv, C()

namespace mem {

constexpr float DL_UNIT = 128.f;
constexpr float DL_IU = 1.f / 128.f;

// massless momentum (E, p_x, p_y, p_z) in units of DL_UNIT
struct DLMom { df v[4]; };

// from an FP32 energy and FP32 direction cosines: E / DL_UNIT is exact and each
// component E n_k is an exact double-float product
__device__ __forceinline__ DLMom dl_mom(float E, float nx, float ny, float nz) {
  const float e = E * DL_IU;
  DLMom m;
  m.v[0] = df(e);
  m.v[1] = two_prod(e, nx);
  m.v[2] = two_prod(e, ny);
  m.v[3] = two_prod(e, nz);
  return m;
}

// from FP64 components in GeV (the solver's test entry point)
__device__ __forceinline__ DLMom dl_mom64(const double* p) {
  DLMom m;
  for (int k = 0; k < 4; ++k) m.v[k] = df_from_double(p[k] / (double)DL_UNIT);
  return m;
}

__device__ __forceinline__ df dl_dot(const DLMom& a, const DLMom& b) {
  return a.v[0] * b.v[0] - a.v[1] * b.v[1] - a.v[2] * b.v[2] - a.v[3] * b.v[3];
}

// A conic q(x, y) = xx x^2 + xy x y + yy y^2 + x1 x + y1 y + c0.
struct DLConic { df xx, xy, yy, x1, y1, c0; };

__device__ __forceinline__ df dl_conic_at(const DLConic& q, df x, df y) {
  return df_fma(x, df_fma(q.xx, x, df_fma(q.xy, y, q.x1)), df_fma(y, df_fma(q.yy, y, q.y1), q.c0));
}

// Massless neutrino with lepton l and b quark: l.nu = A and b.nu = B fix E and p_z as
// affine functions of (p_x, p_y) -- E = e[0] + e[1] x + e[2] y, p_z = z[0] + z[1] x +
// z[2] y. Returns false when the two equations are degenerate in (E, p_z) (the lepton
// and the b share their p_z / E ratio).
struct DLAffine { df e[3], z[3]; };

__device__ __forceinline__ bool dl_affine(const DLMom& l, const DLMom& b, df A, df B, DLAffine& r) {
  // l0 E - lz pz = A + lx x + ly y ;  b0 E - bz pz = B + bx x + by y
  const df det = l.v[3] * b.v[0] - l.v[0] * b.v[3];
  if (!(fabsf(det.hi) > 1e-12f * (fabsf(l.v[0].hi * b.v[3].hi) + fabsf(l.v[3].hi * b.v[0].hi)) + 1e-30f))
    return false;
  const df id = 1.f / det;
  const df ra[3] = {A, l.v[1], l.v[2]}, rb[3] = {B, b.v[1], b.v[2]};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r.e[k] = (l.v[3] * rb[k] - b.v[3] * ra[k]) * id;
    r.z[k] = (l.v[0] * rb[k] - b.v[0] * ra[k]) * id;
  }
  return true;
}

// E^2 - x^2 - y^2 - p_z^2 of the affine neutrino, as a conic in (x, y).
__device__ __forceinline__ DLConic dl_shell(const DLAffine& a) {
  DLConic q;
  q.xx = a.e[1] * a.e[1] - a.z[1] * a.z[1] - 1.f;
  q.yy = a.e[2] * a.e[2] - a.z[2] * a.z[2] - 1.f;
  q.xy = df_ldexp(a.e[1] * a.e[2] - a.z[1] * a.z[2], 2.f);
  q.x1 = df_ldexp(a.e[0] * a.e[1] - a.z[0] * a.z[1], 2.f);
  q.y1 = df_ldexp(a.e[0] * a.e[2] - a.z[0] * a.z[2], 2.f);
  q.c0 = a.e[0] * a.e[0] - a.z[0] * a.z[0];
  return q;
}

// The antineutrino's conic in its own (X, Y), rewritten in the neutrino's (x, y)
// through X = mx - x, Y = my - y.
__device__ __forceinline__ DLConic dl_mirror(const DLConic& q, df mx, df my) {
  DLConic r;
  r.xx = q.xx;
  r.xy = q.xy;
  r.yy = q.yy;
  r.x1 = -df_fma(df_ldexp(q.xx, 2.f), mx, df_fma(q.xy, my, q.x1));
  r.y1 = -df_fma(df_ldexp(q.yy, 2.f), my, df_fma(q.xy, mx, q.y1));
  r.c0 = dl_conic_at(q, mx, my);
  return r;
}

// p(x) and p'(x) of c[0] + c[1] x + ... + c[deg] x^deg (Horner; FP32 or double-float)
template <class T>
__device__ __forceinline__ T dl_horner(const T* c, int deg, T x, T& dp) {
  T p = c[deg], d = T(0.f);
  for (int k = deg - 1; k >= 0; --k) {
    d = d * x + p;
    p = p * x + c[k];
  }
  dp = d;
  return p;
}

// FP32 root of the polynomial c (degree deg) in [a, b], where it changes sign
// (only the sign of fa is used): Newton steps, replaced by bisection whenever a
// step leaves the shrinking bracket, to FP32 resolution.
static __device__ __noinline__ float dl_bracket32(const float* c, int deg, float a, float b, float fa) {
  float x = 0.5f * (a + b);
#pragma unroll 1
  for (int it = 0; it < 64; ++it) {
    float dp;
    const float f = dl_horner(c, deg, x, dp);
    if (f == 0.f) return x;
    if ((f < 0.f) == (fa < 0.f)) a = x;
    else b = x;
    float xn = x - f / dp;
    if (!(xn > a && xn < b)) xn = 0.5f * (a + b);
    if (fabsf(xn - x) <= 2e-7f * (1.f + fabsf(x))) return xn;
    x = xn;
  }
  return x;
}

// Double-float root of c in [a, b] (a sign change, fa = c(a)) from the start x0, to
// |step| <= tol (1 + |x|): Newton steps that multiply by an FP32 reciprocal of the
// derivative (near the root the iteration then contracts by ~1e-7 per step, which from
// an FP32-accurate start is the same two steps), bisection whenever a step leaves the
// shrinking bracket.
static __device__ __noinline__ df dl_bracket_root(const df* c, int deg, df a, df b, df fa, df x0,
                                                  float tol) {
  df x = (x0 > a && x0 < b) ? x0 : df_ldexp(a + b, 0.5f);
#pragma unroll 1
  for (int it = 0; it < 96; ++it) {
    df dp;
    const df f = dl_horner(c, deg, x, dp);
    if (f.hi == 0.f) return x;
    if ((f.hi < 0.f) == (fa.hi < 0.f)) {
      a = x;
      fa = f;
    } else {
      b = x;
    }
    const float dpf = fabsf(dp.hi);
    df xn = df_ldexp(a + b, 0.5f);   // bisection unless the Newton step stays in the bracket
    if (dpf > 1e-30f && dpf < 1e30f) {
      const df t = x - f * (1.f / dp.hi);
      if (t > a && t < b) xn = t;
    }
    if (fabsf((xn - x).hi) <= tol * (1.f + fabsf(x.hi))) return xn;
    x = xn;
  }
  return x;
}

// Relative step at which the double-float Newton iterations stop. They divide by an
// FP32 reciprocal of the derivative, so near a simple root each step contracts the
// error by ~1e-7: after a step of 1e-11 the error left is ~1e-18, below double-float
// resolution. (Next to a double root, where the contraction is weaker, the roots are
// ill-conditioned at the 1e-7 level of the integrand's FP32 inputs anyway.)
constexpr float DL_DF_TOL = 1e-11f;

// p at a bracket end x, where only its sign matters unless it is small: the FP32
// monic copy cf (p = lead cf) decides when |cf(x)| exceeds 1e-5 of its terms (the
// copy's rounding and the FP32 evaluation stay below ~3e-7 of them); otherwise the
// double-float polynomial is evaluated. mag = sum_k |c_k| |x|^k.
__device__ __forceinline__ df dl_end_value(const df* c, const float* cf, int deg, float lead, df x,
                                           float& mag) {
  const float ax = fabsf(x.hi);
  float m = 0.f, pw = 1.f;
  for (int k = 0; k <= deg; ++k, pw *= ax) m = fmaf(fabsf(cf[k]), pw, m);
  mag = m * fabsf(lead);
  float dp32;
  const float p32 = dl_horner(cf, deg, x.hi, dp32);
  if (fabsf(p32) > 1e-5f * m) return df(p32 * lead);
  df dp;
  return dl_horner(c, deg, x, dp);
}

// Real roots (ascending) of c[0] + c[1] x + ... + c[deg] x^deg, 1 <= deg <= 4,
// c[deg] != 0. The critical points -- the real roots of the derivative chain
// (linear, quadratic in closed form, cubic by bracketed Newton) -- are found in FP32
// on the monic polynomial: they only separate the roots. Which intervals between them
// hold a root is decided by the signs of the double-float polynomial at their ends (at
// a critical point the polynomial is flat, so an FP32-accurate location gives the
// exact sign, except next to a double root: see below); each root is located in FP32
// and finished by double-float Newton steps inside its bracket. Where the polynomial is
// far from zero at a bracket end, the FP32 copy gives its sign (dl_end_value). A
// critical point where the polynomial vanishes to rounding is a double root and is
// kept once.
static __device__ __noinline__ int dl_real_roots(const df* c, int deg, df* roots) {
  const float lead = c[deg].hi;
  const float ilead = 1.f / lead;
  float cf[5];
  float bound = 0.f;
  for (int k = 0; k < deg; ++k) {
    cf[k] = c[k].hi * ilead;
    bound = fmaxf(bound, fabsf(cf[k]));
  }
  cf[deg] = 1.f;
  bound += 1.f;   // Cauchy bound on every root and critical point (Gauss-Lucas)
  float crit[3];
  int ncrit = 0;
#pragma unroll 1
  for (int m = deg - 1; m >= 1; --m) {
    // level m: the m-th derivative, degree deg - m <= 3
    const int dm = deg - m;
    float d[4];
    for (int k = 0; k <= dm; ++k) {
      float f = cf[k + m];
      for (int j = k + 1; j <= k + m; ++j) f *= (float)j;   // (k+m)! / k!
      d[k] = f;
    }
    float out[3];
    int n = 0;
    if (dm == 1) {
      out[n++] = -d[0] / d[1];
    } else if (dm == 2) {
      const float disc = d[1] * d[1] - 4.f * d[2] * d[0];
      if (disc >= 0.f) {
        const float q = -0.5f * (d[1] + copysignf(sqrtf(disc), d[1]));
        float r1 = q / d[2], r2 = q != 0.f ? d[0] / q : r1;
        if (r1 > r2) {
          const float t = r1;
          r1 = r2;
          r2 = t;
        }
        out[n++] = r1;
        if (r2 > r1) out[n++] = r2;
      }
    } else {
      float a = -bound, dpa;
      float fa = dl_horner(d, dm, a, dpa);
      for (int i = 0; i <= ncrit; ++i) {
        const float b = i < ncrit ? fminf(fmaxf(crit[i], -bound), bound) : bound;
        float dpb;
        const float fb = dl_horner(d, dm, b, dpb);
        if (b > a && ((fa < 0.f && fb > 0.f) || (fa > 0.f && fb < 0.f)))
          out[n++] = dl_bracket32(d, dm, a, b, fa);
        a = b;
        fa = fb;
        if (n >= dm) break;
      }
    }
    ncrit = n;
    for (int k = 0; k < n; ++k) crit[k] = out[k];
  }
  // level 0: double-float signs at the bracket ends, FP32 location, double-float finish
  int n = 0;
  const df B(bound);
  df a = -B;
  float mag_a;
  df fa = dl_end_value(c, cf, deg, lead, a, mag_a);
  // derivative coefficients for refining critical points next to a double root
  df c1[4];
  for (int k = 0; k < deg; ++k) c1[k] = c[k + 1] * (float)(k + 1);
  for (int i = 0; i <= ncrit; ++i) {
    df b = i < ncrit ? df(fminf(fmaxf(crit[i], -bound), bound)) : B;
    df dpb;
    float mag;
    df fb = dl_end_value(c, cf, deg, lead, b, mag);
    if (i < ncrit && deg >= 2 && fabsf(fb.hi) <= 1e-6f * mag) {
      // Where the polynomial is small at a critical point, two roots may lie closer
      // together than the FP32 critical point's error, which would put both on one
      // side of it and lose them: move it to double-float accuracy (Newton on p').
      const df hi = i + 1 < ncrit ? df(fminf(fmaxf(crit[i + 1], -bound), bound)) : B;
#pragma unroll 1
      for (int it = 0; it < 4; ++it) {
        df d2p;   // p''(b), from the Horner pass over p'
        const df p1 = dl_horner(c1, deg - 1, b, d2p);
        if (!(d2p.hi != 0.f)) break;
        const df bn = b - p1 * (1.f / d2p.hi);
        if (!(bn > a && bn < hi)) break;
        const bool done = fabsf((bn - b).hi) <= DL_DF_TOL * (1.f + fabsf(b.hi));
        b = bn;
        if (done) break;
      }
      fb = dl_horner(c, deg, b, dpb);
    }
    if (b > a && ((fa.hi < 0.f && fb.hi > 0.f) || (fa.hi > 0.f && fb.hi < 0.f))) {
      // the monic FP32 copy has the sign of c times that of the leading coefficient
      const float sa = ((fa.hi < 0.f) != (lead < 0.f)) ? -1.f : 1.f;
      const float x0 = dl_bracket32(cf, deg, a.hi, b.hi, sa);
      roots[n++] = dl_bracket_root(c, deg, a, b, fa, df(x0), DL_DF_TOL);
    } else if (i < ncrit && (n == 0 || roots[n - 1] < b)) {
      // touches zero at the critical point: |p| at the rounding level of its terms
      // (a double-float Horner pass rounds at ~1e-14 of them)
      if (fabsf(fb.hi) <= 2e-12f * mag) roots[n++] = b;
    }
    a = b;
    fa = fb;
    if (n >= deg) break;
  }
  return n;
}

// Newton steps in (x, y) on the intersection of two conics, to a step of 1e-12
// relative (far below the FP32 that the solution feeds): residuals and gradients in
// double-float, the step through an FP32 reciprocal of the determinant.
__device__ __forceinline__ void dl_polish(const DLConic& p, const DLConic& q, df& x, df& y) {
#pragma unroll 1
  for (int it = 0; it < 4; ++it) {
    const df f = dl_conic_at(p, x, y), g = dl_conic_at(q, x, y);
    const df fx = df_fma(df_ldexp(p.xx, 2.f), x, df_fma(p.xy, y, p.x1));
    const df fy = df_fma(p.xy, x, df_fma(df_ldexp(p.yy, 2.f), y, p.y1));
    const df gx = df_fma(df_ldexp(q.xx, 2.f), x, df_fma(q.xy, y, q.x1));
    const df gy = df_fma(q.xy, x, df_fma(df_ldexp(q.yy, 2.f), y, q.y1));
    const df det = fx * gy - fy * gx;
    if (det.hi == 0.f) return;
    const float id = 1.f / det.hi;
    const df dx = (f * gy - g * fy) * id, dy = (g * fx - f * gx) * id;
    x = x - dx;
    y = y - dy;
    if (fabsf(dx.hi) + fabsf(dy.hi) < 1e-12f * (1.f + fabsf(x.hi) + fabsf(y.hi))) return;
  }
}

// The conics and the resultant quartic of one phase-space point (momenta in units of
// DL_UNIT, virtualities in DL_UNIT^2).
struct DLSystem {
  DLAffine n1, n2;       // neutrino (in its x, y) and antineutrino (in its X, Y)
  DLConic c1, c2;        // mass shells in the neutrino's (x, y)
  df u[3], v[2];         // y = -u(x) / v(x) on the common points
  df mx, my;             // missing transverse momentum
};

// Builds the system; returns the number of real roots x of the resultant (in xr).
// (mx, my): the missing pT, the negative visible pT sum of the event's own final state
// (dilepton ttbar adds the four objects; dilepton ttH and ttbb the extra pair too).
static __device__ __noinline__ int dl_system_met(const DLMom& b, const DLMom& bb, const DLMom& lp,
                                                 const DLMom& lm, df mx, df my, df q2wp, df q2wm,
                                                 df q2t, df q2tb, DLSystem& S, df* xr) {
  S.mx = mx;
  S.my = my;
  // 2 l.nu = q^2_W and 2 b.nu = q^2_t - q^2_W - 2 b.l (massless b, l, nu)
  const df blp = dl_dot(b, lp), bblm = dl_dot(bb, lm);
  if (!dl_affine(lp, b, df_ldexp(q2wp, 0.5f), df_ldexp(q2t - q2wp, 0.5f) - blp, S.n1)) return 0;
  if (!dl_affine(lm, bb, df_ldexp(q2wm, 0.5f), df_ldexp(q2tb - q2wm, 0.5f) - bblm, S.n2)) return 0;
  S.c1 = dl_shell(S.n1);
  S.c2 = dl_mirror(dl_shell(S.n2), S.mx, S.my);
  // each conic as a_i y^2 + (p_i + r_i x) y + (s_i + t_i x + w_i x^2)
  const DLConic& P = S.c1;
  const DLConic& Q = S.c2;
  const df a1 = P.yy, a2 = Q.yy;
  // u = a1 C2 - a2 C1 (quadratic), v = a1 B2 - a2 B1 (linear), w = B1 C2 - B2 C1 (cubic)
  S.u[0] = a1 * Q.c0 - a2 * P.c0;
  S.u[1] = a1 * Q.x1 - a2 * P.x1;
  S.u[2] = a1 * Q.xx - a2 * P.xx;
  S.v[0] = a1 * Q.y1 - a2 * P.y1;
  S.v[1] = a1 * Q.xy - a2 * P.xy;
  df w[4];
  w[0] = P.y1 * Q.c0 - Q.y1 * P.c0;
  w[1] = (P.y1 * Q.x1 - Q.y1 * P.x1) + (P.xy * Q.c0 - Q.xy * P.c0);
  w[2] = (P.y1 * Q.xx - Q.y1 * P.xx) + (P.xy * Q.x1 - Q.xy * P.x1);
  w[3] = P.xy * Q.xx - Q.xy * P.xx;
  // resultant in y: u^2 - v w
  df R[5];
  R[0] = S.u[0] * S.u[0] - S.v[0] * w[0];
  R[1] = df_ldexp(S.u[0] * S.u[1], 2.f) - (S.v[0] * w[1] + S.v[1] * w[0]);
  R[2] = (S.u[1] * S.u[1] + df_ldexp(S.u[0] * S.u[2], 2.f)) - (S.v[0] * w[2] + S.v[1] * w[1]);
  R[3] = df_ldexp(S.u[1] * S.u[2], 2.f) - (S.v[0] * w[3] + S.v[1] * w[2]);
  R[4] = S.u[2] * S.u[2] - S.v[1] * w[3];
  float scale = 0.f;
  for (int k = 0; k < 5; ++k) scale = fmaxf(scale, fabsf(R[k].hi));
  if (scale == 0.f) return 0;
  int deg = 4;
  while (deg > 0 && fabsf(R[deg].hi) <= 2e-12f * scale) --deg;
  if (deg == 0) return 0;
  return dl_real_roots(R, deg, xr);
}

// One neutrino solution from a root x of the resultant: y, conic polish, the residual
// and positive-energy checks. Returns false when the root is rejected.
static __device__ __noinline__ bool dl_point(const DLSystem& S, df xr, df& x, df& y) {
  const df num = -df_fma(df_fma(S.u[2], xr, S.u[1]), xr, S.u[0]);
  const df den = df_fma(S.v[1], xr, S.v[0]);
  if (fabsf(den.hi) > 1e-12f * (fabsf(num.hi) + 1.f)) {
    y = num / den;
  } else {
    // v vanishes: y from the first conic's quadratic, the branch on the second
    const df a = S.c1.yy, bq = df_fma(S.c1.xy, xr, S.c1.y1);
    const df cq = df_fma(df_fma(S.c1.xx, xr, S.c1.x1), xr, S.c1.c0);
    const df disc = bq * bq - df_ldexp(a * cq, 4.f);
    if (disc.hi < 0.f || a.hi == 0.f) return false;
    const df sd = df_sqrt(disc), ia = 0.5f / a;
    const df y1 = (sd - bq) * ia, y2 = -(bq + sd) * ia;
    y = fabsf(dl_conic_at(S.c2, xr, y1).hi) < fabsf(dl_conic_at(S.c2, xr, y2).hi) ? y1 : y2;
  }
  x = xr;
  dl_polish(S.c1, S.c2, x, y);
  const float tol = 1e-8f * (1.f + x.hi * x.hi + y.hi * y.hi);
  if (fabsf(dl_conic_at(S.c1, x, y).hi) > tol || fabsf(dl_conic_at(S.c2, x, y).hi) > tol) return false;
  const df E = S.n1.e[0] + S.n1.e[1] * x + S.n1.e[2] * y;
  const df X = S.mx - x, Y = S.my - y;
  const df Eb = S.n2.e[0] + S.n2.e[1] * X + S.n2.e[2] * Y;
  return E.hi > 0.f && Eb.hi > 0.f;
}

// The neutrino and antineutrino four-momenta of a solution (x, y) = nu_T.
static __device__ __noinline__ void dl_neutrinos(const DLSystem& S, df x, df y, DLMom& nu, DLMom& nub) {
  nu.v[1] = x;
  nu.v[2] = y;
  nu.v[3] = S.n1.z[0] + S.n1.z[1] * x + S.n1.z[2] * y;
  nu.v[0] = df_sqrt(x * x + y * y + nu.v[3] * nu.v[3]);
  nub.v[1] = S.mx - x;
  nub.v[2] = S.my - y;
  nub.v[3] = S.n2.z[0] + S.n2.z[1] * nub.v[1] + S.n2.z[2] * nub.v[2];
  nub.v[0] = df_sqrt(nub.v[1] * nub.v[1] + nub.v[2] * nub.v[2] + nub.v[3] * nub.v[3]);
}

// |det d(q^2_W+, q^2_t, q^2_W-, q^2_tbar) / d(nu_x, nu_y, nu_z, nubar_z)| for on-shell
// nu, nubar, in units of DL_UNIT^4 (the Jacobian of Eq. "dilepsolv" is its inverse).
static __device__ __noinline__ df dl_det(const DLMom& b, const DLMom& bb, const DLMom& lp,
                                     const DLMom& lm, const DLMom& nu, const DLMom& nub) {
  // d (P + nu)^2 / d nu_k = 2 (P_0 nu_k / E - P_k) for massless nu; the common factor
  // 2 of every entry gives 2^4 in the determinant
  df M[4][4];
  const df ie = 1.f / nu.v[0], ieb = 1.f / nub.v[0];
  const df blp0 = b.v[0] + lp.v[0], bblm0 = bb.v[0] + lm.v[0];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const df nk = nu.v[1 + k] * ie;
    M[0][k] = lp.v[0] * nk - lp.v[1 + k];
    M[1][k] = blp0 * nk - (b.v[1 + k] + lp.v[1 + k]);
  }
  M[0][3] = M[1][3] = df(0.f);
#pragma unroll
  for (int k = 0; k < 2; ++k) {   // nubar_T = MET - nu_T
    const df nk = nub.v[1 + k] * ieb;
    M[2][k] = -(lm.v[0] * nk - lm.v[1 + k]);
    M[3][k] = -(bblm0 * nk - (bb.v[1 + k] + lm.v[1 + k]));
  }
  M[2][2] = M[3][2] = df(0.f);
  const df nz = nub.v[3] * ieb;
  M[2][3] = lm.v[0] * nz - lm.v[3];
  M[3][3] = bblm0 * nz - (bb.v[3] + lm.v[3]);
  // Laplace expansion along the last two columns: column 2 (nu_z) is nonzero only in
  // rows 0, 1 and column 3 (nubar_z) only in rows 2, 3, so
  // det = sum_{r in {0,1}, s in {2,3}} (-1)^(r+s+1) M[r][2] M[s][3] (M[r'][0] M[s'][1] - M[r'][1] M[s'][0])
  // with r' = 1 - r and s' = 5 - s.
  df det(0.f);
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int t = 2; t < 4; ++t) {
      const int rc = 1 - r, tc = 5 - t;
      const df minor = M[rc][0] * M[tc][1] - M[rc][1] * M[tc][0];
      const df term = M[r][2] * M[t][3] * minor;
      det = ((r + t + 1) & 1) ? det - term : det + term;
    }
  return df_ldexp(df_abs(det), 16.f);
}

// FP32 light-cone form (GeV) of a massless momentum in DL_UNIT: the larger of
// E +- p_z directly, the smaller from pT^2 over it (no cancellation).
__device__ __forceinline__ LCv dl_lc(const DLMom& p) {
  const float E = p.v[0].hi * DL_UNIT, px = p.v[1].hi * DL_UNIT, py = p.v[2].hi * DL_UNIT;
  const float pz = p.v[3].hi * DL_UNIT;
  const float t2 = fmaf(px, px, py * py);
  const float big = E + fabsf(pz), small = t2 / big;
  LCv o;
  o.pp = pz >= 0.f ? big : small;
  o.pm = pz >= 0.f ? small : big;
  o.pt = C(px, py);
  return o;
}

// The decay factor of a solution, (p_b.p_nu)(p_bbar.p_nubar) / (E_nu E_nubar |det|)
// in GeV^-2 (det in GeV^4): the b-neutrino invariants of the top decays over the
// neutrinos' 1/(2E) phase-space energies (the 1/4 is in the caller's constants) and
// the Jacobian of Eq. "dilepsolv".
__device__ __forceinline__ float dl_decay_factor(const DLMom& b, const DLMom& bb, const DLMom& nu,
                                                 const DLMom& nub, df det) {
  if (!(det.hi > 0.f)) return 0.f;
  const float pbn = dl_dot(b, nu).hi, pbbn = dl_dot(bb, nub).hi;   // DL_UNIT^2
  // (pbn U^2)(pbbn U^2) / ((E U)(Eb U) det U^4) = pbn pbbn / (E Eb det U^2)
  return (pbn / nu.v[0].hi) * (pbbn / nub.v[0].hi) / (det.hi * (DL_UNIT * DL_UNIT));
}

// de-duplication of solutions: two roots that give the same (x, y) to 1e-9 relative
__device__ __forceinline__ bool dl_same(df x1, df y1, df x2, df y2) {
  return fabsf((x1 - x2).hi) + fabsf((y1 - y2).hi) < 1e-9f * (1.f + fabsf(x2.hi) + fabsf(y2.hi));
}

}  // namespace mem

// Dilepton ttbar integrand (Sec. 3-4: the final state of the hadron-level
// analysis without the Higgs), g g / q qbar -> t tbar -> (b l+ nu)(bbar mu- nubar).
//
// Variables (6): E_b and E_bbar (log-uniform over their jet windows), q^2 of the
// W+ and of the W- (Breit-Wigner maps over [0, s]), q^2 of the top over
// [q^2_W+ + 2 p_b.p_l+, s] and of the antitop over [q^2_W- + 2 p_bbar.p_mu-, s]
// (Breit-Wigner maps; the lower ends are where p_b.p_nu = 0). Leptons are measured
// exactly; the missing transverse momentum at each point is the visible imbalance
// -(l+ + mu- + b + bbar)_T, so the final state carries no total pT and no
// transverse boost is needed. The two neutrinos follow from the four virtualities
// and that imbalance (Eq. "dilepsolv"): up to four solutions, each weighted by
// 1 / |det d(q^2_W+, q^2_t, q^2_W-, q^2_tbar) / d(nu_x, nu_y, nu_z, nubar_z)|.
//
// Precision: the neutrino solution's algebra runs in FP64. Eliminating the neutrino
// energies and p_z leaves two conics in (nu_x, nu_y) whose resultant is a quartic;
// its coefficients are products of four conic coefficients and cancel by several
// orders of magnitude, beyond FP32's seven digits. The iterative root search runs
// in FP32 wherever its result is only a bracket or a starting point (FP64 is ~1/64
// of the FP32 rate on this part). Everything else (maps, transfer functions,
// amplitudes, PDFs) is FP32 as in the other processes.
//
// Real roots of the quartic: every real root of a polynomial lies between two
// consecutive real roots of its derivative (Rolle), so the roots of the linear,
// quadratic and cubic derivatives (in FP32: they only separate roots) bracket
// those of the quartic, whose signs at the bracket ends are taken in FP64; each
// root is then located in FP32 and finished by FP64 Newton steps. Roots are then
// polished on the two conics (Newton in 2D, FP64).
//
// The solver's stages (dl_system(_met), dl_real_roots, dl_bracket_root, dl_point) are
// kept out of line. Inlined into the integrand, this build (nvcc 13.0, sm_103a)
// returned incomplete solution sets on about a third of the points of a test
// batch -- the same functions called from a small kernel, or out of line, agree
// with a host build of this file and with the FP64 reference to 1e-12 in the
// roots. Out of line they also keep the integrand's register count down.
//
// |M|^2: the semileptonic amplitude of mem_ttbar.cuh with mu- in the role of the
// d quark and nubar in that of the ubar (the Fierz-collapsed antitop chain has
// the same form for W- -> mu- nubar), divided by the 6 channels (3 colours x 2
// generations) that the hadronic W- decay carries in its couplings.
#pragma once
#include "mem_ttbar.cuh"

namespace mem {

struct DLCache {
  float b_lo, Lb, bb_lo, Lbb;                    // jet windows: lo and ln(hi / lo)
  float bnx, bny, bnz, blcp, blcm;               // b jet direction, light-cone fractions
  float bbnx, bbny, bbnz, bblcp, bblcm;          // bbar jet
  float Ebm, Ebbm;                               // measured jet energies
  float Elp, lpnx, lpny, lpnz, lplcp, lplcm;     // l+
  float Elm, lmnx, lmny, lmnz, lmlcp, lmlcm;     // mu-
  float omc_bl, omc_bbl;                         // 1 - n_b.n_l+, 1 - n_bbar.n_mu-
  float psi_w, psi_t;                            // atan2(m G, s - m^2) of the W and top maps
  float core_w, tail_w, inv_core, inv_tail;      // double Gaussian (as in TTCache)
  float cst;
  int ok;
};

// ------------------------------------------------------------- FP64 solver
// A conic q(x, y) = xx x^2 + xy x y + yy y^2 + x1 x + y1 y + c0.
struct DLConic { double xx, xy, yy, x1, y1, c0; };

__device__ __forceinline__ double dl_conic_at(const DLConic& q, double x, double y) {
  return fma(x, fma(q.xx, x, fma(q.xy, y, q.x1)), fma(y, fma(q.yy, y, q.y1), q.c0));
}

// Massless neutrino with lepton l and b quark (scaled units): l.nu = A and b.nu = B
// fix E and p_z as affine functions of (p_x, p_y) -- E = e[0] + e[1] x + e[2] y,
// p_z = z[0] + z[1] x + z[2] y. Returns false when the two equations are degenerate
// in (E, p_z) (the lepton and the b share their p_z / E ratio).
struct DLAffine { double e[3], z[3]; };

__device__ __forceinline__ bool dl_affine(const double* l, const double* b, double A, double B,
                                          DLAffine& r) {
  // l0 E - lz pz = A + lx x + ly y ;  b0 E - bz pz = B + bx x + by y
  const double det = l[3] * b[0] - l[0] * b[3];
  if (!(fabs(det) > 1e-12 * (fabs(l[0] * b[3]) + fabs(l[3] * b[0]) + 1e-300))) return false;
  const double id = 1.0 / det;
  const double ra[3] = {A, l[1], l[2]}, rb[3] = {B, b[1], b[2]};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r.e[k] = (l[3] * rb[k] - b[3] * ra[k]) * id;
    r.z[k] = (l[0] * rb[k] - b[0] * ra[k]) * id;
  }
  return true;
}

// E^2 - x^2 - y^2 - p_z^2 of the affine neutrino, as a conic in (x, y).
__device__ __forceinline__ DLConic dl_shell(const DLAffine& a) {
  DLConic q;
  q.xx = a.e[1] * a.e[1] - a.z[1] * a.z[1] - 1.0;
  q.yy = a.e[2] * a.e[2] - a.z[2] * a.z[2] - 1.0;
  q.xy = 2.0 * (a.e[1] * a.e[2] - a.z[1] * a.z[2]);
  q.x1 = 2.0 * (a.e[0] * a.e[1] - a.z[0] * a.z[1]);
  q.y1 = 2.0 * (a.e[0] * a.e[2] - a.z[0] * a.z[2]);
  q.c0 = a.e[0] * a.e[0] - a.z[0] * a.z[0];
  return q;
}

// The antineutrino's conic in its own (X, Y), rewritten in the neutrino's (x, y)
// through X = mx - x, Y = my - y.
__device__ __forceinline__ DLConic dl_mirror(const DLConic& q, double mx, double my) {
  DLConic r;
  r.xx = q.xx;
  r.xy = q.xy;
  r.yy = q.yy;
  r.x1 = -(2.0 * q.xx * mx + q.xy * my + q.x1);
  r.y1 = -(2.0 * q.yy * my + q.xy * mx + q.y1);
  r.c0 = dl_conic_at(q, mx, my);
  return r;
}

template <class T>
__device__ __forceinline__ T dl_horner(const T* c, int deg, T x, T& dp) {
  T p = c[deg], d = T(0);
  for (int k = deg - 1; k >= 0; --k) {
    d = fma(d, x, p);
    p = fma(p, x, c[k]);
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

// FP64 root of c in [a, b] (a sign change, fa = c(a)) from the start x0, to
// |step| <= tol (1 + |x|): Newton steps that divide by an FP32 reciprocal of the
// derivative (FP64 division costs several FP64 instructions on this part; near
// the root the iteration then contracts by ~1e-7 per step, which from an
// FP32-accurate start is the same two steps), bisection whenever a step leaves
// the shrinking bracket.
static __device__ __noinline__ double dl_bracket_root(const double* c, int deg, double a, double b,
                                               double fa, double x0, double tol) {
  double x = (x0 > a && x0 < b) ? x0 : 0.5 * (a + b);
#pragma unroll 1
  for (int it = 0; it < 96; ++it) {
    double dp;
    const double f = dl_horner(c, deg, x, dp);
    if (f == 0.0) return x;
    if ((f < 0.0) == (fa < 0.0)) {
      a = x;
      fa = f;
    } else {
      b = x;
    }
    const float dpf = fabsf((float)dp);
    double xn = 0.5 * (a + b);   // bisection unless the Newton step stays in the bracket
    if (dpf > 1e-30f && dpf < 1e30f) {
      const double t = x - f * (double)(1.f / (float)dp);
      if (t > a && t < b) xn = t;
    }
    if (fabs(xn - x) <= tol * (1.0 + fabs(x))) return xn;
    x = xn;
  }
  return x;
}

// Real roots (ascending) of c[0] + c[1] x + ... + c[deg] x^deg, 1 <= deg <= 4,
// c[deg] != 0. The critical points -- the real roots of the derivative chain
// (linear, quadratic in closed form, cubic by bracketed Newton) -- are found in
// FP32 on the monic polynomial: they only separate the roots. Which intervals
// between them hold a root is decided by the signs of the FP64 polynomial at
// their ends (at a critical point the polynomial is flat, so an FP32-accurate
// location gives the exact sign); each root is located in FP32 and finished by
// FP64 Newton steps inside its bracket. A critical point where the polynomial
// vanishes to rounding is a double root and is kept once.
static __device__ __noinline__ int dl_real_roots(const double* c, int deg, double* roots) {
  const double ilead = 1.0 / c[deg];
  float cf[5];
  float bound = 0.f;
  for (int k = 0; k < deg; ++k) {
    cf[k] = (float)(c[k] * ilead);
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
  // level 0: FP64 signs at the bracket ends, FP32 location, FP64 finish
  int n = 0;
  const double B = (double)bound;
  double a = -B, dpa;
  double fa = dl_horner(c, deg, a, dpa);
  // derivative coefficients (FP64) for refining critical points near a double root
  double c1[4];
  for (int k = 0; k < deg; ++k) c1[k] = (k + 1) * c[k + 1];
  for (int i = 0; i <= ncrit; ++i) {
    double b = i < ncrit ? fmin(fmax((double)crit[i], -B), B) : B;
    double dpb;
    double fb = dl_horner(c, deg, b, dpb);
    if (i < ncrit && deg >= 2) {
      // Where the polynomial is small at a critical point, two roots may lie closer
      // together than the FP32 critical point's error, which would put both on one
      // side of it and lose them: move it to FP64 accuracy (Newton on p') first.
      double mag = 0.0, pw = 1.0;
      for (int k = 0; k <= deg; ++k, pw *= fabs(b)) mag += fabs(c[k]) * pw;
      if (fabs(fb) <= 1e-6 * mag) {
        const double hi = i + 1 < ncrit ? fmin(fmax((double)crit[i + 1], -B), B) : B;
#pragma unroll 1
        for (int it = 0; it < 4; ++it) {
          double d2p;   // p''(b), from the Horner pass over p'
          const double p1 = dl_horner(c1, deg - 1, b, d2p);
          if (!(d2p != 0.0)) break;
          const double bn = b - p1 / d2p;
          if (!(bn > a && bn < hi)) break;
          const bool done = fabs(bn - b) <= 1e-15 * (1.0 + fabs(b));
          b = bn;
          if (done) break;
        }
        fb = dl_horner(c, deg, b, dpb);
      }
    }
    if (b > a && ((fa < 0.0 && fb > 0.0) || (fa > 0.0 && fb < 0.0))) {
      // the monic FP32 copy has the sign of c times that of the leading coefficient
      const float sa = ((fa < 0.0) != (ilead < 0.0)) ? -1.f : 1.f;
      const float x0 = dl_bracket32(cf, deg, (float)a, (float)b, sa);
      roots[n++] = dl_bracket_root(c, deg, a, b, fa, (double)x0, 1e-15);
    } else if (i < ncrit && (n == 0 || roots[n - 1] < b)) {
      // touches zero at the critical point: |p| at the rounding level of its terms
      double mag = 0.0, pw = 1.0;
      for (int k = 0; k <= deg; ++k, pw *= fabs(b)) mag += fabs(c[k]) * pw;
      if (fabs(fb) <= 1e-13 * mag) roots[n++] = b;
    }
    a = b;
    fa = fb;
    if (n >= deg) break;
  }
  return n;
}

// Newton steps in (x, y) on the intersection of two conics, to a step of 1e-12
// relative (far below the FP32 that the solution feeds; the conic coefficients
// themselves carry more rounding than that, so a tighter target only makes the
// iteration dither until its cap).
__device__ __forceinline__ void dl_polish(const DLConic& p, const DLConic& q, double& x, double& y) {
#pragma unroll 1
  for (int it = 0; it < 4; ++it) {
    const double f = dl_conic_at(p, x, y), g = dl_conic_at(q, x, y);
    const double fx = fma(2.0 * p.xx, x, fma(p.xy, y, p.x1)), fy = fma(p.xy, x, fma(2.0 * p.yy, y, p.y1));
    const double gx = fma(2.0 * q.xx, x, fma(q.xy, y, q.x1)), gy = fma(q.xy, x, fma(2.0 * q.yy, y, q.y1));
    const double det = fx * gy - fy * gx;
    if (det == 0.0) return;
    const double id = 1.0 / det;
    const double dx = (f * gy - g * fy) * id, dy = (g * fx - f * gx) * id;
    x -= dx;
    y -= dy;
    if (fabs(dx) + fabs(dy) < 1e-12 * (1.0 + fabs(x) + fabs(y))) return;
  }
}

// The conics and the resultant quartic of one phase-space point. Momenta in
// units of DL_UNIT GeV, virtualities in DL_UNIT^2.
constexpr double DL_UNIT = 100.0;

struct DLSystem {
  DLAffine n1, n2;       // neutrino (in its x, y) and antineutrino (in its X, Y)
  DLConic c1, c2;        // mass shells in the neutrino's (x, y)
  double u[3], v[2];     // y = -u(x) / v(x) on the common points
  double mx, my;
};

// Builds the system; returns the number of real roots x of the resultant (in xr).
// The missing pT (mx, my) is given: the negative visible pT sum of the event's own
// final state (the dilepton ttbar form below adds the four objects; dilepton ttH
// adds the Higgs pair too).
static __device__ __noinline__ int dl_system_met(const double* b, const double* bb, const double* lp,
                                          const double* lm, double mx, double my, double q2wp,
                                          double q2wm, double q2t, double q2tb, DLSystem& S,
                                          double* xr) {
  S.mx = mx;
  S.my = my;
  // 2 l.nu = q^2_W and 2 b.nu = q^2_t - q^2_W - 2 b.l (massless b, l, nu)
  const double blp = b[0] * lp[0] - b[1] * lp[1] - b[2] * lp[2] - b[3] * lp[3];
  const double bblm = bb[0] * lm[0] - bb[1] * lm[1] - bb[2] * lm[2] - bb[3] * lm[3];
  if (!dl_affine(lp, b, 0.5 * q2wp, 0.5 * (q2t - q2wp) - blp, S.n1)) return 0;
  if (!dl_affine(lm, bb, 0.5 * q2wm, 0.5 * (q2tb - q2wm) - bblm, S.n2)) return 0;
  S.c1 = dl_shell(S.n1);
  S.c2 = dl_mirror(dl_shell(S.n2), S.mx, S.my);
  // each conic as a_i y^2 + (p_i + r_i x) y + (s_i + t_i x + w_i x^2)
  const DLConic& P = S.c1;
  const DLConic& Q = S.c2;
  const double a1 = P.yy, a2 = Q.yy;
  // u = a1 C2 - a2 C1 (quadratic), v = a1 B2 - a2 B1 (linear), w = B1 C2 - B2 C1 (cubic)
  S.u[0] = a1 * Q.c0 - a2 * P.c0;
  S.u[1] = a1 * Q.x1 - a2 * P.x1;
  S.u[2] = a1 * Q.xx - a2 * P.xx;
  S.v[0] = a1 * Q.y1 - a2 * P.y1;
  S.v[1] = a1 * Q.xy - a2 * P.xy;
  double w[4];
  w[0] = P.y1 * Q.c0 - Q.y1 * P.c0;
  w[1] = P.y1 * Q.x1 + P.xy * Q.c0 - Q.y1 * P.x1 - Q.xy * P.c0;
  w[2] = P.y1 * Q.xx + P.xy * Q.x1 - Q.y1 * P.xx - Q.xy * P.x1;
  w[3] = P.xy * Q.xx - Q.xy * P.xx;
  // resultant in y: u^2 - v w
  double R[5];
  R[0] = S.u[0] * S.u[0] - S.v[0] * w[0];
  R[1] = 2.0 * S.u[0] * S.u[1] - S.v[0] * w[1] - S.v[1] * w[0];
  R[2] = S.u[1] * S.u[1] + 2.0 * S.u[0] * S.u[2] - S.v[0] * w[2] - S.v[1] * w[1];
  R[3] = 2.0 * S.u[1] * S.u[2] - S.v[0] * w[3] - S.v[1] * w[2];
  R[4] = S.u[2] * S.u[2] - S.v[1] * w[3];
  double scale = 0.0;
  for (int k = 0; k < 5; ++k) scale = fmax(scale, fabs(R[k]));
  if (scale == 0.0) return 0;
  int deg = 4;
  while (deg > 0 && fabs(R[deg]) <= 1e-13 * scale) --deg;
  if (deg == 0) return 0;
  return dl_real_roots(R, deg, xr);
}

static __device__ __noinline__ int dl_system(const double* b, const double* bb, const double* lp,
                                      const double* lm, double q2wp, double q2wm, double q2t,
                                      double q2tb, DLSystem& S, double* xr) {
  return dl_system_met(b, bb, lp, lm, -(lp[1] + lm[1] + b[1] + bb[1]),
                       -(lp[2] + lm[2] + b[2] + bb[2]), q2wp, q2wm, q2t, q2tb, S, xr);
}

// One neutrino solution from a root x of the resultant: y, conic polish, the
// residual and positive-energy checks. Returns false when the root is rejected.
static __device__ __noinline__ bool dl_point(const DLSystem& S, double xr, double& x, double& y) {
  const double num = -fma(fma(S.u[2], xr, S.u[1]), xr, S.u[0]);
  const double den = fma(S.v[1], xr, S.v[0]);
  if (fabs(den) > 1e-12 * (fabs(num) + 1.0)) {
    y = num / den;
  } else {
    // v vanishes: y from the first conic's quadratic, the branch on the second
    const double a = S.c1.yy, bq = fma(S.c1.xy, xr, S.c1.y1);
    const double cq = fma(fma(S.c1.xx, xr, S.c1.x1), xr, S.c1.c0);
    const double disc = bq * bq - 4.0 * a * cq;
    if (disc < 0.0 || a == 0.0) return false;
    const double y1 = (-bq + sqrt(disc)) / (2.0 * a), y2 = (-bq - sqrt(disc)) / (2.0 * a);
    y = fabs(dl_conic_at(S.c2, xr, y1)) < fabs(dl_conic_at(S.c2, xr, y2)) ? y1 : y2;
  }
  x = xr;
  dl_polish(S.c1, S.c2, x, y);
  const double tol = 1e-8 * (1.0 + x * x + y * y);
  if (fabs(dl_conic_at(S.c1, x, y)) > tol || fabs(dl_conic_at(S.c2, x, y)) > tol) return false;
  const double E = S.n1.e[0] + S.n1.e[1] * x + S.n1.e[2] * y;
  const double X = S.mx - x, Y = S.my - y;
  const double Eb = S.n2.e[0] + S.n2.e[1] * X + S.n2.e[2] * Y;
  return E > 0.0 && Eb > 0.0;
}

// 1 / |det d(q^2_W+, q^2_t, q^2_W-, q^2_tbar) / d(nu_x, nu_y, nu_z, nubar_z)| in
// GeV^-4 for on-shell nu, nub (scaled units in, GeV units out).
__device__ __forceinline__ double dl_jacobian(const double* b, const double* bb, const double* lp,
                                              const double* lm, const double* nu,
                                              const double* nub) {
  // d (P + nu)^2 / d nu_k = 2 (P_0 nu_k / E - P_k) for massless nu
  double M[4][4];
  const double ie = 1.0 / nu[0], ieb = 1.0 / nub[0];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    M[0][k] = 2.0 * (lp[0] * nu[1 + k] * ie - lp[1 + k]);
    M[1][k] = 2.0 * ((b[0] + lp[0]) * nu[1 + k] * ie - (b[1 + k] + lp[1 + k]));
  }
  M[0][3] = M[1][3] = 0.0;
#pragma unroll
  for (int k = 0; k < 2; ++k) {   // nubar_T = MET - nu_T
    M[2][k] = -2.0 * (lm[0] * nub[1 + k] * ieb - lm[1 + k]);
    M[3][k] = -2.0 * ((bb[0] + lm[0]) * nub[1 + k] * ieb - (bb[1 + k] + lm[1 + k]));
  }
  M[2][2] = M[3][2] = 0.0;
  M[2][3] = 2.0 * (lm[0] * nub[3] * ieb - lm[3]);
  M[3][3] = 2.0 * ((bb[0] + lm[0]) * nub[3] * ieb - (bb[3] + lm[3]));
  // Laplace expansion along the last two columns: column 2 (nu_z) is nonzero only in
  // rows 0, 1 and column 3 (nubar_z) only in rows 2, 3, so
  // det = sum_{r in {0,1}, s in {2,3}} (-1)^(r+s+1) M[r][2] M[s][3] (M[r'][0] M[s'][1] - M[r'][1] M[s'][0])
  // with r' = 1 - r and s' = 5 - s.
  double det = 0.0;
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int t = 2; t < 4; ++t) {
      const int rc = 1 - r, tc = 5 - t;
      const double minor = M[rc][0] * M[tc][1] - M[rc][1] * M[tc][0];
      const double term = M[r][2] * M[t][3] * minor;
      det += ((r + t + 1) & 1) ? -term : term;
    }
  const double u4 = DL_UNIT * DL_UNIT * DL_UNIT * DL_UNIT;   // each entry is in GeV / DL_UNIT
  return det == 0.0 ? 0.0 : 1.0 / (fabs(det) * u4);
}

// Light-cone form of an FP64 massless momentum (larger component direct, the
// smaller from pT^2 over it).
__device__ __forceinline__ LCv dl_lc(const double* p) {
  double pp = p[0] + p[3], pm = p[0] - p[3];
  const double t2 = p[1] * p[1] + p[2] * p[2];
  if (pp >= pm) pm = t2 / pp;
  else pp = t2 / pm;
  LCv o;
  o.pp = (float)pp;
  o.pm = (float)pm;
  o.pt = C((float)p[1], (float)p[2]);
  return o;
}

template <int PDFM>
struct PhysTTDL_ {
  static constexpr int D = 6;
  static constexpr int NPERM = 2;
  using Cache = DLCache;

  __device__ static void setup(const float* rec, int perm, const ProcConst& P, const TFConst& T,
                               Cache& c) {
    // perm 0: object 2 is the b jet and object 3 the bbar; perm 1 the reverse
    const int ob = 2 + (perm == 1), obb = 3 - (perm == 1);
    c.ok = perm >= 0 && perm < 2 && rec[3] == 4.f && rec[7] == 1.f && rec[11] == 5.f &&
           rec[15] == 5.f && rec[0] > 0.f && rec[4] > 0.f && rec[8] > 0.f && rec[12] > 0.f &&
           T.jet_core > 0.f && T.jet_tail > 0.f;
    double n[4][3], sn[4], lc[4][2];
    const int objs[4] = {ob, obb, 0, 1};
    for (int k = 0; k < 4; ++k) {
      const int o = objs[k];
      const double eta = rec[4 * o + 1], phi = rec[4 * o + 2], ch = cosh(eta);
      n[k][0] = cos(phi) / ch;
      n[k][1] = sin(phi) / ch;
      n[k][2] = tanh(eta);
      sn[k] = 1.0 / ch;
      lc[k][0] = exp(eta) / ch;
      lc[k][1] = exp(-eta) / ch;
    }
    const double smax = 0.5 * (double)P.sqrt_s;
    double L[2];
    float lo[2];
    for (int k = 0; k < 2; ++k) {
      const double E = rec[4 * objs[k]];
      const double l = E / (double)T.jet_lo_div;
      double h = E * (double)T.jet_hi_mul;
      h = h < smax ? h : smax;
      c.ok = c.ok && h > l;
      lo[k] = (float)l;
      L[k] = c.ok ? log(h / l) : 0.0;
    }
    c.b_lo = lo[0];
    c.Lb = (float)L[0];
    c.bb_lo = lo[1];
    c.Lbb = (float)L[1];
    c.bnx = (float)n[0][0];
    c.bny = (float)n[0][1];
    c.bnz = (float)n[0][2];
    c.blcp = (float)lc[0][0];
    c.blcm = (float)lc[0][1];
    c.bbnx = (float)n[1][0];
    c.bbny = (float)n[1][1];
    c.bbnz = (float)n[1][2];
    c.bblcp = (float)lc[1][0];
    c.bblcm = (float)lc[1][1];
    c.Ebm = rec[4 * ob];
    c.Ebbm = rec[4 * obb];
    c.Elp = rec[0];
    c.lpnx = (float)n[2][0];
    c.lpny = (float)n[2][1];
    c.lpnz = (float)n[2][2];
    c.lplcp = (float)lc[2][0];
    c.lplcm = (float)lc[2][1];
    c.Elm = rec[4];
    c.lmnx = (float)n[3][0];
    c.lmny = (float)n[3][1];
    c.lmnz = (float)n[3][2];
    c.lmlcp = (float)lc[3][0];
    c.lmlcm = (float)lc[3][1];
    auto omc = [](const double* a, const double* b) {   // 1 - a.b = |a - b|^2 / 2
      const double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
      return 0.5 * (dx * dx + dy * dy + dz * dz);
    };
    c.omc_bl = (float)omc(n[0], n[2]);
    c.omc_bbl = (float)omc(n[1], n[3]);
    c.psi_w = (float)atan2((double)P.mwgw, (double)P.s - (double)P.mw2);
    c.psi_t = (float)atan2((double)P.mtgt, (double)P.s - (double)P.mt2);
    const double tw = T.jet_tail_w;
    c.core_w = (float)((1.0 - tw) / T.jet_core);
    c.tail_w = (float)(tw / T.jet_tail);
    c.inv_core = (float)(1.0 / T.jet_core);
    c.inv_tail = (float)(1.0 / T.jet_tail);
    // per jet: E^2 sin(theta) (measure) x 1/E (phase space, the 1/2 and (2 pi)^-3 are
    // in the prefactor) x 1/(E sqrt(2 pi)) (TF normalisation) x E L (log map) =
    // E sin(theta) L / sqrt(2 pi) -- E and the TF exponentials are per point.
    // Leptons: 1/E each. Resonances: R / (m G) per Breit-Wigner map. W- -> mu- nubar:
    // 1/6 of the hadronic couplings in tt_gg, tt_qq.
    const double mgw = (double)P.mwgw, mgt = (double)P.mtgt;
    c.cst = (float)(sn[0] * sn[1] * L[0] * L[1] / (2.0 * PI_D) / ((double)rec[0] * (double)rec[4]) /
                    (mgw * mgw * mgt * mgt) / 6.0 * TT_WEIGHT_SCALE);
  }

  __device__ static float eval(const Cache& c, const ProcConst& P, const float (&x)[D],
                               const float (&xc)[D]) {
    const float Eb = c.b_lo * __expf(x[0] * c.Lb);
    const float Ebb = c.bb_lo * __expf(x[1] * c.Lbb);
    const BW wp = bw_map(0.f, P.s, P.mw2, P.mwgw, x[2], xc[2], c.psi_w);
    const BW wm = bw_map(0.f, P.s, P.mw2, P.mwgw, x[3], xc[3], c.psi_w);
    const float lo_t = fmaf(2.f * Eb * c.Elp, c.omc_bl, wp.q2);
    const float lo_tb = fmaf(2.f * Ebb * c.Elm, c.omc_bbl, wm.q2);
    if (!(lo_t < P.s && lo_tb < P.s)) return 0.f;
    const BW tq = bw_map(lo_t, P.s - lo_t, P.mt2, P.mtgt, x[4], xc[4], c.psi_t);
    const BW tbq = bw_map(lo_tb, P.s - lo_tb, P.mt2, P.mtgt, x[5], xc[5], c.psi_t);
    // FP64 momenta in units of DL_UNIT
    const double iu = 1.0 / DL_UNIT, iu2 = iu * iu;
    const double eb = (double)Eb * iu, ebb = (double)Ebb * iu;
    const double elp = (double)c.Elp * iu, elm = (double)c.Elm * iu;
    const double b[4] = {eb, eb * c.bnx, eb * c.bny, eb * c.bnz};
    const double bb[4] = {ebb, ebb * c.bbnx, ebb * c.bbny, ebb * c.bbnz};
    const double lp[4] = {elp, elp * c.lpnx, elp * c.lpny, elp * c.lpnz};
    const double lm[4] = {elm, elm * c.lmnx, elm * c.lmny, elm * c.lmnz};
    DLSystem S;
    double xr[4];
    const int nr = dl_system(b, bb, lp, lm, (double)wp.q2 * iu2, (double)wm.q2 * iu2,
                             (double)tq.q2 * iu2, (double)tbq.q2 * iu2, S, xr);
    if (nr == 0) return 0.f;
    const float m = sqrtf(P.mt2);
    // FP32 light-cone momenta of the measured partons
    LCv Lb, Lbb, Llp, Llm;
    Lb.pp = Eb * c.blcp; Lb.pm = Eb * c.blcm; Lb.pt = C(Eb * c.bnx, Eb * c.bny);
    Lbb.pp = Ebb * c.bblcp; Lbb.pm = Ebb * c.bblcm; Lbb.pt = C(Ebb * c.bbnx, Ebb * c.bbny);
    Llp.pp = c.Elp * c.lplcp; Llp.pm = c.Elp * c.lplcm; Llp.pt = C(c.Elp * c.lpnx, c.Elp * c.lpny);
    Llm.pp = c.Elm * c.lmlcp; Llm.pm = c.Elm * c.lmlcm; Llm.pt = C(c.Elm * c.lmnx, c.Elm * c.lmny);
    double seen[4][2];
    int ns = 0;
    float acc = 0.f;
#pragma unroll 1
    for (int r = 0; r < nr; ++r) {
      double px, py;
      if (!dl_point(S, xr[r], px, py)) continue;
      bool dup = false;
      for (int k = 0; k < ns; ++k)
        dup = dup || fabs(seen[k][0] - px) + fabs(seen[k][1] - py) < 1e-9 * (1.0 + fabs(px) + fabs(py));
      if (dup) continue;
      seen[ns][0] = px;
      seen[ns][1] = py;
      ++ns;
      double nu[4], nub[4];
      nu[1] = px;
      nu[2] = py;
      nu[3] = S.n1.z[0] + S.n1.z[1] * px + S.n1.z[2] * py;
      nu[0] = sqrt(px * px + py * py + nu[3] * nu[3]);
      nub[1] = S.mx - px;
      nub[2] = S.my - py;
      nub[3] = S.n2.z[0] + S.n2.z[1] * nub[1] + S.n2.z[2] * nub[2];
      nub[0] = sqrt(nub[1] * nub[1] + nub[2] * nub[2] + nub[3] * nub[3]);
      const double jnu = dl_jacobian(b, bb, lp, lm, nu, nub);
      // decay invariants p_b.p_nu and p_bbar.p_nubar (GeV^2)
      const double pbn = (b[0] * nu[0] - b[1] * nu[1] - b[2] * nu[2] - b[3] * nu[3]) * DL_UNIT * DL_UNIT;
      const double pbbn = (bb[0] * nub[0] - bb[1] * nub[1] - bb[2] * nub[2] - bb[3] * nub[3]) * DL_UNIT * DL_UNIT;
      double nug[4], nubg[4];
      for (int k = 0; k < 4; ++k) {
        nug[k] = nu[k] * DL_UNIT;
        nubg[k] = nub[k] * DL_UNIT;
      }
      const LCv Ln = dl_lc(nug), Lnb = dl_lc(nubg);
      LCv tp, tm;
      tp.pp = Lb.pp + Llp.pp + Ln.pp;
      tp.pm = Lb.pm + Llp.pm + Ln.pm;
      tp.pt = Lb.pt + Llp.pt + Ln.pt;
      tm.pp = Lbb.pp + Llm.pp + Lnb.pp;
      tm.pm = Lbb.pm + Llm.pm + Lnb.pm;
      tm.pt = Lbb.pt + Llm.pt + Lnb.pt;
      const float k1p = tp.pp + tm.pp;   // x1 sqrt(s): no total pT, no boost
      const float k2m = tp.pm + tm.pm;   // x2 sqrt(s)
      const float x1 = k1p / P.sqrt_s, x2 = k2m / P.sqrt_s;
      if (!(x1 < 1.f && x2 < 1.f)) continue;
      const float shat = k1p * k2m;
      const TTAmp2 amp = tt_amp2(Llp, Llm, tp, tm, m, P.mt2, k1p, k2m, shat);
      PdfX f1, f2;
      pdf_pair<PDFM>(P, x1, x2, f1, f2);
      const float init = fmaf(P.tt_gg * f1.g * f2.g, amp.gg,
                              P.tt_qq * 2.f * fmaf(f1.q, f2.qb, f1.qb * f2.q) * amp.qq);
      const float dec = (float)(pbn * pbbn * jnu / (nug[0] * nubg[0]));
      acc += init * (4.f / shat) * dec;
    }
    if (acc == 0.f) return 0.f;
    const float gb = dgauss_g(c, c.Ebm, Eb), gbb = dgauss_g(c, c.Ebbm, Ebb);
    return c.cst * Eb * Ebb * gb * gbb * (wp.R * wm.R) * (tq.R * tbq.R) * acc;
  }
};
using PhysTTDL = PhysTTDL_<PDF_ANY>;

}  // namespace mem

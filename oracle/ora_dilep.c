/* Dilepton ttbar kinematics of the oracle (test infrastructure; see oracle.h):
 * the coupled two-neutrino solution of Sec. 3, Eq. "dilepsolv".
 *
 * Given the b, bbar, l+, l- momenta (massless), the missing transverse momentum
 * and the four virtualities q2_W+ = (l+ + nu)^2, q2_t = (b + l+ + nu)^2,
 * q2_W- = (l- + nubar)^2, q2_tbar = (bbar + l- + nubar)^2, the two massless
 * neutrinos with nu_T + nubar_T = MET are found as follows (derived here from the
 * constraint equations):
 *  - for each neutrino the two virtualities are linear in its 4-momentum
 *    (2 l.nu = q2_W, 2 b.nu = q2_t - q2_W - (b + l)^2), which fixes its energy and
 *    p_z as linear functions of its (p_x, p_y);
 *  - its mass shell E^2 = |p|^2 then is a conic in (p_x, p_y); the antineutrino's
 *    conic, written in the neutrino's (p_x, p_y) through nubar_T = MET - nu_T,
 *    is a second conic;
 *  - the common points of the two conics: the resultant in p_y is a quartic in
 *    p_x (roots by the Durand-Kerner iteration in complex FP64, real ones polished
 *    by Newton steps on the two conics), p_y from the linear combination of the
 *    conics without the p_y^2 term; solutions with positive neutrino energies are
 *    kept and refined by Newton steps on the four virtualities themselves with
 *    exactly massless neutrinos (the conic coefficients lose digits to
 *    cancellation; the direct residual does not).
 * Each solution carries 1 / |det d(q2_W+, q2_t, q2_W-, q2_tbar) / d(nu_x, nu_y,
 * nu_z, nubar_z)|, the Jacobian of trading the neutrino momenta (with the MET
 * constraint applied) for the four virtualities.
 */
#include <complex.h>
#include <math.h>
#include <string.h>

#include "oracle.h"

/* conic C(x, y) = c[0] x^2 + c[1] x y + c[2] y^2 + c[3] x + c[4] y + c[5] */
typedef struct {
  double c[6];
} conic_t;

static double conic_at(const conic_t* q, double x, double y) {
  return q->c[0] * x * x + q->c[1] * x * y + q->c[2] * y * y + q->c[3] * x + q->c[4] * y + q->c[5];
}

/* Energy and p_z of a massless neutrino as linear functions e0 + ex x + ey y and
 * z0 + zx x + zy y of its (x, y) = (p_x, p_y), from 2 l.nu = h1' and 2 b.nu = h2'. */
typedef struct {
  double e0, ex, ey, z0, zx, zy;
  int ok;
} linear_t;

static linear_t nu_linear(const double* l, const double* b, double q2w, double q2t) {
  linear_t r;
  const double m2bl = 2.0 * (b[0] * l[0] - b[1] * l[1] - b[2] * l[2] - b[3] * l[3]);
  const double h1 = 0.5 * q2w, h2 = 0.5 * (q2t - q2w - m2bl);
  /* E_l E - l_z z = h1 + l_x x + l_y y ;  E_b E - b_z z = h2 + b_x x + b_y y */
  const double det = -l[0] * b[3] + l[3] * b[0];
  r.ok = fabs(det) > 1e-12 * (fabs(l[0] * b[3]) + fabs(l[3] * b[0]) + 1e-300);
  if (!r.ok) return r;
  r.e0 = (-b[3] * h1 + l[3] * h2) / det;
  r.ex = (-b[3] * l[1] + l[3] * b[1]) / det;
  r.ey = (-b[3] * l[2] + l[3] * b[2]) / det;
  r.z0 = (l[0] * h2 - b[0] * h1) / det;
  r.zx = (l[0] * b[1] - b[0] * l[1]) / det;
  r.zy = (l[0] * b[2] - b[0] * l[2]) / det;
  return r;
}

/* E^2 - x^2 - y^2 - z^2 with E, z linear in (x, y) */
static conic_t shell_conic(const linear_t* L) {
  conic_t q;
  q.c[0] = L->ex * L->ex - 1.0 - L->zx * L->zx;
  q.c[1] = 2.0 * (L->ex * L->ey - L->zx * L->zy);
  q.c[2] = L->ey * L->ey - 1.0 - L->zy * L->zy;
  q.c[3] = 2.0 * (L->e0 * L->ex - L->z0 * L->zx);
  q.c[4] = 2.0 * (L->e0 * L->ey - L->z0 * L->zy);
  q.c[5] = L->e0 * L->e0 - L->z0 * L->z0;
  return q;
}

/* the conic C(X, Y) written in (x, y) with X = mx - x, Y = my - y */
static conic_t reflect(const conic_t* q, double mx, double my) {
  conic_t r;
  const double* c = q->c;
  r.c[0] = c[0];
  r.c[1] = c[1];
  r.c[2] = c[2];
  r.c[3] = -2.0 * c[0] * mx - c[1] * my - c[3];
  r.c[4] = -2.0 * c[2] * my - c[1] * mx - c[4];
  r.c[5] = c[0] * mx * mx + c[1] * mx * my + c[2] * my * my + c[3] * mx + c[4] * my + c[5];
  return r;
}

/* polynomials in x: p[k] = coefficient of x^k */
static void pmul(const double* a, int na, const double* b, int nb, double* out) {
  for (int k = 0; k < na + nb - 1; ++k) out[k] = 0.0;
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < nb; ++j) out[i + j] += a[i] * b[j];
}

/* All roots of the polynomial p (degree n <= 4, p[n] != 0) by the Durand-Kerner
 * (Weierstrass) simultaneous iteration in complex FP64. */
static int poly_roots(const double* p, int n, double complex* z) {
  double m[5];
  for (int k = 0; k <= n; ++k) m[k] = p[k] / p[n];
  double R = 1.0;
  for (int k = 0; k < n; ++k) R = fmax(R, 1.0 + fabs(m[k]));
  for (int i = 0; i < n; ++i) z[i] = R * cpow(0.4 + 0.9 * I, i) * 0.5;
  for (int it = 0; it < 2000; ++it) {
    double change = 0.0;
    for (int i = 0; i < n; ++i) {
      double complex v = 1.0;
      for (int k = n - 1; k >= 0; --k) v = v * z[i] + m[k];
      double complex d = 1.0;
      for (int j = 0; j < n; ++j)
        if (j != i) d *= z[i] - z[j];
      if (cabs(d) == 0.0) d = 1e-300;
      const double complex step = v / d;
      z[i] -= step;
      change = fmax(change, cabs(step) / (1.0 + cabs(z[i])));
    }
    if (change < 1e-15) break;
  }
  return n;
}

/* Newton steps on the two conics in (x, y) */
static void polish(const conic_t* a, const conic_t* b, double* x, double* y) {
  for (int it = 0; it < 8; ++it) {
    const double f = conic_at(a, *x, *y), g = conic_at(b, *x, *y);
    const double fx = 2 * a->c[0] * *x + a->c[1] * *y + a->c[3];
    const double fy = a->c[1] * *x + 2 * a->c[2] * *y + a->c[4];
    const double gx = 2 * b->c[0] * *x + b->c[1] * *y + b->c[3];
    const double gy = b->c[1] * *x + 2 * b->c[2] * *y + b->c[4];
    const double det = fx * gy - fy * gx;
    if (det == 0.0) return;
    const double dx = (f * gy - g * fy) / det, dy = (g * fx - f * gx) / det;
    *x -= dx;
    *y -= dy;
    if (fabs(dx) + fabs(dy) < 1e-14 * (1.0 + fabs(*x) + fabs(*y))) return;
  }
}

static double m2sum(const double* a, const double* b, const double* c) {
  double t[4];
  for (int k = 0; k < 4; ++k) t[k] = a[k] + b[k] + (c ? c[k] : 0.0);
  return t[0] * t[0] - t[1] * t[1] - t[2] * t[2] - t[3] * t[3];
}

/* The four virtualities (W+, t, W-, tbar) of on-shell neutrinos with free
 * components f = (nu_x, nu_y, nu_z, nubar_z), nubar_T = MET - nu_T, and their
 * derivatives M = d(q2) / d(f) (scaled units). */
static void forward(const double* b, const double* bb, const double* lp, const double* lm,
                    double mx, double my, const double* f, double* q, double M[4][4], double* nu,
                    double* nub) {
  nu[1] = f[0];
  nu[2] = f[1];
  nu[3] = f[2];
  nu[0] = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  nub[1] = mx - f[0];
  nub[2] = my - f[1];
  nub[3] = f[3];
  nub[0] = sqrt(nub[1] * nub[1] + nub[2] * nub[2] + nub[3] * nub[3]);
  q[0] = m2sum(lp, nu, NULL);
  q[1] = m2sum(b, lp, nu);
  q[2] = m2sum(lm, nub, NULL);
  q[3] = m2sum(bb, lm, nub);
  /* d(P + nu)^2 / d nu_k = 2 (P_0 nu_k / E - P_k) for massless nu */
  for (int k = 0; k < 3; ++k) {
    M[0][k] = 2.0 * (lp[0] * nu[1 + k] / nu[0] - lp[1 + k]);
    M[1][k] = 2.0 * ((b[0] + lp[0]) * nu[1 + k] / nu[0] - (b[1 + k] + lp[1 + k]));
  }
  M[0][3] = M[1][3] = 0.0;
  /* nubar_x = mx - nu_x, nubar_y = my - nu_y: d/dnu_x, d/dnu_y carry a minus sign */
  for (int k = 0; k < 2; ++k) {
    M[2][k] = -2.0 * (lm[0] * nub[1 + k] / nub[0] - lm[1 + k]);
    M[3][k] = -2.0 * ((bb[0] + lm[0]) * nub[1 + k] / nub[0] - (bb[1 + k] + lm[1 + k]));
  }
  M[2][2] = M[3][2] = 0.0;
  M[2][3] = 2.0 * (lm[0] * nub[3] / nub[0] - lm[3]);
  M[3][3] = 2.0 * ((bb[0] + lm[0]) * nub[3] / nub[0] - (bb[3] + lm[3]));
}

/* Solves M d = r (4x4, partial pivoting); returns 0 when singular. */
static int solve4(double m[4][4], double* r) {
  double a[4][5];
  for (int i = 0; i < 4; ++i) {
    for (int k = 0; k < 4; ++k) a[i][k] = m[i][k];
    a[i][4] = r[i];
  }
  for (int c = 0; c < 4; ++c) {
    int p = c;
    for (int i = c + 1; i < 4; ++i)
      if (fabs(a[i][c]) > fabs(a[p][c])) p = i;
    if (a[p][c] == 0.0) return 0;
    for (int k = 0; k < 5; ++k) {
      const double t = a[c][k];
      a[c][k] = a[p][k];
      a[p][k] = t;
    }
    for (int i = c + 1; i < 4; ++i) {
      const double f = a[i][c] / a[c][c];
      for (int k = c; k < 5; ++k) a[i][k] -= f * a[c][k];
    }
  }
  for (int c = 3; c >= 0; --c) {
    double v = a[c][4];
    for (int k = c + 1; k < 4; ++k) v -= a[c][k] * r[k];
    r[c] = v / a[c][c];
  }
  return 1;
}

static double det4(double m[4][4]) {
  double a[4][4];
  memcpy(a, m, sizeof(a));
  double det = 1.0;
  for (int c = 0; c < 4; ++c) {
    int p = c;
    for (int r = c + 1; r < 4; ++r)
      if (fabs(a[r][c]) > fabs(a[p][c])) p = r;
    if (a[p][c] == 0.0) return 0.0;
    if (p != c) {
      for (int k = 0; k < 4; ++k) {
        double t = a[c][k];
        a[c][k] = a[p][k];
        a[p][k] = t;
      }
      det = -det;
    }
    det *= a[c][c];
    for (int r = c + 1; r < 4; ++r) {
      const double f = a[r][c] / a[c][c];
      for (int k = c; k < 4; ++k) a[r][k] -= f * a[c][k];
    }
  }
  return det;
}

int ora_dilep_nu(const double* pb, const double* pbb, const double* plp, const double* plm,
                 double metx, double mety, double q2wp, double q2wm, double q2t, double q2tb,
                 double* nu_out, double* nub_out, double* jac_out) {
  /* work in units of S GeV (numbers of order 1) */
  const double S = 100.0, S2 = S * S;
  double b[4], bb[4], lp[4], lm[4];
  for (int k = 0; k < 4; ++k) {
    b[k] = pb[k] / S;
    bb[k] = pbb[k] / S;
    lp[k] = plp[k] / S;
    lm[k] = plm[k] / S;
  }
  const double mx = metx / S, my = mety / S;
  const linear_t L1 = nu_linear(lp, b, q2wp / S2, q2t / S2);
  const linear_t L2 = nu_linear(lm, bb, q2wm / S2, q2tb / S2);
  if (!L1.ok || !L2.ok) return 0;
  const conic_t c1 = shell_conic(&L1);
  const conic_t s2 = shell_conic(&L2);
  const conic_t c2 = reflect(&s2, mx, my);
  /* as polynomials in y: a y^2 + b(x) y + c(x) */
  const double a1 = c1.c[2], a2 = c2.c[2];
  const double b1[2] = {c1.c[4], c1.c[1]}, b2[2] = {c2.c[4], c2.c[1]};
  const double cc1[3] = {c1.c[5], c1.c[3], c1.c[0]}, cc2[3] = {c2.c[5], c2.c[3], c2.c[0]};
  /* resultant: (a1 c2 - a2 c1)^2 - (a1 b2 - a2 b1)(b1 c2 - b2 c1) */
  double u[3], v[2], w[4], t1[4], t2[4], sq[5], pr[5], R[5];
  for (int k = 0; k < 3; ++k) u[k] = a1 * cc2[k] - a2 * cc1[k];
  for (int k = 0; k < 2; ++k) v[k] = a1 * b2[k] - a2 * b1[k];
  pmul(b1, 2, cc2, 3, t1);
  pmul(b2, 2, cc1, 3, t2);
  for (int k = 0; k < 4; ++k) w[k] = t1[k] - t2[k];
  pmul(u, 3, u, 3, sq);
  pmul(v, 2, w, 4, pr);
  double scale = 0.0;
  for (int k = 0; k < 5; ++k) {
    R[k] = sq[k] - pr[k];
    scale = fmax(scale, fabs(R[k]));
  }
  if (scale == 0.0) return 0;
  int deg = 4;
  while (deg > 0 && fabs(R[deg]) <= 1e-13 * scale) --deg;
  if (deg == 0) return 0;
  double complex z[4];
  poly_roots(R, deg, z);
  int n = 0;
  double sols[4][2];
  for (int i = 0; i < deg; ++i) {
    const double xr = creal(z[i]);
    if (fabs(cimag(z[i])) > 1e-6 * (1.0 + fabs(xr))) continue;
    double y;
    const double den = v[0] + v[1] * xr;
    const double num = -(u[0] + u[1] * xr + u[2] * xr * xr);
    if (fabs(den) > 1e-12 * (fabs(num) + 1.0)) {
      y = num / den;
    } else {
      /* common y from the first conic's quadratic, the one that fits the second */
      const double bq = b1[0] + b1[1] * xr, cq = cc1[0] + cc1[1] * xr + cc1[2] * xr * xr;
      const double disc = bq * bq - 4.0 * a1 * cq;
      if (disc < 0.0 || a1 == 0.0) continue;
      const double y1 = (-bq + sqrt(disc)) / (2.0 * a1), y2 = (-bq - sqrt(disc)) / (2.0 * a1);
      y = fabs(conic_at(&c2, xr, y1)) < fabs(conic_at(&c2, xr, y2)) ? y1 : y2;
    }
    double x = xr;
    polish(&c1, &c2, &x, &y);
    /* both conics satisfied, and not a duplicate of an earlier solution */
    const double tol = 1e-8 * (1.0 + x * x + y * y);
    if (fabs(conic_at(&c1, x, y)) > tol || fabs(conic_at(&c2, x, y)) > tol) continue;
    int dup = 0;
    for (int k = 0; k < n; ++k)
      if (fabs(sols[k][0] - x) + fabs(sols[k][1] - y) < 1e-9 * (1.0 + fabs(x) + fabs(y))) dup = 1;
    if (dup) continue;
    const double E = L1.e0 + L1.ex * x + L1.ey * y, zz = L1.z0 + L1.zx * x + L1.zy * y;
    const double X = mx - x, Y = my - y;
    const double Eb = L2.e0 + L2.ex * X + L2.ey * Y, zb = L2.z0 + L2.zx * X + L2.zy * Y;
    if (!(E > 0.0 && Eb > 0.0)) continue;
    sols[n][0] = x;
    sols[n][1] = y;
    /* Newton steps on the original four equations with exactly massless neutrinos:
     * the conic coefficients carry cancellations that the direct residual has not */
    double f[4] = {x, y, zz, zb}, q[4], M[4][4], nv[4], nb[4];
    const double tq[4] = {q2wp / S2, q2t / S2, q2wm / S2, q2tb / S2};
    for (int it = 0; it < 3; ++it) {
      forward(b, bb, lp, lm, mx, my, f, q, M, nv, nb);
      double r[4];
      for (int k = 0; k < 4; ++k) r[k] = q[k] - tq[k];
      if (!solve4(M, r)) break;
      for (int k = 0; k < 4; ++k) f[k] -= r[k];
    }
    forward(b, bb, lp, lm, mx, my, f, q, M, nv, nb);
    /* Jacobian d(q2_W+, q2_t, q2_W-, q2_tbar) / d(nu_x, nu_y, nu_z, nubar_z), GeV units */
    /* q2 in units of S^2 and momenta in units of S: each entry scales by S */
    const double det = det4(M) * S2 * S2;
    if (det == 0.0) continue;
    double* no = nu_out + 4 * n;
    double* nbo = nub_out + 4 * n;
    for (int k = 0; k < 4; ++k) {
      no[k] = nv[k] * S;
      nbo[k] = nb[k] * S;
    }
    jac_out[n] = 1.0 / fabs(det);
    ++n;
  }
  return n;
}

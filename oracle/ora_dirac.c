/* Dirac matrices, slashes and spinors for the oracle (test infrastructure;
 * see oracle.h). Textbook Dirac representation, no shortcuts. */
#include <math.h>

#include "ora_dirac.h"

rv4 rv(double e, double x, double y, double z) {
  rv4 r = {{e, x, y, z}};
  return r;
}
rv4 rv_add(rv4 a, rv4 b) {
  for (int i = 0; i < 4; ++i) a.v[i] += b.v[i];
  return a;
}
rv4 rv_sub(rv4 a, rv4 b) {
  for (int i = 0; i < 4; ++i) a.v[i] -= b.v[i];
  return a;
}
rv4 rv_scale(rv4 a, double s) {
  for (int i = 0; i < 4; ++i) a.v[i] *= s;
  return a;
}
double rv_dot(rv4 a, rv4 b) {
  return a.v[0] * b.v[0] - a.v[1] * b.v[1] - a.v[2] * b.v[2] - a.v[3] * b.v[3];
}
cv4 cv_from_rv(rv4 a) {
  cv4 c;
  for (int i = 0; i < 4; ++i) c.v[i] = a.v[i];
  return c;
}
cplx cv_dot(cv4 a, cv4 b) {
  return a.v[0] * b.v[0] - a.v[1] * b.v[1] - a.v[2] * b.v[2] - a.v[3] * b.v[3];
}
cv4 cv_lin(cplx a, cv4 x, cplx b, cv4 y) {
  cv4 r;
  for (int i = 0; i < 4; ++i) r.v[i] = a * x.v[i] + b * y.v[i];
  return r;
}

dmat d_zero(void) {
  dmat z;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) z.m[i][j] = 0;
  return z;
}
dmat d_unit(void) {
  dmat z = d_zero();
  for (int i = 0; i < 4; ++i) z.m[i][i] = 1;
  return z;
}

/* Pauli matrices sigma_k, k = 1..3 */
static cplx pauli(int k, int i, int j) {
  if (k == 1) return (i != j) ? 1.0 : 0.0;
  if (k == 2) {
    if (i == 0 && j == 1) return -I;
    if (i == 1 && j == 0) return I;
    return 0.0;
  }
  if (i != j) return 0.0;
  return i == 0 ? 1.0 : -1.0;
}

dmat d_gamma(int mu) {
  dmat g = d_zero();
  if (mu == 0) {
    g.m[0][0] = 1; g.m[1][1] = 1; g.m[2][2] = -1; g.m[3][3] = -1;
    return g;
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      g.m[i][2 + j] = pauli(mu, i, j);
      g.m[2 + i][j] = -pauli(mu, i, j);
    }
  return g;
}
dmat d_gamma5(void) {
  dmat g = d_zero();
  g.m[0][2] = 1; g.m[1][3] = 1; g.m[2][0] = 1; g.m[3][1] = 1;
  return g;
}
dmat d_add(dmat a, dmat b) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) a.m[i][j] += b.m[i][j];
  return a;
}
dmat d_scale(dmat a, cplx s) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) a.m[i][j] *= s;
  return a;
}
dmat d_PL(void) { return d_scale(d_add(d_unit(), d_scale(d_gamma5(), -1.0)), 0.5); }
dmat d_PR(void) { return d_scale(d_add(d_unit(), d_gamma5()), 0.5); }
dmat d_mul(dmat a, dmat b) {
  dmat c = d_zero();
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      cplx s = 0;
      for (int k = 0; k < 4; ++k) s += a.m[i][k] * b.m[k][j];
      c.m[i][j] = s;
    }
  return c;
}
dmat d_slash(cv4 a) {
  /* a_mu gamma^mu = a^0 gamma^0 - a^k gamma^k */
  dmat s = d_scale(d_gamma(0), a.v[0]);
  for (int k = 1; k < 4; ++k) s = d_add(s, d_scale(d_gamma(k), -a.v[k]));
  return s;
}
dmat d_slash_r(rv4 a) { return d_slash(cv_from_rv(a)); }
spin d_mv(dmat a, spin x) {
  spin y;
  for (int i = 0; i < 4; ++i) {
    cplx s = 0;
    for (int k = 0; k < 4; ++k) s += a.m[i][k] * x.s[k];
    y.s[i] = s;
  }
  return y;
}
spin d_vm(spin row, dmat a) {
  spin y;
  for (int j = 0; j < 4; ++j) {
    cplx s = 0;
    for (int k = 0; k < 4; ++k) s += row.s[k] * a.m[k][j];
    y.s[j] = s;
  }
  return y;
}
cplx d_rc(spin row, spin col) {
  cplx s = 0;
  for (int k = 0; k < 4; ++k) s += row.s[k] * col.s[k];
  return s;
}
spin d_bar(spin u) {
  spin r;
  r.s[0] = conj(u.s[0]);
  r.s[1] = conj(u.s[1]);
  r.s[2] = -conj(u.s[2]);
  r.s[3] = -conj(u.s[3]);
  return r;
}

/* (sigma . a) chi for a real 3-vector a and basis vector chi_s */
static void sigma_dot(const double* a3, int s, cplx* out2) {
  for (int i = 0; i < 2; ++i) {
    cplx acc = 0;
    for (int k = 1; k <= 3; ++k) acc += a3[k - 1] * pauli(k, i, s);
    out2[i] = acc;
  }
}

spin d_massless(rv4 p, int s) {
  double E = p.v[0];
  double a3[3] = {p.v[1] / E, p.v[2] / E, p.v[3] / E};
  cplx lo[2];
  sigma_dot(a3, s, lo);
  double r = sqrt(E);
  spin u;
  u.s[0] = (s == 0) ? r : 0.0;
  u.s[1] = (s == 1) ? r : 0.0;
  u.s[2] = r * lo[0];
  u.s[3] = r * lo[1];
  return u;
}
spin d_massive_u(rv4 p, double m, int s) {
  double E = p.v[0];
  double a3[3] = {p.v[1], p.v[2], p.v[3]};
  cplx lo[2];
  sigma_dot(a3, s, lo);
  double r = sqrt(E + m);
  spin u;
  u.s[0] = (s == 0) ? r : 0.0;
  u.s[1] = (s == 1) ? r : 0.0;
  u.s[2] = lo[0] / r;
  u.s[3] = lo[1] / r;
  return u;
}
spin d_massive_v(rv4 p, double m, int s) {
  double E = p.v[0];
  double a3[3] = {p.v[1], p.v[2], p.v[3]};
  cplx up[2];
  sigma_dot(a3, s, up);
  double r = sqrt(E + m);
  spin v;
  v.s[0] = up[0] / r;
  v.s[1] = up[1] / r;
  v.s[2] = (s == 0) ? r : 0.0;
  v.s[3] = (s == 1) ? r : 0.0;
  return v;
}
cv4 d_current(spin row, dmat P, spin col) {
  cv4 J;
  spin pc = d_mv(P, col);
  for (int mu = 0; mu < 4; ++mu) J.v[mu] = d_rc(row, d_mv(d_gamma(mu), pc));
  return J;
}

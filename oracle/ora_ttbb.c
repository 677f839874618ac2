/* Tree-level |M|^2 of g g -> t tbar b bbar and q qbar -> t tbar b bbar (the ttbb
 * background of Sec. 3-4) for the oracle (test infrastructure; see oracle.h).
 *
 * Written out diagram by diagram from the QCD Feynman rules (Feynman gauge):
 *   quark-gluon vertex      i g gamma^mu t^a
 *   quark propagator        i (q/ + m) / (q^2 - m^2)
 *   gluon propagator        -i g_{mu nu} delta^{ab} / q^2
 *   three-gluon vertex      g f^{abc} [g^{mu nu}(k - p)^rho + g^{nu rho}(p - q)^mu
 *                                      + g^{rho mu}(q - k)^nu], all momenta incoming
 *   four-gluon vertex       -i g^2 [f^{abe}f^{cde}(g^{mu rho}g^{nu sigma} - g^{mu sigma}g^{nu rho})
 *                                  + f^{ace}f^{bde}(g^{mu nu}g^{rho sigma} - g^{mu sigma}g^{nu rho})
 *                                  + f^{ade}f^{bce}(g^{mu nu}g^{rho sigma} - g^{mu rho}g^{nu sigma})].
 * Each diagram is split into a Lorentz part (a number per helicity configuration) and a
 * colour tensor over the external colours, evaluated by explicit sums over the internal
 * colours with the Gell-Mann generators t^a = lambda^a / 2. The colour-summed |M|^2 is
 * L^dagger K L with K_nm = sum over external colours of conj(C_n) C_m.
 *
 * g g: 36 diagrams (38 terms: the four-gluon vertex has three colour structures):
 *   A (6)  both gluons and the b bbar gluon on the top line, every order;
 *   B (6)  both gluons and the t tbar gluon on the b line;
 *   C (8)  one gluon on each line, the lines joined by a gluon, every order;
 *   D (4)  g g -> g* (three-gluon vertex) onto one line, the other pair from that line;
 *   E (8)  one external gluon and the two pair gluons meet at a three-gluon vertex whose
 *          third gluon joins the line that carries the other external gluon;
 *   F (1)  the four-gluon vertex joining both gluons and both pair gluons;
 *   G (3)  two three-gluon vertices (s-channel g* -> two pair gluons, and the two
 *          exchanges of a gluon between (g1, t tbar) and (g2, b bbar) vertices).
 * q qbar (q a light quark, massless): 7 diagrams -- q qbar -> g* onto the top line with
 * the b bbar gluon from it or onto the b line with the t tbar gluon (4), q qbar -> g* ->
 * the two pair gluons (1), and both pair gluons from the light line (2).
 */
#include <math.h>
#include <string.h>

#include "oracle.h"
#include "ora_dirac.h"

/* ------------------------------------------------------------ SU(3) */
static cplx Tm[8][3][3];
static double Ff[8][8][8];
static int su3_ready = 0;

static void su3_init(void) {
  if (su3_ready) return;
  memset(Tm, 0, sizeof(Tm));
  const double h = 0.5, r3 = 1.0 / sqrt(3.0);
  Tm[0][0][1] = h; Tm[0][1][0] = h;
  Tm[1][0][1] = -I * h; Tm[1][1][0] = I * h;
  Tm[2][0][0] = h; Tm[2][1][1] = -h;
  Tm[3][0][2] = h; Tm[3][2][0] = h;
  Tm[4][0][2] = -I * h; Tm[4][2][0] = I * h;
  Tm[5][1][2] = h; Tm[5][2][1] = h;
  Tm[6][1][2] = -I * h; Tm[6][2][1] = I * h;
  Tm[7][0][0] = h * r3; Tm[7][1][1] = h * r3; Tm[7][2][2] = -2.0 * h * r3;
  /* f^{abc} = -2 i Tr([t^a, t^b] t^c) */
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b)
      for (int c = 0; c < 8; ++c) {
        cplx tr = 0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
              tr += (Tm[a][i][j] * Tm[b][j][k] - Tm[b][i][j] * Tm[a][j][k]) * Tm[c][k][i];
        Ff[a][b][c] = creal(-2.0 * I * tr);
      }
  su3_ready = 1;
}

/* (t^{x1} t^{x2} ... )_{ij} for a list of adjoint indices */
static cplx tprod(const int* x, int n, int i, int j) {
  cplx M[3][3], R[3][3];
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) M[p][q] = (p == q);
  for (int s = 0; s < n; ++s) {
    for (int p = 0; p < 3; ++p)
      for (int q = 0; q < 3; ++q) {
        R[p][q] = 0;
        for (int r = 0; r < 3; ++r) R[p][q] += M[p][r] * Tm[x[s]][r][q];
      }
    memcpy(M, R, sizeof(M));
  }
  return M[i][j];
}

/* ------------------------------------------------------------ Lorentz pieces */
typedef struct {
  const ora_process* P;
  double g, m;
} ctx_t;

/* i g gamma^mu v_mu (v contravariant) */
static dmat vtx(const ctx_t* c, cv4 v) { return d_scale(d_slash(v), I * c->g); }
/* i g gamma^mu for an open index mu */
static dmat vtx_open(const ctx_t* c, int mu) { return d_scale(d_gamma(mu), I * c->g); }
static dmat qprop(rv4 q, double m) {
  return d_scale(d_add(d_slash_r(q), d_scale(d_unit(), m)), I / (rv_dot(q, q) - m * m));
}

/* row X1 S(q1) X2 S(q2) ... Xn col, q1 = p_out - in1, q2 = q1 - in2, ... */
static cplx chain(spin row, spin col, rv4 pout, double m, int n, const dmat* X, const rv4* kin) {
  dmat M = X[0];
  rv4 q = pout;
  for (int s = 1; s < n; ++s) {
    q = rv_sub(q, kin[s - 1]);
    M = d_mul(d_mul(M, qprop(q, m)), X[s]);
  }
  return d_rc(row, d_mv(M, col));
}

/* the same with one vertex (position pos) left open: the contravariant vector
 * J^mu = row ... (i g gamma^mu) ... col */
static cv4 chain_open(const ctx_t* c, spin row, spin col, rv4 pout, double m, int n,
                      const dmat* X, const rv4* kin, int pos) {
  dmat Y[4];
  for (int s = 0; s < n; ++s) Y[s] = X[s];
  cv4 J;
  for (int mu = 0; mu < 4; ++mu) {
    Y[pos] = vtx_open(c, mu);
    J.v[mu] = chain(row, col, pout, m, n, Y, kin);
  }
  return J;
}

/* gluon propagator applied to a current: -i J / q^2 */
static cv4 gprop(cv4 J, rv4 q) { return cv_lin(-I / rv_dot(q, q), J, 0.0, J); }

/* three-gluon vertex (Lorentz part, g f^{abc} stripped to g) contracted with A (leg 1,
 * momentum kA), B (leg 2, kB): the vector of leg 3 (incoming momentum kC = -kA - kB) */
static cv4 v3(const ctx_t* c, cv4 A, rv4 kA, cv4 B, rv4 kB) {
  rv4 kC = rv_scale(rv_add(kA, kB), -1.0);
  cv4 kAB = cv_from_rv(rv_sub(kA, kB)), kBC = cv_from_rv(rv_sub(kB, kC)),
      kCA = cv_from_rv(rv_sub(kC, kA));
  cv4 r = cv_lin(cv_dot(A, B), kAB, cv_dot(kBC, A), B);
  r = cv_lin(1.0, r, cv_dot(kCA, B), A);
  return cv_lin(c->g, r, 0.0, r);
}
/* fully contracted three-gluon vertex */
static cplx v3full(const ctx_t* c, cv4 A, rv4 kA, cv4 B, rv4 kB, cv4 C) {
  return cv_dot(v3(c, A, kA, B, kB), C);
}

/* ------------------------------------------------------------ g g -> t tbar b bbar */
#define NT_GG 38

/* Lorentz parts of the 38 terms for one helicity configuration. The colour tensor of
 * term n is gg_colour(n, a, b, i, j, k, l); both lists are in the same order. */
static void gg_lorentz(const ctx_t* c, rv4 k1, rv4 k2, rv4 p1, rv4 p2, rv4 p3, rv4 p4, cv4 e1,
                       cv4 e2, spin rt, spin ct, spin rb, spin cb, cplx* L) {
  const double m = c->m;
  rv4 P12 = rv_add(p1, p2), P34 = rv_add(p3, p4);
  rv4 mP12 = rv_scale(P12, -1.0), mP34 = rv_scale(P34, -1.0);
  /* pair gluons (after their propagators), entering the other side with momentum -Pij */
  dmat one[1];
  cv4 Gt, Gb;
  {
    one[0] = d_unit();
    Gt = gprop(chain_open(c, rt, ct, p1, m, 1, one, NULL, 0), P12);
    Gb = gprop(chain_open(c, rb, cb, p3, 0.0, 1, one, NULL, 0), P34);
  }
  cv4 E[2] = {e1, e2};
  rv4 K[2] = {k1, k2};
  int n = 0;
  /* A: top line with e1, e2, Gb in every order (6) */
  {
    const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    cv4 V[3] = {e1, e2, Gb};
    rv4 kin[3] = {k1, k2, mP34};
    for (int p = 0; p < 6; ++p) {
      dmat X[3];
      rv4 ki[3];
      for (int s = 0; s < 3; ++s) {
        X[s] = vtx(c, V[perm[p][s]]);
        ki[s] = kin[perm[p][s]];
      }
      L[n++] = chain(rt, ct, p1, m, 3, X, ki);
    }
    /* B: b line with e1, e2, Gt (6) */
    cv4 W[3] = {e1, e2, Gt};
    rv4 kw[3] = {k1, k2, mP12};
    for (int p = 0; p < 6; ++p) {
      dmat X[3];
      rv4 ki[3];
      for (int s = 0; s < 3; ++s) {
        X[s] = vtx(c, W[perm[p][s]]);
        ki[s] = kw[perm[p][s]];
      }
      L[n++] = chain(rb, cb, p3, 0.0, 3, X, ki);
    }
  }
  /* C: gluon x on the top line, y on the b line, joined by a gluon (8) */
  for (int x = 0; x < 2; ++x) {
    const int y = 1 - x;
    for (int bo = 0; bo < 2; ++bo) {   /* b-line order: 0 = (e_y, open), 1 = (open, e_y) */
      dmat Xb[2];
      rv4 kb[2];
      rv4 qin = rv_sub(P34, K[y]);     /* momentum the joining gluon brings into the b line */
      Xb[bo] = vtx(c, E[y]);
      kb[bo] = K[y];
      Xb[1 - bo] = d_unit();
      kb[1 - bo] = qin;
      cv4 J = gprop(chain_open(c, rb, cb, p3, 0.0, 2, Xb, kb, 1 - bo), qin);
      for (int to = 0; to < 2; ++to) { /* top-line order: 0 = (e_x, J), 1 = (J, e_x) */
        dmat Xt[2];
        rv4 kt[2];
        Xt[to] = vtx(c, E[x]);
        kt[to] = K[x];
        Xt[1 - to] = vtx(c, J);
        kt[1 - to] = rv_scale(qin, -1.0);
        L[n++] = chain(rt, ct, p1, m, 2, Xt, kt);
      }
    }
  }
  /* D: g g -> g* onto the top line with Gb (2), onto the b line with Gt (2) */
  {
    rv4 K12 = rv_add(k1, k2);
    cv4 Js = gprop(v3(c, e1, k1, e2, k2), K12);
    for (int to = 0; to < 2; ++to) {
      dmat X[2];
      rv4 ki[2];
      X[to] = vtx(c, Js);
      ki[to] = K12;
      X[1 - to] = vtx(c, Gb);
      ki[1 - to] = mP34;
      L[n++] = chain(rt, ct, p1, m, 2, X, ki);
    }
    for (int bo = 0; bo < 2; ++bo) {
      dmat X[2];
      rv4 ki[2];
      X[bo] = vtx(c, Js);
      ki[bo] = K12;
      X[1 - bo] = vtx(c, Gt);
      ki[1 - bo] = mP12;
      L[n++] = chain(rb, cb, p3, 0.0, 2, X, ki);
    }
  }
  /* E: V3(e_x, pair gluon) joining the line with e_y (8) */
  for (int x = 0; x < 2; ++x) {
    const int y = 1 - x;
    /* onto the top line: V3(e_x, Gb) */
    {
      cv4 J = gprop(v3(c, E[x], K[x], Gb, mP34), rv_add(K[x], mP34));
      rv4 qin = rv_add(K[x], mP34);   /* momentum entering the top line */
      for (int to = 0; to < 2; ++to) {
        dmat X[2];
        rv4 ki[2];
        X[to] = vtx(c, E[y]);
        ki[to] = K[y];
        X[1 - to] = vtx(c, J);
        ki[1 - to] = qin;
        L[n++] = chain(rt, ct, p1, m, 2, X, ki);
      }
    }
    /* onto the b line: V3(e_x, Gt) */
    {
      cv4 J = gprop(v3(c, E[x], K[x], Gt, mP12), rv_add(K[x], mP12));
      rv4 qin = rv_add(K[x], mP12);
      for (int bo = 0; bo < 2; ++bo) {
        dmat X[2];
        rv4 ki[2];
        X[bo] = vtx(c, E[y]);
        ki[bo] = K[y];
        X[1 - bo] = vtx(c, J);
        ki[1 - bo] = qin;
        L[n++] = chain(rb, cb, p3, 0.0, 2, X, ki);
      }
    }
  }
  /* F: four-gluon vertex with legs (e1, e2, Gt, Gb), its three structures */
  {
    const cplx ig2 = -I * c->g * c->g;
    cplx e1e2 = cv_dot(e1, e2), e1t = cv_dot(e1, Gt), e1b = cv_dot(e1, Gb);
    cplx e2t = cv_dot(e2, Gt), e2b = cv_dot(e2, Gb), tb = cv_dot(Gt, Gb);
    L[n++] = ig2 * (e1t * e2b - e1b * e2t);      /* f^{abe} f^{cde} */
    L[n++] = ig2 * (e1e2 * tb - e1b * e2t);      /* f^{ace} f^{bde} */
    L[n++] = ig2 * (e1e2 * tb - e1t * e2b);      /* f^{ade} f^{bce} */
  }
  /* G: two three-gluon vertices (3) */
  {
    rv4 K12 = rv_add(k1, k2);
    cv4 Js = gprop(v3(c, e1, k1, e2, k2), K12);
    L[n++] = v3full(c, Js, K12, Gt, mP12, Gb);   /* f^{abe} f^{ecd} */
    cv4 X1 = gprop(v3(c, e1, k1, Gt, mP12), rv_add(k1, mP12));
    L[n++] = v3full(c, e2, k2, Gb, mP34, X1);    /* f^{acx} f^{bdx} */
    cv4 X2 = gprop(v3(c, e2, k2, Gt, mP12), rv_add(k2, mP12));
    L[n++] = v3full(c, e1, k1, Gb, mP34, X2);    /* f^{bcx} f^{adx} */
  }
}

/* colour tensor of term n at external colours (a, b gluons; i, j top, antitop;
 * k, l b, bbar), in gg_lorentz's order */
static cplx gg_colour(int n, int a, int b, int i, int j, int k, int l) {
  cplx s = 0;
  if (n < 6) { /* A: top line t^{x1} t^{x2} t^{x3} with (a, b, c) permuted, t^c on the b line */
    const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int cc = 0; cc < 8; ++cc) {
      int idx[3] = {a, b, cc}, x[3];
      for (int q = 0; q < 3; ++q) x[q] = idx[perm[n][q]];
      s += tprod(x, 3, i, j) * Tm[cc][k][l];
    }
    return s;
  }
  if (n < 12) {
    const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int cc = 0; cc < 8; ++cc) {
      int idx[3] = {a, b, cc}, x[3];
      for (int q = 0; q < 3; ++q) x[q] = idx[perm[n - 6][q]];
      s += tprod(x, 3, k, l) * Tm[cc][i][j];
    }
    return s;
  }
  if (n < 20) { /* C: order x, bo, to as in gg_lorentz */
    const int r = n - 12, xg = r / 4, bo = (r / 2) % 2, to = r % 2;
    const int cx = xg == 0 ? a : b, cy = xg == 0 ? b : a;
    for (int cc = 0; cc < 8; ++cc) {
      int xt[2], xb[2];
      xt[to] = cx;
      xt[1 - to] = cc;
      xb[bo] = cy;
      xb[1 - bo] = cc;
      s += tprod(xt, 2, i, j) * tprod(xb, 2, k, l);
    }
    return s;
  }
  if (n < 24) { /* D: f^{abe}, then e on the line with the pair gluon c */
    const int r = n - 20, line = r / 2, o = r % 2;
    for (int e = 0; e < 8; ++e)
      for (int cc = 0; cc < 8; ++cc) {
        if (Ff[a][b][e] == 0.0) continue;
        int x[2];
        x[o] = e;
        x[1 - o] = cc;
        s += Ff[a][b][e] * (line == 0 ? tprod(x, 2, i, j) * Tm[cc][k][l]
                                      : tprod(x, 2, k, l) * Tm[cc][i][j]);
      }
    return s;
  }
  if (n < 32) { /* E: f^{x c e} (legs e_x, pair gluon c, joining gluon e) */
    const int r = n - 24, xg = r / 4, line = (r / 2) % 2, o = r % 2;
    const int cx = xg == 0 ? a : b, cy = xg == 0 ? b : a;
    for (int cc = 0; cc < 8; ++cc)
      for (int e = 0; e < 8; ++e) {
        if (Ff[cx][cc][e] == 0.0) continue;
        int x[2];
        x[o] = cy;
        x[1 - o] = e;
        s += Ff[cx][cc][e] * (line == 0 ? tprod(x, 2, i, j) * Tm[cc][k][l]
                                        : tprod(x, 2, k, l) * Tm[cc][i][j]);
      }
    return s;
  }
  /* F and G: four-f structures with the pair gluons c (top) and d (b) */
  for (int cc = 0; cc < 8; ++cc)
    for (int d = 0; d < 8; ++d) {
      const cplx td = Tm[cc][i][j] * Tm[d][k][l];
      if (td == 0) continue;
      double f = 0.0;
      for (int e = 0; e < 8; ++e) {
        switch (n) {
          case 32: f += Ff[a][b][e] * Ff[cc][d][e]; break;
          case 33: f += Ff[a][cc][e] * Ff[b][d][e]; break;
          case 34: f += Ff[a][d][e] * Ff[b][cc][e]; break;
          case 35: f += Ff[a][b][e] * Ff[e][cc][d]; break;
          case 36: f += Ff[a][cc][e] * Ff[b][d][e]; break;
          case 37: f += Ff[b][cc][e] * Ff[a][d][e]; break;
        }
      }
      s += f * td;
    }
  return s;
}

static double Kgg[NT_GG][NT_GG][2];   /* colour matrix (real, imaginary) */
static int kgg_ready = 0;

static void gg_colour_matrix(void) {
  if (kgg_ready) return;
  su3_init();
  static cplx C[NT_GG][8 * 8 * 81];
  for (int n = 0; n < NT_GG; ++n) {
    int q = 0;
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
              for (int l = 0; l < 3; ++l) C[n][q++] = gg_colour(n, a, b, i, j, k, l);
  }
  for (int n = 0; n < NT_GG; ++n)
    for (int mm = 0; mm < NT_GG; ++mm) {
      cplx s = 0;
      for (int q = 0; q < 8 * 8 * 81; ++q) s += conj(C[n][q]) * C[mm][q];
      Kgg[n][mm][0] = creal(s);
      Kgg[n][mm][1] = cimag(s);
    }
  kgg_ready = 1;
}

/* ------------------------------------------------------------ q qbar -> t tbar b bbar */
#define NT_QQ 7
/* When J_override is given it replaces the light-quark current (before the gluon
 * propagator) in the four g* terms and the g* -> pair gluons term. */
static void qq_lorentz_x(const ctx_t* c, rv4 kq, rv4 kqb, rv4 p1, rv4 p2, rv4 p3, rv4 p4,
                         spin rq, spin cq, spin rt, spin ct, spin rb, spin cb, cplx* L,
                         const cv4* J_override);
static void qq_lorentz(const ctx_t* c, rv4 kq, rv4 kqb, rv4 p1, rv4 p2, rv4 p3, rv4 p4, spin rq,
                       spin cq, spin rt, spin ct, spin rb, spin cb, cplx* L) {
  qq_lorentz_x(c, kq, kqb, p1, p2, p3, p4, rq, cq, rt, ct, rb, cb, L, NULL);
}
static void qq_lorentz_x(const ctx_t* c, rv4 kq, rv4 kqb, rv4 p1, rv4 p2, rv4 p3, rv4 p4,
                         spin rq, spin cq, spin rt, spin ct, spin rb, spin cb, cplx* L,
                         const cv4* J_override) {
  /* light line: row vbar(kqb), column u(kq); momenta "out" of the line's row end: -kqb */
  const double m = c->m;
  rv4 P12 = rv_add(p1, p2), P34 = rv_add(p3, p4), K = rv_add(kq, kqb);
  rv4 mP12 = rv_scale(P12, -1.0), mP34 = rv_scale(P34, -1.0);
  dmat one[1] = {d_unit()};
  cv4 Gt = gprop(chain_open(c, rt, ct, p1, m, 1, one, NULL, 0), P12);
  cv4 Gb = gprop(chain_open(c, rb, cb, p3, 0.0, 1, one, NULL, 0), P34);
  cv4 Js = gprop(J_override ? *J_override
                            : chain_open(c, rq, cq, rv_scale(kqb, -1.0), 0.0, 1, one, NULL, 0),
                 K);
  int n = 0;
  for (int to = 0; to < 2; ++to) { /* g* onto the top line with Gb */
    dmat X[2];
    rv4 ki[2];
    X[to] = vtx(c, Js);
    ki[to] = K;
    X[1 - to] = vtx(c, Gb);
    ki[1 - to] = mP34;
    L[n++] = chain(rt, ct, p1, m, 2, X, ki);
  }
  for (int bo = 0; bo < 2; ++bo) { /* g* onto the b line with Gt */
    dmat X[2];
    rv4 ki[2];
    X[bo] = vtx(c, Js);
    ki[bo] = K;
    X[1 - bo] = vtx(c, Gt);
    ki[1 - bo] = mP12;
    L[n++] = chain(rb, cb, p3, 0.0, 2, X, ki);
  }
  L[n++] = v3full(c, Js, K, Gt, mP12, Gb);   /* g* -> Gt Gb */
  for (int lo = 0; lo < 2; ++lo) {           /* Gt and Gb both from the light line */
    dmat X[2];
    rv4 ki[2];
    X[lo] = vtx(c, Gt);
    ki[lo] = mP12;
    X[1 - lo] = vtx(c, Gb);
    ki[1 - lo] = mP34;
    L[n++] = chain(rq, cq, rv_scale(kqb, -1.0), 0.0, 2, X, ki);
  }
}

/* colour tensors: light-line indices (iq: q, jq: qbar), the light line read from the
 * qbar row to the q column, i.e. (t ...)_{jq iq} */
static cplx qq_colour(int n, int iq, int jq, int i, int j, int k, int l) {
  cplx s = 0;
  if (n < 4) {
    const int line = n / 2, o = n % 2;
    for (int e = 0; e < 8; ++e)
      for (int cc = 0; cc < 8; ++cc) {
        int x[2];
        x[o] = e;
        x[1 - o] = cc;
        s += Tm[e][jq][iq] * (line == 0 ? tprod(x, 2, i, j) * Tm[cc][k][l]
                                        : tprod(x, 2, k, l) * Tm[cc][i][j]);
      }
    return s;
  }
  if (n == 4) {
    for (int e = 0; e < 8; ++e)
      for (int cc = 0; cc < 8; ++cc)
        for (int d = 0; d < 8; ++d)
          if (Ff[e][cc][d] != 0.0) s += Tm[e][jq][iq] * Ff[e][cc][d] * Tm[cc][i][j] * Tm[d][k][l];
    return s;
  }
  const int o = n - 5;
  for (int cc = 0; cc < 8; ++cc)
    for (int d = 0; d < 8; ++d) {
      int x[2];
      x[o] = cc;
      x[1 - o] = d;
      s += tprod(x, 2, jq, iq) * Tm[cc][i][j] * Tm[d][k][l];
    }
  return s;
}

static double Kqq[NT_QQ][NT_QQ][2];
static int kqq_ready = 0;

static void qq_colour_matrix(void) {
  if (kqq_ready) return;
  su3_init();
  static cplx C[NT_QQ][9 * 81];
  for (int n = 0; n < NT_QQ; ++n) {
    int q = 0;
    for (int iq = 0; iq < 3; ++iq)
      for (int jq = 0; jq < 3; ++jq)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
              for (int l = 0; l < 3; ++l) C[n][q++] = qq_colour(n, iq, jq, i, j, k, l);
  }
  for (int n = 0; n < NT_QQ; ++n)
    for (int mm = 0; mm < NT_QQ; ++mm) {
      cplx s = 0;
      for (int q = 0; q < 9 * 81; ++q) s += conj(C[n][q]) * C[mm][q];
      Kqq[n][mm][0] = creal(s);
      Kqq[n][mm][1] = cimag(s);
    }
  kqq_ready = 1;
}

static double quad_form(int gg, const cplx* L) {
  const int N = gg ? NT_GG : NT_QQ;
  double s = 0.0;
  for (int n = 0; n < N; ++n)
    for (int mm = 0; mm < N; ++mm) {
      const double kr = gg ? Kgg[n][mm][0] : Kqq[n][mm][0];
      const double ki = gg ? Kgg[n][mm][1] : Kqq[n][mm][1];
      s += creal(conj(L[n]) * (kr + I * ki) * L[mm]);
    }
  return s;
}

/* gluon polarisations transverse to the beams (beams along z) */
static cv4 tpol(int h) {
  cv4 e;
  e.v[0] = 0;
  e.v[1] = h == 0 ? 1.0 : 0.0;
  e.v[2] = h == 0 ? 0.0 : 1.0;
  e.v[3] = 0;
  return e;
}

double ora_msq_ttbb_production(const ora_process* P, int channel, const double* k1_,
                               const double* k2_, const double* p1_, const double* p2_,
                               const double* p3_, const double* p4_) {
  rv4 k1 = rv(k1_[0], k1_[1], k1_[2], k1_[3]), k2 = rv(k2_[0], k2_[1], k2_[2], k2_[3]);
  rv4 p1 = rv(p1_[0], p1_[1], p1_[2], p1_[3]), p2 = rv(p2_[0], p2_[1], p2_[2], p2_[3]);
  rv4 p3 = rv(p3_[0], p3_[1], p3_[2], p3_[3]), p4 = rv(p4_[0], p4_[1], p4_[2], p4_[3]);
  ctx_t c = {P, sqrt(4.0 * M_PI * P->alpha_s), P->mt};
  double sum = 0.0;
  if (channel == 0) gg_colour_matrix();
  else qq_colour_matrix();
  for (int st = 0; st < 2; ++st)
    for (int stb = 0; stb < 2; ++stb)
      for (int sb = 0; sb < 2; ++sb)
        for (int sbb = 0; sbb < 2; ++sbb) {
          spin rt = d_bar(d_massive_u(p1, c.m, st)), ct = d_massive_v(p2, c.m, stb);
          spin rb = d_bar(d_massless(p3, sb)), cb = d_massless(p4, sbb);
          if (channel == 0) {
            for (int h1 = 0; h1 < 2; ++h1)
              for (int h2 = 0; h2 < 2; ++h2) {
                cplx L[NT_GG];
                gg_lorentz(&c, k1, k2, p1, p2, p3, p4, tpol(h1), tpol(h2), rt, ct, rb, cb, L);
                sum += quad_form(1, L);
              }
          } else {
            for (int sq = 0; sq < 2; ++sq)
              for (int sqb = 0; sqb < 2; ++sqb) {
                cplx L[NT_QQ];
                spin rq = d_bar(d_massless(k2, sqb)), cq = d_massless(k1, sq);
                qq_lorentz(&c, k1, k2, p1, p2, p3, p4, rq, cq, rt, ct, rb, cb, L);
                sum += quad_form(0, L);
              }
          }
        }
  /* averages: gluons 2 x 2 polarisations x 8 x 8 colours; quarks 2 x 2 spins x 3 x 3 */
  return channel == 0 ? sum / (4.0 * 64.0) : sum / (4.0 * 9.0);
}

/* Gauge probe: sum over spins and colours of |M|^2 with gluon `which` given its
 * momentum as polarisation and the other gluon the transverse state hel. */
double ora_ttbb_gauge_probe(const ora_process* P, const double* k1_, const double* k2_,
                            const double* p1_, const double* p2_, const double* p3_,
                            const double* p4_, int which, int hel) {
  rv4 k1 = rv(k1_[0], k1_[1], k1_[2], k1_[3]), k2 = rv(k2_[0], k2_[1], k2_[2], k2_[3]);
  rv4 p1 = rv(p1_[0], p1_[1], p1_[2], p1_[3]), p2 = rv(p2_[0], p2_[1], p2_[2], p2_[3]);
  rv4 p3 = rv(p3_[0], p3_[1], p3_[2], p3_[3]), p4 = rv(p4_[0], p4_[1], p4_[2], p4_[3]);
  ctx_t c = {P, sqrt(4.0 * M_PI * P->alpha_s), P->mt};
  gg_colour_matrix();
  double sum = 0.0;
  for (int st = 0; st < 2; ++st)
    for (int stb = 0; stb < 2; ++stb)
      for (int sb = 0; sb < 2; ++sb)
        for (int sbb = 0; sbb < 2; ++sbb) {
          spin rt = d_bar(d_massive_u(p1, c.m, st)), ct = d_massive_v(p2, c.m, stb);
          spin rb = d_bar(d_massless(p3, sb)), cb = d_massless(p4, sbb);
          cv4 e1 = tpol(hel), e2 = tpol(hel);
          if (which == 0) e1 = cv_from_rv(k1);
          else e2 = cv_from_rv(k2);
          cplx L[NT_GG];
          gg_lorentz(&c, k1, k2, p1, p2, p3, p4, e1, e2, rt, ct, rb, cb, L);
          sum += quad_form(1, L);
        }
  return sum;
}

/* SU(3) checks for the tests: out = (sum_{a,b,i,j} |(t^a t^b)_ij|^2,
 * sum conj((t^a t^b)_ij) (t^b t^a)_ij, sum_a (t^a t^a)_00, sum_{c,d} f^{0cd} f^{0cd},
 * max_{a,b} |Tr(t^a t^b) - delta_ab / 2|). */
void ora_su3_check(double* out) {
  su3_init();
  double s1 = 0.0, cf = 0.0, ca = 0.0, dev = 0.0;
  cplx s2 = 0;
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b) {
      int ab[2] = {a, b}, ba[2] = {b, a};
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          const cplx x = tprod(ab, 2, i, j), y = tprod(ba, 2, i, j);
          s1 += creal(x * conj(x));
          s2 += conj(x) * y;
        }
      cplx tr = 0;
      for (int i = 0; i < 3; ++i) tr += tprod(ab, 2, i, i);
      dev = fmax(dev, cabs(tr - (a == b ? 0.5 : 0.0)));
    }
  for (int a = 0; a < 8; ++a) {
    int aa[2] = {a, a};
    cf += creal(tprod(aa, 2, 0, 0));
  }
  for (int c = 0; c < 8; ++c)
    for (int d = 0; d < 8; ++d) ca += Ff[0][c][d] * Ff[0][c][d];
  out[0] = s1;
  out[1] = creal(s2);
  out[2] = cf;
  out[3] = ca;
  out[4] = dev;
}

/* Ward probe of the q qbar channel: the g* -> t tbar b bbar part (every term but the two
 * with both pair gluons on the light line), its colour-summed square summed over the
 * top and b spins, with the light-quark current replaced by the gluon momentum K
 * (out[0]; zero by current conservation) and by sqrt(s) times a transverse unit vector
 * (out[1], the scale to compare with). */
void ora_ttbb_qq_ward_probe(const ora_process* P, const double* k1_, const double* k2_,
                            const double* p1_, const double* p2_, const double* p3_,
                            const double* p4_, double* out) {
  rv4 k1 = rv(k1_[0], k1_[1], k1_[2], k1_[3]), k2 = rv(k2_[0], k2_[1], k2_[2], k2_[3]);
  rv4 p1 = rv(p1_[0], p1_[1], p1_[2], p1_[3]), p2 = rv(p2_[0], p2_[1], p2_[2], p2_[3]);
  rv4 p3 = rv(p3_[0], p3_[1], p3_[2], p3_[3]), p4 = rv(p4_[0], p4_[1], p4_[2], p4_[3]);
  ctx_t c = {P, sqrt(4.0 * M_PI * P->alpha_s), P->mt};
  qq_colour_matrix();
  rv4 K = rv_add(k1, k2);
  cv4 JK = cv_from_rv(K), JT = tpol(0);
  JT = cv_lin(sqrt(rv_dot(K, K)), JT, 0.0, JT);
  spin rq = d_bar(d_massless(k2, 0)), cq = d_massless(k1, 0);
  out[0] = out[1] = 0.0;
  for (int st = 0; st < 2; ++st)
    for (int stb = 0; stb < 2; ++stb)
      for (int sb = 0; sb < 2; ++sb)
        for (int sbb = 0; sbb < 2; ++sbb) {
          spin rt = d_bar(d_massive_u(p1, c.m, st)), ct = d_massive_v(p2, c.m, stb);
          spin rb = d_bar(d_massless(p3, sb)), cb = d_massless(p4, sbb);
          for (int w = 0; w < 2; ++w) {
            cplx L[NT_QQ];
            qq_lorentz_x(&c, k1, k2, p1, p2, p3, p4, rq, cq, rt, ct, rb, cb, L, w ? &JT : &JK);
            L[5] = L[6] = 0;
            out[w] += quad_form(0, L);
          }
        }
}

/* g g / q qbar -> t tbar b bbar -> (b l+ nu)(bbar mu- nubar) b bbar: the production
 * terms above between the decaying top row and antitop column of ora_msq_ttbar (the
 * W- decaying to mu- nubar), with Breit-Wigner t, tbar, W+, W- propagators; spins and
 * colours summed, the initial ones averaged. (p3, p4) = the extra b, bbar. */
double ora_msq_ttbb(const ora_process* P, int channel, const double* k1_, const double* k2_,
                    const double* pb_, const double* pl_, const double* pn_, const double* pbb_,
                    const double* pm_, const double* pnb_, const double* p3_, const double* p4_) {
  rv4 k1 = rv(k1_[0], k1_[1], k1_[2], k1_[3]), k2 = rv(k2_[0], k2_[1], k2_[2], k2_[3]);
  rv4 pb = rv(pb_[0], pb_[1], pb_[2], pb_[3]), pl = rv(pl_[0], pl_[1], pl_[2], pl_[3]);
  rv4 pn = rv(pn_[0], pn_[1], pn_[2], pn_[3]), pbb = rv(pbb_[0], pbb_[1], pbb_[2], pbb_[3]);
  rv4 pm = rv(pm_[0], pm_[1], pm_[2], pm_[3]), pnb = rv(pnb_[0], pnb_[1], pnb_[2], pnb_[3]);
  rv4 p3 = rv(p3_[0], p3_[1], p3_[2], p3_[3]), p4 = rv(p4_[0], p4_[1], p4_[2], p4_[3]);
  ctx_t c = {P, sqrt(4.0 * M_PI * P->alpha_s), P->mt};
  const double m = c.m;
  rv4 pt = rv_add(pb, rv_add(pl, pn)), ptb = rv_add(pbb, rv_add(pm, pnb));
  rv4 w1 = rv_add(pl, pn), w2 = rv_add(pm, pnb);
  cplx Dt = rv_dot(pt, pt) - m * m + I * m * P->wt;
  cplx Dtb = rv_dot(ptb, ptb) - m * m + I * m * P->wt;
  cplx Dw1 = rv_dot(w1, w1) - P->mw * P->mw + I * P->mw * P->ww;
  cplx Dw2 = rv_dot(w2, w2) - P->mw * P->mw + I * P->mw * P->ww;
  double gw2 = 4.0 * M_PI * P->alpha / P->sw2;
  dmat PL = d_PL();
  dmat ptm = d_add(d_slash_r(pt), d_scale(d_unit(), m));
  dmat ptbm = d_add(d_scale(d_slash_r(ptb), -1.0), d_scale(d_unit(), m));
  if (channel == 0) gg_colour_matrix();
  else qq_colour_matrix();
  double sum = 0.0;
  for (int sbt = 0; sbt < 2; ++sbt)
    for (int sn = 0; sn < 2; ++sn)
      for (int sl = 0; sl < 2; ++sl)
        for (int sbbt = 0; sbbt < 2; ++sbbt)
          for (int sm = 0; sm < 2; ++sm)
            for (int snb = 0; snb < 2; ++snb) {
              cv4 L = d_current(d_bar(d_massless(pn, sn)), PL, d_massless(pl, sl));
              cv4 H = d_current(d_bar(d_massless(pm, sm)), PL, d_massless(pnb, snb));
              spin rt = d_vm(d_vm(d_bar(d_massless(pb, sbt)), d_mul(d_slash(L), PL)), ptm);
              spin ct = d_mv(ptbm, d_mv(d_mul(d_slash(H), PL), d_massless(pbb, sbbt)));
              for (int sb = 0; sb < 2; ++sb)
                for (int sbb = 0; sbb < 2; ++sbb) {
                  spin rb = d_bar(d_massless(p3, sb)), cb = d_massless(p4, sbb);
                  if (channel == 0) {
                    for (int h1 = 0; h1 < 2; ++h1)
                      for (int h2 = 0; h2 < 2; ++h2) {
                        cplx Lt[NT_GG];
                        gg_lorentz(&c, k1, k2, pt, ptb, p3, p4, tpol(h1), tpol(h2), rt, ct, rb, cb,
                                   Lt);
                        sum += quad_form(1, Lt);
                      }
                  } else {
                    for (int sq = 0; sq < 2; ++sq)
                      for (int sqb = 0; sqb < 2; ++sqb) {
                        cplx Lt[NT_QQ];
                        spin rq = d_bar(d_massless(k2, sqb)), cq = d_massless(k1, sq);
                        qq_lorentz(&c, k1, k2, pt, ptb, p3, p4, rq, cq, rt, ct, rb, cb, Lt);
                        sum += quad_form(0, Lt);
                      }
                  }
                }
            }
  double dens = creal(Dt * conj(Dt)) * creal(Dtb * conj(Dtb)) * creal(Dw1 * conj(Dw1)) *
                creal(Dw2 * conj(Dw2));
  double coup = pow(0.5 * gw2, 4);   /* four W vertices; g_s is inside the terms */
  double avg = channel == 0 ? 1.0 / (4.0 * 64.0) : 1.0 / (4.0 * 9.0);
  return sum * coup * avg / dens;
}

/* The colour matrices (kgg 38 x 38, kqq 7 x 7; interleaved real, imaginary doubles). */
void ora_ttbb_colour_matrices(double* kgg, double* kqq) {
  gg_colour_matrix();
  qq_colour_matrix();
  for (int n = 0; n < NT_GG; ++n)
    for (int m = 0; m < NT_GG; ++m) {
      kgg[2 * (n * NT_GG + m)] = Kgg[n][m][0];
      kgg[2 * (n * NT_GG + m) + 1] = Kgg[n][m][1];
    }
  for (int n = 0; n < NT_QQ; ++n)
    for (int m = 0; m < NT_QQ; ++m) {
      kqq[2 * (n * NT_QQ + m)] = Kqq[n][m][0];
      kqq[2 * (n * NT_QQ + m) + 1] = Kqq[n][m][1];
    }
}

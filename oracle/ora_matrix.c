/* Tree-level |M|^2 for the oracle, from the Feynman rules written out with
 * explicit 4x4 Dirac matrices and sums over a complete spinor basis for every
 * external fermion (test infrastructure; see oracle.h).
 *
 * The paper obtains |M|^2 from HELAS-based code generated by MadGraph (Sec. 4);
 * here the same amplitudes are written by hand:
 *   Drell-Yan  q qbar -> (photon or Z) -> l- l+
 *   W          u dbar -> W+ -> e+ nu   (d ubar -> W- -> e- nubar)
 *   ttbar      g g / q qbar -> t tbar -> (b l+ nu)(bbar d ubar), resonant t, tbar,
 *              W+, W- propagators with Breit-Wigner widths, full spin correlation.
 *   ttH        g g / q qbar -> t tbar H (production, on-shell tops; Sec. 3's signal
 *              process), Higgs-top Yukawa y_t = m_t / v, v = 2 m_W / g_W.
 * Couplings: e^2 = 4 pi alpha, g_W^2 = e^2 / sin^2(theta_W), g_s^2 = 4 pi alpha_s.
 */
#include <math.h>

#include "oracle.h"
#include "ora_dirac.h"

static rv4 to_rv(const double* p) { return rv(p[0], p[1], p[2], p[3]); }

/* ------------------------------------------------------------ Drell-Yan */
double ora_msq_dy(const ora_process* P, int flavour, const double* kq_, const double* kqb_,
                  const double* plm_, const double* plp_) {
  rv4 kq = to_rv(kq_), kqb = to_rv(kqb_), plm = to_rv(plm_), plp = to_rv(plp_);
  double e2 = 4.0 * M_PI * P->alpha;
  double cw2 = 1.0 - P->sw2;
  double gz = sqrt(e2 / (P->sw2 * cw2));
  double Qq = flavour == 0 ? 2.0 / 3.0 : -1.0 / 3.0;
  double T3q = flavour == 0 ? 0.5 : -0.5;
  double Ql = -1.0, T3l = -0.5;
  double gq[2] = {gz * (T3q - Qq * P->sw2), gz * (-Qq * P->sw2)}; /* L, R */
  double gl[2] = {gz * (T3l - Ql * P->sw2), gz * (-Ql * P->sw2)};
  double shat = rv_dot(rv_add(kq, kqb), rv_add(kq, kqb));
  cplx Dz = shat - P->mz * P->mz + I * P->mz * P->wz;
  dmat Pc[2] = {d_PL(), d_PR()};
  double sum = 0.0;
  for (int sq = 0; sq < 2; ++sq)
    for (int sqb = 0; sqb < 2; ++sqb)
      for (int sl = 0; sl < 2; ++sl)
        for (int slb = 0; slb < 2; ++slb) {
          spin uq = d_massless(kq, sq);
          spin vbq = d_bar(d_massless(kqb, sqb));
          spin ubl = d_bar(d_massless(plm, sl));
          spin vl = d_massless(plp, slb);
          cplx M = 0;
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
              cv4 Jq = d_current(vbq, Pc[a], uq);
              cv4 Jl = d_current(ubl, Pc[b], vl);
              M += cv_dot(Jq, Jl) * (e2 * Qq * Ql / shat + gq[a] * gl[b] / Dz);
            }
          sum += creal(M * conj(M));
        }
  /* average over 4 initial spins; colour: sum 3 over the 9 averaged states */
  return sum / 4.0 / 3.0;
}

/* ------------------------------------------------------------ W */
double ora_msq_w(const ora_process* P, int charge, const double* kq_, const double* kqb_,
                 const double* pl_, const double* pn_) {
  rv4 kq = to_rv(kq_), kqb = to_rv(kqb_), pl = to_rv(pl_), pn = to_rv(pn_);
  double g2 = 4.0 * M_PI * P->alpha / P->sw2;
  double shat = rv_dot(rv_add(kq, kqb), rv_add(kq, kqb));
  cplx Dw = shat - P->mw * P->mw + I * P->mw * P->ww;
  dmat PL = d_PL();
  double sum = 0.0;
  for (int s1 = 0; s1 < 2; ++s1)
    for (int s2 = 0; s2 < 2; ++s2)
      for (int s3 = 0; s3 < 2; ++s3)
        for (int s4 = 0; s4 < 2; ++s4) {
          cv4 Jq = d_current(d_bar(d_massless(kqb, s2)), PL, d_massless(kq, s1));
          cv4 Jl;
          if (charge > 0) /* nu (particle) and e+ (antiparticle) */
            Jl = d_current(d_bar(d_massless(pn, s3)), PL, d_massless(pl, s4));
          else /* e- (particle) and nubar (antiparticle) */
            Jl = d_current(d_bar(d_massless(pl, s3)), PL, d_massless(pn, s4));
          cplx M = 0.5 * g2 * cv_dot(Jq, Jl) / Dw;
          sum += creal(M * conj(M));
        }
  return sum / 4.0 / 3.0;
}

/* ------------------------------------------------------------ ttbar */
/* Gluon polarisation vectors for a gluon moving along +z (dir = +1) or -z
 * (dir = -1): circular states (0, 1, +-i, 0)/sqrt(2) (for -z the helicity
 * labels flip, which does not matter for the summed |M|^2). They are
 * transverse to both beams, i.e. each gluon uses the other as gauge reference. */
static cv4 gluon_pol(int dir, int hel) {
  cv4 e;
  double r = 1.0 / sqrt(2.0);
  double sgn = (hel == 0 ? 1.0 : -1.0) * (dir > 0 ? 1.0 : -1.0);
  e.v[0] = 0;
  e.v[1] = r;
  e.v[2] = sgn * I * r;
  e.v[3] = 0;
  return e;
}

/* Colour-ordered production vertices between the top row spinor and the
 * antitop column spinor for g(k1, e1) g(k2, e2) -> t(pt) tbar:
 *   G1 = e1/ (pt/ - k1/ + m) e2/ / ((pt-k1)^2 - m^2) + V/ / s
 *   G2 = e2/ (pt/ - k2/ + m) e1/ / ((pt-k2)^2 - m^2) - V/ / s
 *   V  = (e1.e2)(k1 - k2) + 2 (k2.e1) e2 - 2 (k1.e2) e1     (three-gluon vertex)
 * multiplying colour factors (T^a T^b) and (T^b T^a). */
static void gg_vertices(rv4 k1, rv4 k2, rv4 pt, double m, cv4 e1, cv4 e2, dmat* G1, dmat* G2) {
  rv4 q1 = rv_sub(pt, k1), q2 = rv_sub(pt, k2);
  double d1 = rv_dot(q1, q1) - m * m, d2 = rv_dot(q2, q2) - m * m;
  double shat = rv_dot(rv_add(k1, k2), rv_add(k1, k2));
  dmat mm = d_scale(d_unit(), m);
  dmat A = d_mul(d_mul(d_slash(e1), d_add(d_slash_r(q1), mm)), d_slash(e2));
  dmat B = d_mul(d_mul(d_slash(e2), d_add(d_slash_r(q2), mm)), d_slash(e1));
  cv4 ck1 = cv_from_rv(k1), ck2 = cv_from_rv(k2);
  cv4 V = cv_lin(cv_dot(e1, e2), cv_lin(1.0, ck1, -1.0, ck2), 0.0, ck1);
  V = cv_lin(1.0, V, 2.0 * cv_dot(ck2, e1), e2);
  V = cv_lin(1.0, V, -2.0 * cv_dot(ck1, e2), e1);
  dmat S = d_scale(d_slash(V), 1.0 / shat);
  *G1 = d_add(d_scale(A, 1.0 / d1), S);
  *G2 = d_add(d_scale(B, 1.0 / d2), d_scale(S, -1.0));
}

/* Sum over gluon helicities of the colour-summed gg amplitude squared between
 * a row and a column spinor. Colour matrix for (T^aT^b, T^bT^a):
 * [[16/3, -2/3], [-2/3, 16/3]]. */
static double gg_colour_sum(rv4 k1, rv4 k2, rv4 pt, double m, spin row, spin col) {
  double s = 0.0;
  for (int h1 = 0; h1 < 2; ++h1)
    for (int h2 = 0; h2 < 2; ++h2) {
      dmat G1, G2;
      gg_vertices(k1, k2, pt, m, gluon_pol(+1, h1), gluon_pol(-1, h2), &G1, &G2);
      cplx A1 = d_rc(row, d_mv(G1, col));
      cplx A2 = d_rc(row, d_mv(G2, col));
      s += 16.0 / 3.0 * (creal(A1 * conj(A1)) + creal(A2 * conj(A2))) -
           2.0 * 2.0 / 3.0 * creal(A1 * conj(A2));
    }
  return s;
}

/* q(kq) qbar(kqb) -> g* -> t tbar: sum over light-quark spins of |row J/ col|^2 / s^2,
 * J^mu = vbar(kqb) gamma^mu u(kq); colour sum Tr(T^aT^b)Tr(T^aT^b) = 2. */
static double qq_colour_sum(rv4 kq, rv4 kqb, spin row, spin col) {
  double shat = rv_dot(rv_add(kq, kqb), rv_add(kq, kqb));
  double s = 0.0;
  dmat one = d_unit();
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      cv4 J = d_current(d_bar(d_massless(kqb, b)), one, d_massless(kq, a));
      cplx A = d_rc(row, d_mv(d_slash(J), col)) / shat;
      s += 2.0 * creal(A * conj(A));
    }
  return s;
}

double ora_msq_ttbar(const ora_process* P, int channel, const double* k1_, const double* k2_,
                     const double* pb_, const double* pl_, const double* pn_, const double* pbb_,
                     const double* pd_, const double* pu_) {
  rv4 k1 = to_rv(k1_), k2 = to_rv(k2_);
  rv4 pb = to_rv(pb_), pl = to_rv(pl_), pn = to_rv(pn_);
  rv4 pbb = to_rv(pbb_), pd = to_rv(pd_), pu = to_rv(pu_);
  double m = P->mt;
  rv4 pt = rv_add(pb, rv_add(pl, pn));
  rv4 ptb = rv_add(pbb, rv_add(pd, pu));
  rv4 w1 = rv_add(pl, pn), w2 = rv_add(pd, pu);
  cplx Dt = rv_dot(pt, pt) - m * m + I * m * P->wt;
  cplx Dtb = rv_dot(ptb, ptb) - m * m + I * m * P->wt;
  cplx Dw1 = rv_dot(w1, w1) - P->mw * P->mw + I * P->mw * P->ww;
  cplx Dw2 = rv_dot(w2, w2) - P->mw * P->mw + I * P->mw * P->ww;
  double gs2 = 4.0 * M_PI * P->alpha_s;
  double gw2 = 4.0 * M_PI * P->alpha / P->sw2;
  dmat PL = d_PL();
  dmat ptm = d_add(d_slash_r(pt), d_scale(d_unit(), m));                 /* pt/ + m */
  dmat ptbm = d_add(d_scale(d_slash_r(ptb), -1.0), d_scale(d_unit(), m)); /* -ptb/ + m */
  double sum = 0.0;
  for (int sb = 0; sb < 2; ++sb)
    for (int sn = 0; sn < 2; ++sn)
      for (int sl = 0; sl < 2; ++sl)
        for (int sbb = 0; sbb < 2; ++sbb)
          for (int sd = 0; sd < 2; ++sd)
            for (int su = 0; su < 2; ++su) {
              /* W+ -> nu l+ current, W- -> d ubar current (vertex g/sqrt2 gamma P_L) */
              cv4 L = d_current(d_bar(d_massless(pn, sn)), PL, d_massless(pl, sl));
              cv4 H = d_current(d_bar(d_massless(pd, sd)), PL, d_massless(pu, su));
              /* top row: ubar(b) L/ P_L (pt/ + m); antitop column: (-ptb/ + m) H/ P_L v(bbar) */
              spin row = d_vm(d_vm(d_bar(d_massless(pb, sb)), d_mul(d_slash(L), PL)), ptm);
              spin col = d_mv(ptbm, d_mv(d_mul(d_slash(H), PL), d_massless(pbb, sbb)));
              if (channel == 0)
                sum += gg_colour_sum(k1, k2, pt, m, row, col);
              else
                sum += qq_colour_sum(k1, k2, row, col);
            }
  double dens = creal(Dt * conj(Dt)) * creal(Dtb * conj(Dtb)) * creal(Dw1 * conj(Dw1)) *
                creal(Dw2 * conj(Dw2));
  /* couplings: g_s^4 (production) x (g_W/sqrt2)^8 (four W vertices);
   * W- -> q qbar': colour 3, two light generations (d ubar, s cbar) */
  double coup = gs2 * gs2 * pow(0.5 * gw2, 4) * 3.0 * 2.0;
  double avg = channel == 0 ? 1.0 / (4.0 * 64.0) : 1.0 / (4.0 * 9.0);
  return sum * coup * avg / dens;
}

double ora_msq_ttbar_production(const ora_process* P, int channel, const double* k1_,
                                const double* k2_, const double* pt_, const double* ptb_) {
  rv4 k1 = to_rv(k1_), k2 = to_rv(k2_), pt = to_rv(pt_), ptb = to_rv(ptb_);
  double m = P->mt;
  double gs2 = 4.0 * M_PI * P->alpha_s;
  double sum = 0.0;
  for (int s = 0; s < 2; ++s)
    for (int sb = 0; sb < 2; ++sb) {
      spin row = d_bar(d_massive_u(pt, m, s));
      spin col = d_massive_v(ptb, m, sb);
      sum += channel == 0 ? gg_colour_sum(k1, k2, pt, m, row, col)
                          : qq_colour_sum(k1, k2, row, col);
    }
  double avg = channel == 0 ? 1.0 / (4.0 * 64.0) : 1.0 / (4.0 * 9.0);
  return sum * gs2 * gs2 * avg;
}

double ora_ttbar_gauge_probe(const ora_process* P, const double* k1_, const double* k2_,
                             const double* pt_, const double* ptb_, int which, int hel) {
  rv4 k1 = to_rv(k1_), k2 = to_rv(k2_), pt = to_rv(pt_), ptb = to_rv(ptb_);
  double m = P->mt;
  double tot = 0.0;
  for (int s = 0; s < 2; ++s)
    for (int sb = 0; sb < 2; ++sb) {
      spin row = d_bar(d_massive_u(pt, m, s));
      spin col = d_massive_v(ptb, m, sb);
      cv4 e1 = gluon_pol(+1, hel), e2 = gluon_pol(-1, hel);
      if (which == 0) e1 = cv_from_rv(k1);
      else e2 = cv_from_rv(k2);
      dmat G1, G2;
      gg_vertices(k1, k2, pt, m, e1, e2, &G1, &G2);
      cplx A1 = d_rc(row, d_mv(G1, col)), A2 = d_rc(row, d_mv(G2, col));
      tot += creal(A1 * conj(A1)) + creal(A2 * conj(A2));
    }
  return tot;
}

void ora_top_decay_probe(const ora_process* P, const double* pb_, const double* pl_,
                         const double* pn_, double* out2) {
  rv4 pb = to_rv(pb_), pl = to_rv(pl_), pn = to_rv(pn_);
  double m = P->mt;
  rv4 pt = rv(m, 0, 0, 0);
  dmat PL = d_PL();
  dmat ptm = d_add(d_slash_r(pt), d_scale(d_unit(), m));
  for (int s = 0; s < 2; ++s) {
    double acc = 0.0;
    spin ut = d_massive_u(pt, m, s);
    for (int sb = 0; sb < 2; ++sb)
      for (int sn = 0; sn < 2; ++sn)
        for (int sl = 0; sl < 2; ++sl) {
          cv4 L = d_current(d_bar(d_massless(pn, sn)), PL, d_massless(pl, sl));
          spin row = d_vm(d_vm(d_bar(d_massless(pb, sb)), d_mul(d_slash(L), PL)), ptm);
          cplx a = d_rc(row, ut);
          acc += creal(a * conj(a));
        }
    out2[s] = acc;
  }
}

void ora_antitop_decay_probe(const ora_process* P, const double* pbb_, const double* pd_,
                             const double* pu_, double* out2) {
  rv4 pbb = to_rv(pbb_), pd = to_rv(pd_), pu = to_rv(pu_);
  double m = P->mt;
  rv4 ptb = rv(m, 0, 0, 0);
  dmat PL = d_PL();
  dmat ptbm = d_add(d_scale(d_slash_r(ptb), -1.0), d_scale(d_unit(), m));
  for (int s = 0; s < 2; ++s) {
    double acc = 0.0;
    spin vbt = d_bar(d_massive_v(ptb, m, s));
    for (int sbb = 0; sbb < 2; ++sbb)
      for (int sd = 0; sd < 2; ++sd)
        for (int su = 0; su < 2; ++su) {
          cv4 H = d_current(d_bar(d_massless(pd, sd)), PL, d_massless(pu, su));
          spin col = d_mv(ptbm, d_mv(d_mul(d_slash(H), PL), d_massless(pbb, sbb)));
          cplx a = d_rc(vbt, col);
          acc += creal(a * conj(a));
        }
    out2[s] = acc;
  }
}

/* ------------------------------------------------------------ ttH */
/* Fermion propagator (q/ + m) / (q^2 - m^2). */
static dmat fprop(rv4 q, double m) {
  return d_scale(d_add(d_slash_r(q), d_scale(d_unit(), m)), 1.0 / (rv_dot(q, q) - m * m));
}

/* X1 S(q1) X2 S(q2) X3 along the top line read from the top (row) side: each
 * vertex takes in the momentum in_j, so q1 = pt - in1 and q2 = q1 - in2. */
static dmat chain3(dmat X1, rv4 in1, dmat X2, rv4 in2, dmat X3, rv4 pt, double m) {
  rv4 q1 = rv_sub(pt, in1), q2 = rv_sub(q1, in2);
  return d_mul(d_mul(d_mul(d_mul(X1, fprop(q1, m)), X2), fprop(q2, m)), X3);
}
static dmat chain2(dmat X1, rv4 in1, dmat X2, rv4 pt, double m) {
  return d_mul(d_mul(X1, fprop(rv_sub(pt, in1), m)), X2);
}

/* Colour-ordered vertices of g(k1, e1) g(k2, e2) -> t(pt) tbar H(pH) between the top
 * row and the antitop column, Yukawa and g_s factors left out: the two gluons and
 * the Higgs (unit scalar vertex, momentum -pH entering) in every order on the top
 * line, and the s-channel gluon V/ / s with the Higgs before or after it.
 *   G1 = orders with e1 before e2 (from the top side) + S_H    (colour T^a T^b)
 *   G2 = orders with e2 before e1                    - S_H    (colour T^b T^a) */
static void tth_gg_vertices(rv4 k1, rv4 k2, rv4 pt, rv4 pH, double m, cv4 e1, cv4 e2, dmat* G1,
                            dmat* G2) {
  dmat E1 = d_slash(e1), E2 = d_slash(e2), H = d_unit();
  rv4 mh = rv_scale(pH, -1.0), K = rv_add(k1, k2);
  *G1 = d_add(d_add(chain3(E1, k1, E2, k2, H, pt, m), chain3(E1, k1, H, mh, E2, pt, m)),
              chain3(H, mh, E1, k1, E2, pt, m));
  *G2 = d_add(d_add(chain3(E2, k2, E1, k1, H, pt, m), chain3(E2, k2, H, mh, E1, pt, m)),
              chain3(H, mh, E2, k2, E1, pt, m));
  double shat = rv_dot(K, K);
  cv4 ck1 = cv_from_rv(k1), ck2 = cv_from_rv(k2);
  cv4 V = cv_lin(cv_dot(e1, e2), cv_lin(1.0, ck1, -1.0, ck2), 0.0, ck1);
  V = cv_lin(1.0, V, 2.0 * cv_dot(ck2, e1), e2);
  V = cv_lin(1.0, V, -2.0 * cv_dot(ck1, e2), e1);
  dmat VS = d_scale(d_slash(V), 1.0 / shat);
  dmat SH = d_add(chain2(VS, K, H, pt, m), chain2(H, mh, VS, pt, m));
  *G1 = d_add(*G1, SH);
  *G2 = d_add(*G2, d_scale(SH, -1.0));
}

static double tth_gg_colour_sum(rv4 k1, rv4 k2, rv4 pt, rv4 pH, double m, spin row, spin col) {
  double s = 0.0;
  for (int h1 = 0; h1 < 2; ++h1)
    for (int h2 = 0; h2 < 2; ++h2) {
      dmat G1, G2;
      tth_gg_vertices(k1, k2, pt, pH, m, gluon_pol(+1, h1), gluon_pol(-1, h2), &G1, &G2);
      cplx A1 = d_rc(row, d_mv(G1, col));
      cplx A2 = d_rc(row, d_mv(G2, col));
      s += 16.0 / 3.0 * (creal(A1 * conj(A1)) + creal(A2 * conj(A2))) -
           2.0 * 2.0 / 3.0 * creal(A1 * conj(A2));
    }
  return s;
}

/* q(kq) qbar(kqb) -> g* -> t tbar H: the Higgs before or after the gluon vertex on
 * the top line (the massless light quarks do not couple to it); colour sum 2. */
static double tth_qq_colour_sum(rv4 kq, rv4 kqb, rv4 pt, rv4 pH, double m, spin row, spin col) {
  rv4 K = rv_add(kq, kqb), mh = rv_scale(pH, -1.0);
  double shat = rv_dot(K, K);
  double s = 0.0;
  dmat one = d_unit();
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      cv4 J = d_current(d_bar(d_massless(kqb, b)), one, d_massless(kq, a));
      dmat JS = d_slash(J);
      dmat G = d_add(chain2(JS, K, one, pt, m), chain2(one, mh, JS, pt, m));
      cplx A = d_rc(row, d_mv(G, col)) / shat;
      s += 2.0 * creal(A * conj(A));
    }
  return s;
}

static double yukawa_top(const ora_process* P) {
  double gw2 = 4.0 * M_PI * P->alpha / P->sw2;
  double v = 2.0 * P->mw / sqrt(gw2);
  return P->mt / v;
}

double ora_msq_tth_production(const ora_process* P, int channel, const double* k1_,
                              const double* k2_, const double* pt_, const double* ptb_,
                              const double* pH_) {
  rv4 k1 = to_rv(k1_), k2 = to_rv(k2_), pt = to_rv(pt_), ptb = to_rv(ptb_), pH = to_rv(pH_);
  double m = P->mt;
  double gs2 = 4.0 * M_PI * P->alpha_s;
  double y = yukawa_top(P);
  double sum = 0.0;
  for (int s = 0; s < 2; ++s)
    for (int sb = 0; sb < 2; ++sb) {
      spin row = d_bar(d_massive_u(pt, m, s));
      spin col = d_massive_v(ptb, m, sb);
      sum += channel == 0 ? tth_gg_colour_sum(k1, k2, pt, pH, m, row, col)
                          : tth_qq_colour_sum(k1, k2, pt, pH, m, row, col);
    }
  double avg = channel == 0 ? 1.0 / (4.0 * 64.0) : 1.0 / (4.0 * 9.0);
  return sum * gs2 * gs2 * y * y * avg;
}

/* Gauge probe of the colour-ordered ttH amplitudes: sum over top spins of
 * |A(T^aT^b)|^2 + |A(T^bT^a)|^2 with gluon `which` (0 or 1) given its momentum as
 * polarisation and the other gluon the transverse state hel. */
double ora_tth_gauge_probe(const ora_process* P, const double* k1_, const double* k2_,
                           const double* pt_, const double* ptb_, const double* pH_, int which,
                           int hel) {
  rv4 k1 = to_rv(k1_), k2 = to_rv(k2_), pt = to_rv(pt_), ptb = to_rv(ptb_), pH = to_rv(pH_);
  double m = P->mt;
  double tot = 0.0;
  for (int s = 0; s < 2; ++s)
    for (int sb = 0; sb < 2; ++sb) {
      spin row = d_bar(d_massive_u(pt, m, s));
      spin col = d_massive_v(ptb, m, sb);
      cv4 e1 = gluon_pol(+1, hel), e2 = gluon_pol(-1, hel);
      if (which == 0) e1 = cv_from_rv(k1);
      else e2 = cv_from_rv(k2);
      dmat G1, G2;
      tth_gg_vertices(k1, k2, pt, pH, m, e1, e2, &G1, &G2);
      cplx A1 = d_rc(row, d_mv(G1, col)), A2 = d_rc(row, d_mv(G2, col));
      tot += creal(A1 * conj(A1)) + creal(A2 * conj(A2));
    }
  return tot;
}

/* g g / q qbar -> t tbar H -> (b l+ nu)(bbar mu- nubar)(b1 b2): the production
 * vertices above between the decaying top row and antitop column of ora_msq_ttbar
 * (here with the W- decaying to mu- nubar), times the Higgs decay
 * y_b ubar(b1) v(b2) (colour singlet: 3 colour states) and the Higgs propagator
 * 1 / (q_H^2 - m_H^2 + i m_H G_H), y_b = m_b / v; resonant t, tbar, W+, W-
 * Breit-Wigner propagators as in ora_msq_ttbar. Colour and spins summed, the
 * initial ones averaged. */
double ora_msq_tth(const ora_process* P, int channel, const double* k1_, const double* k2_,
                   const double* pb_, const double* pl_, const double* pn_, const double* pbb_,
                   const double* pm_, const double* pnb_, const double* ph1_, const double* ph2_) {
  rv4 k1 = to_rv(k1_), k2 = to_rv(k2_);
  rv4 pb = to_rv(pb_), pl = to_rv(pl_), pn = to_rv(pn_);
  rv4 pbb = to_rv(pbb_), pm = to_rv(pm_), pnb = to_rv(pnb_);
  rv4 ph1 = to_rv(ph1_), ph2 = to_rv(ph2_);
  double m = P->mt;
  rv4 pt = rv_add(pb, rv_add(pl, pn));
  rv4 ptb = rv_add(pbb, rv_add(pm, pnb));
  rv4 pH = rv_add(ph1, ph2);
  rv4 w1 = rv_add(pl, pn), w2 = rv_add(pm, pnb);
  cplx Dt = rv_dot(pt, pt) - m * m + I * m * P->wt;
  cplx Dtb = rv_dot(ptb, ptb) - m * m + I * m * P->wt;
  cplx Dw1 = rv_dot(w1, w1) - P->mw * P->mw + I * P->mw * P->ww;
  cplx Dw2 = rv_dot(w2, w2) - P->mw * P->mw + I * P->mw * P->ww;
  cplx Dh = rv_dot(pH, pH) - P->mh * P->mh + I * P->mh * P->wh;
  double gs2 = 4.0 * M_PI * P->alpha_s;
  double gw2 = 4.0 * M_PI * P->alpha / P->sw2;
  double yt = yukawa_top(P), yb = yt * P->mb / P->mt;
  dmat PL = d_PL();
  dmat ptm = d_add(d_slash_r(pt), d_scale(d_unit(), m));
  dmat ptbm = d_add(d_scale(d_slash_r(ptb), -1.0), d_scale(d_unit(), m));
  double sum = 0.0;
  for (int sb = 0; sb < 2; ++sb)
    for (int sn = 0; sn < 2; ++sn)
      for (int sl = 0; sl < 2; ++sl)
        for (int sbb = 0; sbb < 2; ++sbb)
          for (int sm = 0; sm < 2; ++sm)
            for (int snb = 0; snb < 2; ++snb) {
              cv4 L = d_current(d_bar(d_massless(pn, sn)), PL, d_massless(pl, sl));
              cv4 H = d_current(d_bar(d_massless(pm, sm)), PL, d_massless(pnb, snb));
              spin row = d_vm(d_vm(d_bar(d_massless(pb, sb)), d_mul(d_slash(L), PL)), ptm);
              spin col = d_mv(ptbm, d_mv(d_mul(d_slash(H), PL), d_massless(pbb, sbb)));
              sum += channel == 0 ? tth_gg_colour_sum(k1, k2, pt, pH, m, row, col)
                                  : tth_qq_colour_sum(k1, k2, pt, pH, m, row, col);
            }
  /* Higgs decay: sum over the b1, b2 spins of |ubar(b1) v(b2)|^2 */
  double hdec = 0.0;
  for (int s1 = 0; s1 < 2; ++s1)
    for (int s2 = 0; s2 < 2; ++s2) {
      cplx a = d_rc(d_bar(d_massless(ph1, s1)), d_massless(ph2, s2));
      hdec += creal(a * conj(a));
    }
  double dens = creal(Dt * conj(Dt)) * creal(Dtb * conj(Dtb)) * creal(Dw1 * conj(Dw1)) *
                creal(Dw2 * conj(Dw2)) * creal(Dh * conj(Dh));
  double coup = gs2 * gs2 * yt * yt * pow(0.5 * gw2, 4) * yb * yb * 3.0;
  double avg = channel == 0 ? 1.0 / (4.0 * 64.0) : 1.0 / (4.0 * 9.0);
  return sum * hdec * coup * avg / dens;
}

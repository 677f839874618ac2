// Dilepton ttH integrand (Sec. 3-4: the signal of the paper's hadron-level
// analysis, Eq. "integrand" with Eq. "mhsolve"), g g / q qbar -> t tbar H ->
// (b l+ nu)(bbar mu- nubar)(b bbar).
//
// Variables (8): those of dilepton ttbar (mem_ttdl.cuh: E_b, E_bbar, q^2 of W+, W-,
// t, tbar) and the Higgs pair's m_H^2 = 2 E1 E2 (1 - cos theta_12) (Breit-Wigner map
// over [2 (1 - cos) lo1 lo2, 2 (1 - cos) hi1 hi2], the values the two jet windows
// allow) and f = E1 + E2 over its image at that K = E1 E2: the larger energy runs over
// [A, B] = [max(lo1, K/hi2), min(hi1, K/lo2)], f = E + K/E over [f_min, f_max], mapped
// as f_min + (f_max - f_min) v^2 so that the 1 / sqrt(f^2 - 4K) of the inverse map is
// cancelled. E1,2 = (f +- sqrt(f^2 - 4K)) / 2 in both orderings, each with
// 1 / (2 (1 - cos theta_12) sqrt(f^2 - 4K)); at least one ordering lies inside both
// windows by construction, one that leaves a window has no weight. The
// missing pT is the visible imbalance including the Higgs pair, and the neutrinos
// follow from Eq. "dilepsolv" with the double-float solver of mem_dlsolve.cuh. 12 jet
// assignments: the (perm / 3)-th jet is the b, the (perm % 3)-th of the other three
// the bbar, the remaining two (in object order) the Higgs pair.
//
// |M|^2: the Fierz-collapsed top row and antitop column of mem_ttbar.cuh (mu- in
// the d slot, nubar in the ubar slot) around the ttH production vertices: the two
// gluons and the Higgs (unit scalar vertex) in every order on the top line and the
// s-channel gluon with the Higgs before or after it, in the two colour orderings;
// q qbar -> g* -> t tbar H with the Higgs before or after the gluon vertex. Every top
// propagator denominator is written as a sum of same-sign terms in light-cone
// components (k1 carries only p+, k2 only p-). The Higgs decay gives
// 3 y_b^2 4 p_b1.p_b2 = 3 y_b^2 2 m_H^2; its propagator cancels against the m_H^2
// map's Jacobian like the t and W ones.
#pragma once
#include "mem_ttdl.cuh"

namespace mem {

struct THCache {
  float b_lo, Lb, bb_lo, Lbb;                   // b, bbar jet windows: lo, ln(hi / lo)
  float h1_lo, h1_hi, h2_lo, h2_hi;             // Higgs-pair jet windows
  float m_lo, m_rng, psi_h, Lm;                 // pair m^2 window [m_lo, m_lo + m_rng], atan2(m G, hi - m^2),
                                                // ln(hi / lo)
  float bnx, bny, bnz, blcp, blcm;
  float bbnx, bbny, bbnz, bblcp, bblcm;
  float h1nx, h1ny, h1nz, h1lcp, h1lcm;
  float h2nx, h2ny, h2nz, h2lcp, h2lcm;
  float Ebm, Ebbm, E1m, E2m;                    // measured jet energies
  float Elp, lpnx, lpny, lpnz, lplcp, lplcm;    // l+
  float Elm, lmnx, lmny, lmnz, lmlcp, lmlcm;    // mu-
  float omc_bl, omc_bbl, omc_h;                 // 1 - cos of (b, l+), (bbar, mu-), (b1, b2)
  float psi_w, psi_t;
  float core_w, tail_w, inv_core, inv_tail;
  float cst;
  int ok;
};

// The pair's m^2 = 2 E1 E2 (1 - cos theta_12) window: the values the two jet windows
// allow (FP64 set-up, once per item).
__device__ inline void th_pair_window(THCache& c, const ProcConst& P, double lo1, double hi1,
                                      double lo2, double hi2, double omc) {
  const double mlo = 2.0 * omc * lo1 * lo2, mhi = 2.0 * omc * hi1 * hi2;
  c.m_lo = (float)mlo;
  c.m_rng = (float)(mhi - mlo);
  c.psi_h = (float)atan2((double)P.mhgh, mhi - (double)P.mh2);
  c.Lm = (float)log(mhi / mlo);
}

// Eq. "mhsolve" at a point: with K = E1 E2 = m^2 / (2 (1 - cos)) fixed, E1 runs over
// [A, B] = [max(lo1, K / hi2), min(hi1, K / lo2)] and f = E1 + K / E1 over its image
// [f_min, f_max] (f_min = 2 sqrt(K) when sqrt(K) is inside); f = f_min + (f_max - f_min) v^2,
// whose square cancels the 1/sqrt(f - 2 sqrt(K)) end point of 1 / |d(f, m^2)/d(E1, E2)|.
// Everything is written as distances from 2 sqrt(K) (no cancellation). Returns false
// when the windows leave no room; else the larger and smaller energies and the
// Jacobian (d f / d v) / (2 (1 - cos) |E1 - E2|).
__device__ __forceinline__ bool th_pair(const THCache& c, float m2, float v, float& e_big,
                                        float& e_small, float& jac) {
  const float K = m2 * (0.5f / c.omc_h);
  const float A = fmaxf(c.h1_lo, K / c.h2_hi), B = fminf(c.h1_hi, K / c.h2_lo);
  if (!(A < B)) return false;
  const float r = sqrtf(K);
  const float dA = (A - r) * (A - r) / A, dB = (B - r) * (B - r) / B;   // f(A) - 2r, f(B) - 2r
  const float dmn = (A <= r && r <= B) ? 0.f : fminf(dA, dB);
  const float span = fmaxf(dA, dB) - dmn;
  const float d = fmaf(span, v * v, dmn);                                // f - 2r
  const float f = fmaf(2.f, r, d);
  const float sq = sqrtf(d * (f + 2.f * r));                             // sqrt(f^2 - 4K)
  if (!(sq > 0.f)) return false;
  e_big = 0.5f * (f + sq);
  e_small = K / e_big;
  jac = 2.f * v * span / (2.f * c.omc_h * sq);
  return true;
}

__device__ __forceinline__ Sp sp_scale(float s, const Sp& a) {
  return {s * a.l1, s * a.l2, s * a.r1, s * a.r2};
}
// row x (q/ + m) / den
__device__ __forceinline__ Sp row_prop(const Sp& r, const LCv& q, float m, float den) {
  return sp_scale(1.f / den, row_slash_m(r, q, m));
}
__device__ __forceinline__ Sp row_e(const Sp& r, int pol) { return pol ? row_ey(r) : row_ex(r); }
__device__ __forceinline__ LCv lc(float pp, float pm, cf pt) {
  LCv o;
  o.pp = pp;
  o.pm = pm;
  o.pt = pt;
  return o;
}

// Helicity-summed squared production amplitudes of g g -> t tbar H (gg, with its
// colour matrix) and q qbar -> g* -> t tbar H (qq) between the Fierz-collapsed top
// row and antitop column built from l+ (l), mu- (d), the top (tp), antitop (tm) and
// Higgs (h) light-cone momenta; k1p = x1 sqrt(s), k2m = x2 sqrt(s), shat = k1p k2m.
// Couplings, averages and the decay factors are applied by the caller.
static __device__ __noinline__ TTAmp2 tth_amp2(const LCv& l, const LCv& d, const LCv& tp, const LCv& tm,
                                        const LCv& h, float m, float m2, float k1p, float k2m,
                                        float shat) {
  cf la, lb, da, db;
  weyl(l, la, lb);
  weyl(d, da, db);
  const cf w1 = lb, w2 = -la;
  const cf z1 = conjf(db), z2 = -conjf(da);
  Sp U;
  U.l1 = m * w1;
  U.l2 = m * w2;
  U.r1 = tp.pm * w1 - w2 * tp.pt;
  U.r2 = tp.pp * w2 - w1 * conjf(tp.pt);
  Sp Y;
  Y.l1 = conjf(tm.pt) * z2 - tm.pm * z1;
  Y.l2 = tm.pt * z1 - tm.pp * z2;
  Y.r1 = m * z1;
  Y.r2 = m * z2;
  // top-line momenta between the vertices (see the header) and their denominators
  const cf tpt = tp.pt, tht = tp.pt + h.pt, mht = -(tm.pt + h.pt);
  const float a_pp = tm.pp + h.pp, b_pm = tm.pm + h.pm;
  const LCv A = lc(-a_pp, tp.pm, tpt);                      // p_t - k1
  const float dA = -(fmaf(a_pp, tp.pm, norm2(tpt)) + m2);
  const LCv B = lc(tp.pp, -b_pm, tpt);                      // p_t - k2
  const float dB = -(fmaf(tp.pp, b_pm, norm2(tpt)) + m2);
  const LCv Cq = lc(tp.pp + h.pp, tp.pm + h.pm, tht);       // p_t + p_H
  const float dC = fmaf(Cq.pp, Cq.pm, -norm2(tht)) - m2;
  const LCv D = lc(-a_pp, -b_pm, mht);                      // p_t - k1 - k2 = -(p_tbar + p_H)
  const float dD = fmaf(a_pp, b_pm, -norm2(mht)) - m2;
  const LCv E = lc(-tm.pp, tp.pm + h.pm, tht);              // p_t - k1 + p_H
  const float dE = -(fmaf(tm.pp, tp.pm + h.pm, norm2(tht)) + m2);
  const LCv F = lc(tp.pp + h.pp, -tm.pm, tht);              // p_t - k2 + p_H
  const float dF = -(fmaf(tp.pp + h.pp, tm.pm, norm2(tht)) + m2);
  const Sp UC = row_prop(U, Cq, m, dC);                     // Higgs first
  // s-channel gluon with the Higgs after or before it: (e1.e2)(k1 - k2)/ / s, e1.e2 = -delta
  const LCv kk = lc(k1p, -k2m, C(0.f));
  const cf sq = (-1.f / shat) * (dot4(row_prop(row_slash_m(U, kk, 0.f), D, m, dD), Y) +
                                 dot4(row_slash_m(UC, kk, 0.f), Y));
  float gg = 0.f;
#pragma unroll 1
  for (int ab = 0; ab < 4; ++ab) {
    const int ia = ab >> 1, ib = ab & 1;
    const Sp U1 = row_prop(row_e(U, ia), A, m, dA);         // e1 first
    const Sp U2 = row_prop(row_e(U, ib), B, m, dB);         // e2 first
    cf A1 = dot4(row_prop(row_e(U1, ib), D, m, dD), Y) +                   // e1 e2 H
            dot4(row_e(row_prop(U1, E, m, dE), ib), Y) +                   // e1 H e2
            dot4(row_e(row_prop(row_e(UC, ia), E, m, dE), ib), Y);         // H e1 e2
    cf A2 = dot4(row_prop(row_e(U2, ia), D, m, dD), Y) +                   // e2 e1 H
            dot4(row_e(row_prop(U2, F, m, dF), ia), Y) +                   // e2 H e1
            dot4(row_e(row_prop(row_e(UC, ib), F, m, dF), ia), Y);         // H e2 e1
    if (ia == ib) {
      A1 = A1 + sq;
      A2 = A2 - sq;
    }
    gg += (16.f / 3.f) * (norm2(A1) + norm2(A2)) - (4.f / 3.f) * fmaf(A1.re, A2.re, A1.im * A2.im);
  }
  float qq = 0.f;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const cf T = dot4(row_prop(row_e(U, i), D, m, dD), Y) + dot4(row_e(UC, i), Y);
    qq += norm2(T);
  }
  TTAmp2 r;
  r.gg = gg;
  r.qq = (4.f / shat) * qq;
  return r;
}

template <int PDFM>
struct PhysTTH_ {
  static constexpr int D = 8;
  static constexpr int NPERM = 12;
  using Cache = THCache;

  __device__ static void setup(const float* rec, int perm, const ProcConst& P, const TFConst& T,
                               Cache& c) {
    const int ib = perm / 3;
    int rest[3], n = 0;
    for (int j = 0; j < 4; ++j)
      if (j != ib) rest[n++] = j;
    const int ibb = rest[perm % 3];
    int hh[2], k = 0;
    for (int j = 0; j < 3; ++j)
      if (j != perm % 3) hh[k++] = rest[j];
    const int objs[6] = {2 + ib, 2 + ibb, 2 + hh[0], 2 + hh[1], 0, 1};
    c.ok = perm >= 0 && perm < 12 && rec[3] == 4.f && rec[7] == 1.f && rec[0] > 0.f &&
           rec[4] > 0.f && T.jet_core > 0.f && T.jet_tail > 0.f && P.mhgh > 0.f;
    for (int j = 2; j < 6; ++j) c.ok = c.ok && rec[4 * j + 3] == 5.f && rec[4 * j] > 0.f;
    double nv[6][3], sn[6], lcv[6][2];
    for (int q = 0; q < 6; ++q) {
      const int o = objs[q];
      const double eta = rec[4 * o + 1], phi = rec[4 * o + 2], ch = cosh(eta);
      nv[q][0] = cos(phi) / ch;
      nv[q][1] = sin(phi) / ch;
      nv[q][2] = tanh(eta);
      sn[q] = 1.0 / ch;
      lcv[q][0] = exp(eta) / ch;
      lcv[q][1] = exp(-eta) / ch;
    }
    const double smax = 0.5 * (double)P.sqrt_s;
    double lo[4], hi[4];
    for (int q = 0; q < 4; ++q) {
      const double E = rec[4 * objs[q]];
      lo[q] = E / (double)T.jet_lo_div;
      hi[q] = E * (double)T.jet_hi_mul;
      hi[q] = hi[q] < smax ? hi[q] : smax;
      c.ok = c.ok && hi[q] > lo[q];
    }
    const double Lb = c.ok ? log(hi[0] / lo[0]) : 0.0, Lbb = c.ok ? log(hi[1] / lo[1]) : 0.0;
    c.b_lo = (float)lo[0];
    c.Lb = (float)Lb;
    c.bb_lo = (float)lo[1];
    c.Lbb = (float)Lbb;
    c.h1_lo = (float)lo[2];
    c.h1_hi = (float)hi[2];
    c.h2_lo = (float)lo[3];
    c.h2_hi = (float)hi[3];
    float* dirs[4][5] = {{&c.bnx, &c.bny, &c.bnz, &c.blcp, &c.blcm},
                         {&c.bbnx, &c.bbny, &c.bbnz, &c.bblcp, &c.bblcm},
                         {&c.h1nx, &c.h1ny, &c.h1nz, &c.h1lcp, &c.h1lcm},
                         {&c.h2nx, &c.h2ny, &c.h2nz, &c.h2lcp, &c.h2lcm}};
    for (int q = 0; q < 4; ++q) {
      *dirs[q][0] = (float)nv[q][0];
      *dirs[q][1] = (float)nv[q][1];
      *dirs[q][2] = (float)nv[q][2];
      *dirs[q][3] = (float)lcv[q][0];
      *dirs[q][4] = (float)lcv[q][1];
    }
    c.Ebm = rec[4 * objs[0]];
    c.Ebbm = rec[4 * objs[1]];
    c.E1m = rec[4 * objs[2]];
    c.E2m = rec[4 * objs[3]];
    c.Elp = rec[0];
    c.lpnx = (float)nv[4][0];
    c.lpny = (float)nv[4][1];
    c.lpnz = (float)nv[4][2];
    c.lplcp = (float)lcv[4][0];
    c.lplcm = (float)lcv[4][1];
    c.Elm = rec[4];
    c.lmnx = (float)nv[5][0];
    c.lmny = (float)nv[5][1];
    c.lmnz = (float)nv[5][2];
    c.lmlcp = (float)lcv[5][0];
    c.lmlcm = (float)lcv[5][1];
    auto omc = [](const double* a, const double* b) {   // 1 - a.b = |a - b|^2 / 2
      const double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
      return 0.5 * (dx * dx + dy * dy + dz * dz);
    };
    c.omc_bl = (float)omc(nv[0], nv[4]);
    c.omc_bbl = (float)omc(nv[1], nv[5]);
    c.omc_h = (float)omc(nv[2], nv[3]);
    c.ok = c.ok && c.omc_h > 0.f;
    th_pair_window(c, P, lo[2], hi[2], lo[3], hi[3], omc(nv[2], nv[3]));
    c.psi_w = (float)atan2((double)P.mwgw, (double)P.s - (double)P.mw2);
    c.psi_t = (float)atan2((double)P.mtgt, (double)P.s - (double)P.mt2);
    const double tw = T.jet_tail_w;
    c.core_w = (float)((1.0 - tw) / T.jet_core);
    c.tail_w = (float)(tw / T.jet_tail);
    c.inv_core = (float)(1.0 / T.jet_core);
    c.inv_tail = (float)(1.0 / T.jet_tail);
    // b, bbar: E sin(theta) L / sqrt(2 pi) per jet with E per point; Higgs-pair jets:
    // sin(theta) / sqrt(2 pi) (their measure E^2 sin(theta), phase space 1/E and TF 1/E;
    // the f and m_H^2 Jacobians are per point); leptons 1/E each; R / (m G) per
    // Breit-Wigner map (W+, W-, t, tbar, H); P.tth_c: y_t^2 x 3 y_b^2 / 6 (the W- decays
    // to one lepton channel where the semileptonic couplings count 6); x TTH_WEIGHT_SCALE.
    const double mgw = (double)P.mwgw, mgt = (double)P.mtgt, mgh = (double)P.mhgh;
    c.cst = (float)(sn[0] * sn[1] * sn[2] * sn[3] * Lb * Lbb / (4.0 * PI_D * PI_D) /
                    ((double)rec[0] * (double)rec[4]) / (mgw * mgw * mgt * mgt * mgh) *
                    (double)P.tth_c * TTH_WEIGHT_SCALE);
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
    // the Higgs pair: m_H^2 (Breit-Wigner over its window), then f -> (E1, E2)
    const BW hq = bw_map(c.m_lo, c.m_rng, P.mh2, P.mhgh, x[7], xc[7], c.psi_h);
    float e_big, e_small, Jf;
    if (!th_pair(c, hq.q2, x[6], e_big, e_small, Jf)) return 0.f;
    // double-float momenta and virtualities in units of DL_UNIT (exact from FP32)
    const DLMom b = dl_mom(Eb, c.bnx, c.bny, c.bnz), bb = dl_mom(Ebb, c.bbnx, c.bbny, c.bbnz);
    const DLMom lp = dl_mom(c.Elp, c.lpnx, c.lpny, c.lpnz), lm = dl_mom(c.Elm, c.lmnx, c.lmny, c.lmnz);
    constexpr float iu2 = DL_IU * DL_IU;
    const df vx = ((lp.v[1] + lm.v[1]) + b.v[1]) + bb.v[1];   // visible pT of the four objects
    const df vy = ((lp.v[2] + lm.v[2]) + b.v[2]) + bb.v[2];
    const float m = sqrtf(P.mt2);
    LCv Lb, Lbb, Llp, Llm;
    Lb.pp = Eb * c.blcp; Lb.pm = Eb * c.blcm; Lb.pt = C(Eb * c.bnx, Eb * c.bny);
    Lbb.pp = Ebb * c.bblcp; Lbb.pm = Ebb * c.bblcm; Lbb.pt = C(Ebb * c.bbnx, Ebb * c.bbny);
    Llp.pp = c.Elp * c.lplcp; Llp.pm = c.Elp * c.lplcm; Llp.pt = C(c.Elp * c.lpnx, c.Elp * c.lpny);
    Llm.pp = c.Elm * c.lmlcp; Llm.pm = c.Elm * c.lmlcm; Llm.pt = C(c.Elm * c.lmnx, c.Elm * c.lmny);
    float total = 0.f;
#pragma unroll 1
    for (int o = 0; o < 2; ++o) {
      const float E1 = o == 0 ? e_big : e_small, E2 = o == 0 ? e_small : e_big;
      if (!(E1 >= c.h1_lo && E1 <= c.h1_hi && E2 >= c.h2_lo && E2 <= c.h2_hi)) continue;
      const float e1 = E1 * DL_IU, e2 = E2 * DL_IU;
      const df mx = -((vx + two_prod(e1, c.h1nx)) + two_prod(e2, c.h2nx));
      const df my = -((vy + two_prod(e1, c.h1ny)) + two_prod(e2, c.h2ny));
      DLSystem S;
      df xr[4];
      const int nr = dl_system_met(b, bb, lp, lm, mx, my, df(wp.q2 * iu2), df(wm.q2 * iu2),
                                   df(tq.q2 * iu2), df(tbq.q2 * iu2), S, xr);
      if (nr == 0) continue;
      LCv Lh;
      Lh.pp = fmaf(E1, c.h1lcp, E2 * c.h2lcp);
      Lh.pm = fmaf(E1, c.h1lcm, E2 * c.h2lcm);
      Lh.pt = C(fmaf(E1, c.h1nx, E2 * c.h2nx), fmaf(E1, c.h1ny, E2 * c.h2ny));
      df seen[4][2];
      int ns = 0;
      float acc = 0.f;
#pragma unroll 1
      for (int r = 0; r < nr; ++r) {
        df px, py;
        if (!dl_point(S, xr[r], px, py)) continue;
        bool dup = false;
        for (int k = 0; k < ns; ++k) dup = dup || dl_same(seen[k][0], seen[k][1], px, py);
        if (dup) continue;
        seen[ns][0] = px;
        seen[ns][1] = py;
        ++ns;
        DLMom nu, nub;
        dl_neutrinos(S, px, py, nu, nub);
        const float dec = dl_decay_factor(b, bb, nu, nub, dl_det(b, bb, lp, lm, nu, nub));
        const LCv Ln = dl_lc(nu), Lnb = dl_lc(nub);
        LCv tp, tm;
        tp.pp = Lb.pp + Llp.pp + Ln.pp;
        tp.pm = Lb.pm + Llp.pm + Ln.pm;
        tp.pt = Lb.pt + Llp.pt + Ln.pt;
        tm.pp = Lbb.pp + Llm.pp + Lnb.pp;
        tm.pm = Lbb.pm + Llm.pm + Lnb.pm;
        tm.pt = Lbb.pt + Llm.pt + Lnb.pt;
        const float k1p = tp.pp + tm.pp + Lh.pp;   // no total pT: no boost
        const float k2m = tp.pm + tm.pm + Lh.pm;
        const float x1 = k1p / P.sqrt_s, x2 = k2m / P.sqrt_s;
        if (!(x1 < 1.f && x2 < 1.f)) continue;
        const float shat = k1p * k2m;
        const TTAmp2 amp = tth_amp2(Llp, Llm, tp, tm, Lh, m, P.mt2, k1p, k2m, shat);
        PdfX f1, f2;
        pdf_pair<PDFM>(P, x1, x2, f1, f2);
        const float init = fmaf(P.tt_gg * f1.g * f2.g, amp.gg,
                                P.tt_qq * 2.f * fmaf(f1.q, f2.qb, f1.qb * f2.q) * amp.qq);
        acc += init * (4.f / shat) * (dec * (float)TTH_DEC_SCALE);
      }
      if (acc != 0.f) total += acc * dgauss_g(c, c.E1m, E1) * dgauss_g(c, c.E2m, E2);
    }
    if (total == 0.f) return 0.f;
    const float gb = dgauss_g(c, c.Ebm, Eb), gbb = dgauss_g(c, c.Ebbm, Ebb);
    // Higgs decay 2 m_H^2, the f map's and the (E1, E2) Jacobians
    return (c.cst * Eb * Ebb * gb * gbb * (wp.R * wm.R) * (tq.R * tbq.R) * hq.R *
           (2.f * hq.q2) * Jf * total) * TTH_OUT_SCALE;
  }
};
using PhysTTH = PhysTTH_<PDF_ANY>;

}  // namespace mem

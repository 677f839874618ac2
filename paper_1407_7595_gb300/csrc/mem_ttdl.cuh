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
// Precision: the neutrino solution (mem_dlsolve.cuh) runs in double-float on the FP32
// pipe: its resultant's coefficients cancel beyond FP32's seven digits. Everything else
// (maps, transfer functions, amplitudes, PDFs) is FP32 as in the other processes.
//
// |M|^2: the semileptonic amplitude of mem_ttbar.cuh with mu- in the role of the
// d quark and nubar in that of the ubar (the Fierz-collapsed antitop chain has
// the same form for W- -> mu- nubar), divided by the 6 channels (3 colours x 2
// generations) that the hadronic W- decay carries in its couplings.
#pragma once
#include "mem_ttbar.cuh"
#include "mem_dlsolve.cuh"

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
    // double-float momenta and virtualities in units of DL_UNIT (exact from FP32)
    const DLMom b = dl_mom(Eb, c.bnx, c.bny, c.bnz), bb = dl_mom(Ebb, c.bbnx, c.bbny, c.bbnz);
    const DLMom lp = dl_mom(c.Elp, c.lpnx, c.lpny, c.lpnz), lm = dl_mom(c.Elm, c.lmnx, c.lmny, c.lmnz);
    constexpr float iu2 = DL_IU * DL_IU;
    DLSystem S;
    df xr[4];
    // the missing pT: minus the visible pT of the four objects
    const df mx = -(((lp.v[1] + lm.v[1]) + b.v[1]) + bb.v[1]);
    const df my = -(((lp.v[2] + lm.v[2]) + b.v[2]) + bb.v[2]);
    const int nr = dl_system_met(b, bb, lp, lm, mx, my, df(wp.q2 * iu2), df(wm.q2 * iu2),
                                 df(tq.q2 * iu2), df(tbq.q2 * iu2), S, xr);
    if (nr == 0) return 0.f;
    const float m = sqrtf(P.mt2);
    // FP32 light-cone momenta of the measured partons
    LCv Lb, Lbb, Llp, Llm;
    Lb.pp = Eb * c.blcp; Lb.pm = Eb * c.blcm; Lb.pt = C(Eb * c.bnx, Eb * c.bny);
    Lbb.pp = Ebb * c.bblcp; Lbb.pm = Ebb * c.bblcm; Lbb.pt = C(Ebb * c.bbnx, Ebb * c.bbny);
    Llp.pp = c.Elp * c.lplcp; Llp.pm = c.Elp * c.lplcm; Llp.pt = C(c.Elp * c.lpnx, c.Elp * c.lpny);
    Llm.pp = c.Elm * c.lmlcp; Llm.pm = c.Elm * c.lmlcm; Llm.pt = C(c.Elm * c.lmnx, c.Elm * c.lmny);
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
      acc += init * (4.f / shat) * dec;
    }
    if (acc == 0.f) return 0.f;
    const float gb = dgauss_g(c, c.Ebm, Eb), gbb = dgauss_g(c, c.Ebbm, Ebb);
    return c.cst * Eb * Ebb * gb * gbb * (wp.R * wm.R) * (tq.R * tbq.R) * acc;
  }
};
using PhysTTDL = PhysTTDL_<PDF_ANY>;

}  // namespace mem

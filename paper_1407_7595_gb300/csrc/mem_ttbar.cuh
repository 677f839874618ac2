// Semileptonic ttbar integrand (the hot path of Eq. "integrand", Sec. 3, for
// g g / q qbar -> t tbar -> (b l+ nu)(bbar d ubar)), FP32.
//
// Variables (7): E_d (log-uniform over its jet window), q^2 of the hadronic W
// (-> E_ubar), q^2 of the antitop (-> E_bbar), neutrino px, py (MET box),
// q^2 of the leptonic W (-> neutrino pz, two roots), q^2 of the top (-> E_b,
// per root). All four virtualities use the Breit-Wigner map, so the four
// resonant propagators cancel analytically against their map Jacobians
// (Sec. 3: propagator virtualities as integration variables).
//
// |M|^2: the top decay chain ubar(b) g^mu P_L (p_t/ + m) ... [ubar(nu) g_mu P_L v(l)]
// collapses by the Fierz identity sigma-bar^mu_{ij} sigma-bar_mu,kl = 2 eps_ik eps_jl
// to 2 <b nu> x (row spinor (m w, w^T (p_t.sigma))), w = eps lambda(l+): the
// charged lepton is the spin analyser. Likewise the antitop chain gives
// 2 [bbar ubar] x (column (-(p_tbar.sigma) z, m z)), z = eps conj(lambda(d)).
// Then |M|^2 = couplings x 64 (p_b.p_nu)(p_bbar.p_ubar) x |row Gamma column|^2,
// with Gamma the g g -> t tbar vertices (t- and u-channel top exchange and the
// s-channel gluon, colour orderings T^aT^b / T^bT^a, colour matrix
// [[16/3, -2/3], [-2/3, 16/3]]) or the q qbar -> g* vertex. Gluon polarisations
// are real linear vectors transverse to the beams (each gluon's gauge reference
// is the other beam), which gives the same helicity sum as circular ones.
//
// Kinematics are carried in light-cone form (p+ = E + pz, p- = E - pz, pT = px
// + i py). After the transverse boost, k1+ and k2- are the sums of the
// final-state p+ and p-, and the t/u-channel momenta are p_t - k1 = k2 - p_tbar
// and p_t - k2 = k1 - p_tbar, so their denominators are sums of same-sign terms.
#pragma once
#include "mem_physics.cuh"

namespace mem {

// ---------------------------------------------------------------- complex
struct cf { float re, im; };
__device__ __forceinline__ cf C(float r, float i = 0.f) { return {r, i}; }
__device__ __forceinline__ cf operator+(cf a, cf b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cf operator-(cf a, cf b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cf operator-(cf a) { return {-a.re, -a.im}; }
__device__ __forceinline__ cf operator*(cf a, cf b) {
  return {fmaf(a.re, b.re, -a.im * b.im), fmaf(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ cf operator*(float s, cf a) { return {s * a.re, s * a.im}; }
__device__ __forceinline__ cf conjf(cf a) { return {a.re, -a.im}; }
__device__ __forceinline__ cf mul_i(cf a) { return {-a.im, a.re}; }       // i a
__device__ __forceinline__ cf mul_mi(cf a) { return {a.im, -a.re}; }      // -i a
__device__ __forceinline__ cf fma_c(cf a, cf b, cf c) {                    // a b + c
  return {fmaf(a.re, b.re, fmaf(-a.im, b.im, c.re)), fmaf(a.re, b.im, fmaf(a.im, b.re, c.im))};
}
__device__ __forceinline__ float norm2(cf a) { return fmaf(a.re, a.re, a.im * a.im); }

// Dirac row/column spinor in the chiral basis: (L1, L2, R1, R2).
struct Sp { cf l1, l2, r1, r2; };

__device__ __forceinline__ cf dot4(const Sp& r, const Sp& c) {
  return fma_c(r.l1, c.l1, fma_c(r.l2, c.l2, fma_c(r.r1, c.r1, r.r2 * c.r2)));
}

// Light-cone 4-vector: pp = E + pz, pm = E - pz, pt = px + i py.
struct LCv { float pp, pm; cf pt; };

// row x (a-slash + m): (rR (a.sigma-bar) + m rL, rL (a.sigma) + m rR) with
// a.sigma = [[a-, -conj(aT)], [-aT, a+]], a.sigma-bar = [[a+, conj(aT)], [aT, a-]]
__device__ __forceinline__ Sp row_slash_m(const Sp& r, const LCv& a, float m) {
  const cf act = conjf(a.pt);
  Sp o;
  o.l1 = fma_c(r.r2, a.pt, a.pp * r.r1) + m * r.l1;
  o.l2 = fma_c(r.r1, act, a.pm * r.r2) + m * r.l2;
  o.r1 = a.pm * r.l1 - r.l2 * a.pt + m * r.r1;
  o.r2 = a.pp * r.l2 - r.l1 * act + m * r.r2;
  return o;
}
// row x eps-slash for the real transverse polarisations x^ and y^
__device__ __forceinline__ Sp row_ex(const Sp& r) { return {r.r2, r.r1, -r.l2, -r.l1}; }
__device__ __forceinline__ Sp row_ey(const Sp& r) {
  return {mul_i(r.r2), mul_mi(r.r1), mul_mi(r.l2), mul_i(r.l1)};
}
// eps-slash x column
__device__ __forceinline__ Sp ex_col(const Sp& c) { return {-c.r2, -c.r1, c.l2, c.l1}; }
__device__ __forceinline__ Sp ey_col(const Sp& c) {
  return {mul_i(c.r2), mul_mi(c.r1), mul_mi(c.l2), mul_i(c.l1)};
}

// Massless Weyl spinor lambda(p) with |lambda|^2 = 2E (a phase per particle is
// irrelevant for |M|^2): (-conj(pT)/sqrt(p+), sqrt(p+)) if p+ >= p-, else
// (-sqrt(p-), pT/sqrt(p-)); both use only the larger light-cone component.
__device__ __forceinline__ void weyl(const LCv& p, cf& a, cf& b) {
  if (p.pp >= p.pm) {
    const float r = rsqrtf(p.pp);
    a = -(r * conjf(p.pt));
    b = C(p.pp * r);
  } else {
    const float r = rsqrtf(p.pm);
    a = C(-p.pm * r);
    b = r * p.pt;
  }
}

// Transverse boost (velocity beta = pT_tot / E_tot) of a massless momentum of
// lab energy E, direction (nx, ny), lab light-cone fractions lp = 1 + tanh(eta)
// and lm = 1 - tanh(eta) (or the neutrino's own components).
struct TBoost { float gm1, gam, g2, bx, by; };

__device__ __forceinline__ LCv boost_lc(float E, float px, float py, float lab_pp, float lab_pm,
                                        const TBoost& b) {
  const float bp = fmaf(b.bx, px, b.by * py);        // beta . pT
  const float gbp = b.gam * bp;
  LCv o;
  o.pp = fmaf(b.gm1, E, lab_pp) - gbp;
  o.pm = fmaf(b.gm1, E, lab_pm) - gbp;
  const float c = fmaf(b.g2, bp, -b.gam * E);         // pT' = pT + c beta
  o.pt = C(fmaf(c, b.bx, px), fmaf(c, b.by, py));
  // the smaller light-cone component from pT'^2 / larger (massless)
  const float t2 = norm2(o.pt);
  if (o.pp >= o.pm) o.pm = t2 / o.pp;
  else o.pp = t2 / o.pm;
  return o;
}

// Helicity-summed squared amplitudes of the Fierz-collapsed production and decay
// chain from the transversely boosted l+, d, top and antitop light-cone momenta
// (k1p = x1 sqrt(s), k2m = x2 sqrt(s), shat = k1p k2m, top mass m, m2 = m^2):
// gg = g g -> t tbar with its colour matrix, qq = q qbar -> g* -> t tbar. The decay
// factors (p_b.p_nu)(p_bbar.p_ubar), couplings, averages and the resonant
// propagators are applied by the caller.
struct TTAmp2 { float gg, qq; };

__device__ __forceinline__ TTAmp2 tt_amp2(const LCv& l, const LCv& d, const LCv& tp,
                                          const LCv& tm, float m, float m2, float k1p,
                                          float k2m, float shat) {
  // effective top row and antitop column (Fierz-collapsed decays)
  cf la, lb, da, db;
  weyl(l, la, lb);
  weyl(d, da, db);
  const cf w1 = lb, w2 = -la;                 // w = eps lambda(l)
  const cf z1 = conjf(db), z2 = -conjf(da);   // z = eps conj(lambda(d))
  Sp U;   // (m w, w^T (p_t.sigma)), p_t.sigma = [[p-, -conj(pT)], [-pT, p+]]
  U.l1 = m * w1;
  U.l2 = m * w2;
  U.r1 = tp.pm * w1 - w2 * tp.pt;
  U.r2 = tp.pp * w2 - w1 * conjf(tp.pt);
  Sp Y;   // (-(p_tbar.sigma) z, m z)
  Y.l1 = conjf(tm.pt) * z2 - tm.pm * z1;
  Y.l2 = tm.pt * z1 - tm.pp * z2;
  Y.r1 = m * z1;
  Y.r2 = m * z2;
  // t- and u-channel top momenta: p_t - k1 = k2 - p_tbar, p_t - k2 = k1 - p_tbar
  LCv q1, q2;
  q1.pp = -tm.pp;
  q1.pm = tp.pm;
  q1.pt = tp.pt;
  q2.pp = tp.pp;
  q2.pm = -tm.pm;
  q2.pt = tp.pt;
  const float ptt2 = norm2(tp.pt);
  const float d1 = -(fmaf(tm.pp, tp.pm, ptt2) + m2);   // (p_t - k1)^2 - m^2 < 0
  const float d2 = -(fmaf(tp.pp, tm.pm, ptt2) + m2);   // (p_t - k2)^2 - m^2 < 0
  const float id1 = 1.f / d1, id2 = 1.f / d2;
  // s-channel: U (k1/ - k2/) Y, k1 - k2 = (p+ = k1p, p- = -k2m, pT = 0)
  LCv kk;
  kk.pp = k1p;
  kk.pm = -k2m;
  kk.pt = C(0.f);
  const cf Q = dot4(row_slash_m(U, kk, 0.f), Y);
  const cf sq = (-1.f / shat) * Q;            // V/ = (e1.e2)(k1 - k2)/, e1.e2 = -delta
  const Sp rx = row_ex(U), ry = row_ey(U);
  const Sp tx = row_slash_m(rx, q1, m), ty = row_slash_m(ry, q1, m);
  const Sp ux = row_slash_m(rx, q2, m), uy = row_slash_m(ry, q2, m);
  const Sp ex = ex_col(Y), ey = ey_col(Y);
  float gg = 0.f;
#pragma unroll
  for (int ab = 0; ab < 4; ++ab) {
    const int ia = ab >> 1, ib = ab & 1;
    const Sp& ta = ia ? ty : tx;
    const Sp& ub = ib ? uy : ux;
    const Sp& eb = ib ? ey : ex;
    const Sp& ea = ia ? ey : ex;
    cf A1 = id1 * dot4(ta, eb);   // U e1/ (q1/ + m) e2/ Y / d1
    cf A2 = id2 * dot4(ub, ea);   // U e2/ (q2/ + m) e1/ Y / d2
    if (ia == ib) {
      A1 = A1 + sq;
      A2 = A2 - sq;
    }
    gg += (16.f / 3.f) * (norm2(A1) + norm2(A2)) -
          (4.f / 3.f) * fmaf(A1.re, A2.re, A1.im * A2.im);
  }
  TTAmp2 r;
  r.gg = gg;
  r.qq = (4.f / shat) * (norm2(dot4(rx, Y)) + norm2(dot4(ry, Y)));
  return r;
}

struct JetC {
  float E, nx, ny, nz, sin_t, lcp, lcm;
  float lo, dw;             // window [lo, lo + dw] of the parton energy
};

struct TTCache {
  JetC j[4];                // b, bbar, d, ubar (jets chosen by the permutation)
  float El, lnx, lny, lnz, lsin, llcp, llcm, lom_sin;   // lepton l+
  float Ld;                 // log(hi/lo) of the d window
  float omc_du, omc_bbd, omc_bbu, omc_bl;   // 1 - n_i . n_j
  float metx, mety, B, kbox;
  float psi_hi_wl;          // atan2(m_W G_W, s - m_W^2)
  float core_w, tail_w, inv_core, inv_tail;  // double Gaussian: weights/sigma_rel, 1/sigma_rel
  float cst;
  int ok;
};

template <class CC>   // any cache with the double-Gaussian constants below
__device__ __forceinline__ float dgauss_g(const CC& c, float Em, float E) {
  // sum_k (w_k / c_k) exp(-z_k^2/2), z_k = (Em/E - 1)/c_k
  const float r = fmaf(Em, 1.f / E, -1.f);
  const float z1 = r * c.inv_core, z2 = r * c.inv_tail;
  return fmaf(c.core_w, __expf(-0.5f * z1 * z1), c.tail_w * __expf(-0.5f * z2 * z2));
}

// Lexicographic permutation `perm` (0..23) of (0,1,2,3): parton slot k
// (b, bbar, d, ubar) takes jet p[k].
__host__ __device__ inline void tt_perm_decode(int perm, int (&p)[4]) {
  int rem = perm, avail[4] = {0, 1, 2, 3}, n = 4;
  const int fact[4] = {6, 2, 1, 1};
  for (int k = 0; k < 4; ++k) {
    const int q = rem / fact[k];
    rem %= fact[k];
    p[k] = avail[q];
    for (int t = q; t < n - 1; ++t) avail[t] = avail[t + 1];
    --n;
  }
}

template <int PDFM>
struct PhysTT_ {
  static constexpr int D = 7;
  static constexpr int NPERM = 24;
  using Cache = TTCache;

  __device__ static void setup(const float* rec, int perm, const ProcConst& P, const TFConst& T,
                               Cache& c) {
    int p[4];
    tt_perm_decode(perm, p);
    c.ok = (rec[3] == 4.f || rec[3] == 2.f) && rec[0] > 0.f && perm >= 0 && perm < 24 &&
           T.jet_core > 0.f && T.jet_tail > 0.f && T.met_sigma > 0.f;
    double nj[4][3];
    const double smax = 0.5 * (double)P.sqrt_s;
    double prod_sin = 1.0;
    for (int k = 0; k < 4; ++k) {
      const int o = 1 + p[k];
      const double E = rec[4 * o], eta = rec[4 * o + 1], phi = rec[4 * o + 2];
      c.ok = c.ok && rec[4 * o + 3] == 5.f && E > 0.0;
      const double ch = cosh(eta);
      nj[k][0] = cos(phi) / ch;
      nj[k][1] = sin(phi) / ch;
      nj[k][2] = tanh(eta);
      JetC& J = c.j[k];
      J.E = (float)E;
      J.nx = (float)nj[k][0];
      J.ny = (float)nj[k][1];
      J.nz = (float)nj[k][2];
      J.sin_t = (float)(1.0 / ch);
      J.lcp = (float)(exp(eta) / ch);
      J.lcm = (float)(exp(-eta) / ch);
      const double lo = E / (double)T.jet_lo_div;
      double hi = E * (double)T.jet_hi_mul;
      hi = hi < smax ? hi : smax;
      J.lo = (float)lo;
      J.dw = (float)(hi - lo);
      if (k == 2) c.Ld = (float)log(hi / lo);
      prod_sin *= 1.0 / ch;
      c.ok = c.ok && hi > lo;
    }
    const double El = rec[0], eta = rec[1], phi = rec[2];
    const double ch = cosh(eta);
    const double nl[3] = {cos(phi) / ch, sin(phi) / ch, tanh(eta)};
    c.El = (float)El;
    c.lnx = (float)nl[0];
    c.lny = (float)nl[1];
    c.lnz = (float)nl[2];
    c.lsin = (float)(1.0 / ch);
    c.llcp = (float)(exp(eta) / ch);
    c.llcm = (float)(exp(-eta) / ch);
    c.lom_sin = (float)((ch - 1.0) / ch);
    auto omc = [](const double* a, const double* b) {
      // 1 - a.b = |a - b|^2 / 2 for unit vectors (no cancellation)
      const double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
      return 0.5 * (dx * dx + dy * dy + dz * dz);
    };
    c.omc_du = (float)omc(nj[2], nj[3]);
    c.omc_bbd = (float)omc(nj[1], nj[2]);
    c.omc_bbu = (float)omc(nj[1], nj[3]);
    c.omc_bl = (float)omc(nj[0], nl);
    c.metx = rec[24];
    c.mety = rec[25];
    c.kbox = T.met_box_k;
    c.B = (float)((double)T.met_box_k * T.met_sigma);
    c.psi_hi_wl = (float)atan2((double)P.mwgw, (double)P.s - (double)P.mw2);
    const double tw = T.jet_tail_w;
    c.core_w = (float)((1.0 - tw) / T.jet_core);
    c.tail_w = (float)(tw / T.jet_tail);
    c.inv_core = (float)(1.0 / T.jet_core);
    c.inv_tail = (float)(1.0 / T.jet_tail);
    const double k = T.met_box_k;
    const double mgw = (double)P.mwgw, mgt = (double)P.mtgt;
    // prod sin(theta_j)/(2 pi)^2 (jet TF normalisations), 1/E_l, MET TF x box (2k)^2/(2 pi),
    // L_d / (2 (1 - n_d.n_u)), 1/(m G)_W^2 1/(m G)_t^2, and 1/4 from the energy/pz Jacobians
    // x TT_WEIGHT_SCALE (undone in the FP64 prefactor) keeps FP32 intermediates of
    // far-tail points above the FP32 normal range
    c.cst = (float)(prod_sin / (4.0 * PI_D * PI_D) / El * (4.0 * k * k) / (2.0 * PI_D) *
                    ((double)c.Ld / (2.0 * omc(nj[2], nj[3]))) / (mgw * mgw) / (mgt * mgt) /
                    4.0 * TT_WEIGHT_SCALE);
    c.ok = c.ok && c.omc_du > 0.f;
  }

  __device__ static float eval(const Cache& c, const ProcConst& P, const float (&x)[D],
                               const float (&xc)[D]) {
    const JetC& jb = c.j[0];
    const JetC& jbb = c.j[1];
    const JetC& jd = c.j[2];
    const JetC& ju = c.j[3];
    // d energy (log-uniform over its window)
    const float Ed = jd.lo * __expf(x[0] * c.Ld);
    // hadronic W: q^2 in [2 Ed omc lo_u, 2 Ed omc hi_u] -> E_ubar = q^2 / (2 Ed omc)
    const float aw = 2.f * Ed * c.omc_du;
    const float lo_wh = aw * ju.lo;
    const float dw_wh = aw * ju.dw;
    const BW bwh = bw_map(lo_wh, dw_wh, P.mw2, P.mwgw, x[1], xc[1],
                          atan2_ypos(P.mwgw, lo_wh + dw_wh - P.mw2));
    const float Eu = ju.lo + bwh.d_lo / aw;
    // antitop: q^2 = q^2_Wh + 2 E_bbar K, K = E_Wh - n_bbar . p_Wh
    const float K = fmaf(Ed, c.omc_bbd, Eu * c.omc_bbu);
    const float lo_tb = fmaf(2.f * K, jbb.lo, bwh.q2);
    const float dw_tb = 2.f * K * jbb.dw;
    const BW btb = bw_map(lo_tb, dw_tb, P.mt2, P.mtgt, x[2], xc[2],
                          atan2_ypos(P.mtgt, lo_tb + dw_tb - P.mt2));
    const float Ebb = jbb.lo + btb.d_lo / (2.f * K);
    // neutrino transverse momentum
    const float sx = fmaf(2.f, x[3], -1.f), sy = fmaf(2.f, x[4], -1.f);
    const float nx = fmaf(c.B, sx, c.metx), ny = fmaf(c.B, sy, c.mety);
    const float zm2 = c.kbox * c.kbox * fmaf(sx, sx, sy * sy);
    // leptonic W: q^2 over [mT^2, s] after v = t^2 -> neutrino pz roots
    const float El = c.El;
    const float plx = El * c.lnx, ply = El * c.lny, plz = El * c.lnz;
    const float pTl = El * c.lsin;
    const float pTn = sqrtf(fmaf(nx, nx, ny * ny));
    const float prod = pTl * pTn;
    const float dotT = fmaf(plx, nx, ply * ny);
    const float cross = fmaf(plx, ny, -ply * nx);
    const float h = dotT > 0.f ? cross * cross / (prod + dotT) : prod - dotT;
    const float mt2 = 2.f * h;
    const float t = x[5];
    const BW bwl = bw_map(mt2, P.s - mt2, P.mw2, P.mwgw, t * t, xc[5] * (1.f + t), c.psi_hi_wl);
    const float half = 0.5f * bwl.d_lo;
    const float sD = sqrtf(half * (half + 2.f * prod));
    const float a = half + prod;
    const float qq = fmaf(a, plz, copysignf(El * sD, plz));
    const float pz1 = qq / (pTl * pTl);
    const float pz2 = (pTn * El * c.lom_sin - half) * (pTn * El + a) / qq;
    // the parts of the weight common to both roots
    const float gd = dgauss_g(c, jd.E, Ed), gu = dgauss_g(c, ju.E, Eu);
    const float gbb = dgauss_g(c, jbb.E, Ebb);
    const float common = c.cst * gd * gu * gbb * __expf(-0.5f * zm2) * bwh.R * btb.R * bwl.R *
                         t / (sD * K);
    const float pbbu = Ebb * Eu * c.omc_bbu;   // p_bbar . p_ubar
    // lab light-cone components of the fixed-direction partons of this point
    const float m = sqrtf(P.mt2);
    float acc = 0.f;
#pragma unroll 1
    for (int rr = 0; rr < 2; ++rr) {
      const float pzn = rr == 0 ? pz1 : pz2;
      const float En = sqrtf(fmaf(pzn, pzn, pTn * pTn));
      // neutrino lab light-cone: larger component direct, smaller from pT^2
      float npp = En + pzn, npm = En - pzn;
      if (pzn >= 0.f) npm = pTn * pTn / npp;
      else npp = pTn * pTn / npm;
      // top: q^2_t = q^2_Wl + 2 E_b K_b, K_b = E_l (1 - n_b.n_l) + (E_nu - n_b . p_nu)
      // E_nu - n_b . p_nu; for nearly parallel b and nu use |n_b x p_nu|^2 / (E_nu + n_b . p_nu)
      const float nbp = fmaf(jb.nx, nx, fmaf(jb.ny, ny, jb.nz * pzn));
      float kbn;
      if (nbp > 0.f) {
        const float cx = fmaf(jb.ny, pzn, -jb.nz * ny);
        const float cy = fmaf(jb.nz, nx, -jb.nx * pzn);
        const float cz = fmaf(jb.nx, ny, -jb.ny * nx);
        kbn = fmaf(cx, cx, fmaf(cy, cy, cz * cz)) / (En + nbp);
      } else {
        kbn = En - nbp;
      }
      const float Kb = fmaf(El, c.omc_bl, kbn);
      const float lo_t = fmaf(2.f * Kb, jb.lo, bwl.q2);
      const float dw_t = 2.f * Kb * jb.dw;
      const BW bt = bw_map(lo_t, dw_t, P.mt2, P.mtgt, x[6], xc[6],
                           atan2_ypos(P.mtgt, lo_t + dw_t - P.mt2));
      const float Eb = jb.lo + bt.d_lo / (2.f * Kb);
      const float pbn = Eb * kbn;              // p_b . p_nu
      // lab totals and the transverse boost
      const float Etot = Eb + El + En + Ebb + Ed + Eu;
      const float Px = Eb * jb.nx + plx + nx + Ebb * jbb.nx + Ed * jd.nx + Eu * ju.nx;
      const float Py = Eb * jb.ny + ply + ny + Ebb * jbb.ny + Ed * jd.ny + Eu * ju.ny;
      const float Ppp = Eb * jb.lcp + El * c.llcp + npp + Ebb * jbb.lcp + Ed * jd.lcp + Eu * ju.lcp;
      const float Ppm = Eb * jb.lcm + El * c.llcm + npm + Ebb * jbb.lcm + Ed * jd.lcm + Eu * ju.lcm;
      const float pt2 = fmaf(Px, Px, Py * Py);
      const float shat_lab = fmaf(Ppp, Ppm, -pt2);           // invariant mass^2
      const float Ep = sqrtf(fmaf(0.25f * (Ppp - Ppm), (Ppp - Ppm), shat_lab));
      TBoost B;
      B.gm1 = pt2 / (Ep * (Etot + Ep));
      B.gam = 1.f + B.gm1;
      B.g2 = B.gam * B.gam / (B.gam + 1.f);
      B.bx = Px / Etot;
      B.by = Py / Etot;
      const LCv b = boost_lc(Eb, Eb * jb.nx, Eb * jb.ny, Eb * jb.lcp, Eb * jb.lcm, B);
      const LCv l = boost_lc(El, plx, ply, El * c.llcp, El * c.llcm, B);
      const LCv n = boost_lc(En, nx, ny, npp, npm, B);
      const LCv bb = boost_lc(Ebb, Ebb * jbb.nx, Ebb * jbb.ny, Ebb * jbb.lcp, Ebb * jbb.lcm, B);
      const LCv d = boost_lc(Ed, Ed * jd.nx, Ed * jd.ny, Ed * jd.lcp, Ed * jd.lcm, B);
      const LCv u = boost_lc(Eu, Eu * ju.nx, Eu * ju.ny, Eu * ju.lcp, Eu * ju.lcm, B);
      LCv tp, tm;  // top and antitop
      tp.pp = b.pp + l.pp + n.pp;
      tp.pm = b.pm + l.pm + n.pm;
      tp.pt = b.pt + l.pt + n.pt;
      tm.pp = bb.pp + d.pp + u.pp;
      tm.pm = bb.pm + d.pm + u.pm;
      tm.pt = bb.pt + d.pt + u.pt;
      const float k1p = tp.pp + tm.pp;   // x1 sqrt(s)
      const float k2m = tp.pm + tm.pm;   // x2 sqrt(s)
      const float x1 = k1p / P.sqrt_s, x2 = k2m / P.sqrt_s;
      if (!(x1 < 1.f && x2 < 1.f)) continue;
      const float shat = k1p * k2m;
      const TTAmp2 amp = tt_amp2(l, d, tp, tm, m, P.mt2, k1p, k2m, shat);
      PdfX f1, f2;
      pdf_pair<PDFM>(P, x1, x2, f1, f2);
      const float fg1 = f1.g, fg2 = f2.g, fq1 = f1.q, fq2 = f2.q, fqb1 = f1.qb, fqb2 = f2.qb;
      const float init = fmaf(P.tt_gg * fg1 * fg2, amp.gg,
                              P.tt_qq * 2.f * fmaf(fq1, fqb2, fqb1 * fq2) * amp.qq);
      const float gb = dgauss_g(c, jb.E, Eb);
      acc += init * (4.f / shat) * pbn * gb * bt.R / Kb;
    }
    return common * pbbu * acc;
  }
};
// Densities chosen per call (parity and learned-sampler kernels); the hot kernels use
// PhysTT_<PDF_PARAM / PDF_GRID>.
using PhysTT = PhysTT_<PDF_ANY>;

}  // namespace mem

// Dilepton ttbb integrand (the background of Sec. 3-4), g g / q qbar -> t tbar b bbar ->
// (b l+ nu)(bbar mu- nubar) b bbar.
//
// Variables and assignments as for dilepton ttH (mem_tth.cuh; Sec. 4 applies the same
// transformations to both processes) with the extra b bbar pair in the Higgs pair's
// place; its mass is not resonant, so m^2 is mapped log-uniformly over the pair's
// window [2 (1 - cos) lo1 lo2, 2 (1 - cos) hi1 hi2].
// The pair's two jets enter |M|^2 as (b, bbar) and as (bbar, b).
//
// |M|^2: the Fierz-collapsed top row and antitop column of mem_ttbar.cuh around the
// g g -> t tbar b bbar production written diagram by diagram from the QCD Feynman
// rules in Feynman gauge (quark-gluon vertex i g gamma^mu t^a, quark propagator
// i (q/ + m)/(q^2 - m^2), gluon propagator -i g_{mu nu}/q^2, three-gluon vertex
// g f^{abc}[...], four-gluon vertex -i g^2 [...]): 36 diagrams in 38 colour terms --
// A: e1, e2 and the b bbar gluon on the top line (6 orders); B: e1, e2 and the t tbar
// gluon on the b line (6); C: one external gluon on each line, the lines joined by a
// gluon (8); D: g g -> g* onto one line with the other pair's gluon (4); E: one external
// gluon and a pair gluon at a three-gluon vertex whose third gluon joins the other line
// (8); F: the four-gluon vertex (3 colour structures); G: two three-gluon vertices (3).
// q qbar -> t tbar b bbar: 7 diagrams (g* onto the top line or the b line with the other
// pair's gluon (4), g* -> the two pair gluons (1), both pair gluons from the light line
// (2)), for either beam carrying the quark (the amplitude is not symmetric under the
// exchange). The colour-summed square of each helicity configuration is L^dagger K L with
// the colour matrices K computed on the host from explicit sums over the SU(3)
// generators. Complex 4-vectors are carried in light-cone form (v+, v-, vT, vTbar) with
// vT = vx + i vy and vTbar = vx - i vy independent. Every propagator momentum is written
// as a sum of final-state light-cone components (k1 carries only p+, k2 only p-).
#pragma once
#include "mem_tth.cuh"

namespace mem {

constexpr int TTBB_NGG = 38;
constexpr int TTBB_NQQ = 7;
// Colour matrices K_nm = sum over external colours of conj(C_n) C_m, factorised on the
// host as K = sum_k u_k u_k^dagger (pivoted Cholesky: K is a Gram matrix, of rank 11 for
// g g and 4 for q qbar): rows conj(u_k), rank x N, row major, and the ranks.
__constant__ float2 c_ttbb_ugg[TTBB_NGG * TTBB_NGG];
__constant__ float2 c_ttbb_uqq[TTBB_NQQ * TTBB_NQQ];
__constant__ int c_ttbb_rank[2];

struct CV { cf p, m, t, tb; };

__device__ __forceinline__ CV cv_of(const LCv& a) { return {C(a.pp), C(a.pm), a.pt, conjf(a.pt)}; }
__device__ __forceinline__ CV cv_add(const CV& a, const CV& b) {
  return {a.p + b.p, a.m + b.m, a.t + b.t, a.tb + b.tb};
}
__device__ __forceinline__ CV cv_scale(cf s, const CV& a) { return {s * a.p, s * a.m, s * a.t, s * a.tb}; }
__device__ __forceinline__ cf mulc(cf a, cf b) { return a * b; }
// Minkowski product in light-cone form
__device__ __forceinline__ cf cvdot(const CV& a, const CV& b) {
  return 0.5f * (a.p * b.m + a.m * b.p) - 0.5f * (a.t * b.tb + a.tb * b.t);
}
// row x V/
__device__ __forceinline__ Sp rowV(const Sp& r, const CV& V) {
  Sp o;
  o.l1 = r.r1 * V.p + r.r2 * V.t;
  o.l2 = r.r1 * V.tb + r.r2 * V.m;
  o.r1 = r.l1 * V.m - r.l2 * V.t;
  o.r2 = r.l2 * V.p - r.l1 * V.tb;
  return o;
}
// V/ x column
__device__ __forceinline__ Sp colV(const CV& V, const Sp& c) {
  Sp o;
  o.l1 = V.m * c.r1 - V.tb * c.r2;
  o.l2 = V.p * c.r2 - V.t * c.r1;
  o.r1 = V.p * c.l1 + V.tb * c.l2;
  o.r2 = V.t * c.l1 + V.m * c.l2;
  return o;
}
// (q/ + m) x column / den
__device__ __forceinline__ Sp col_prop(const LCv& q, float m, float den, const Sp& c) {
  const Sp o = colV(cv_of(q), c);
  const float s = 1.f / den;
  return {s * (o.l1 + m * c.l1), s * (o.l2 + m * c.l2), s * (o.r1 + m * c.r1), s * (o.r2 + m * c.r2)};
}
// J^mu = R gamma^mu C in light-cone form
__device__ __forceinline__ CV current(const Sp& R, const Sp& c) {
  CV J;
  J.m = 2.f * (R.r1 * c.l1 + R.l2 * c.r2);
  J.p = 2.f * (R.r2 * c.l2 + R.l1 * c.r1);
  J.tb = -2.f * (R.r2 * c.l1 - R.l2 * c.r1);
  J.t = -2.f * (R.r1 * c.l2 - R.l1 * c.r2);
  return J;
}
// massless column spinors of p (both chiralities), |.|^2 = 2E; a row is the
// conjugate of the other chirality's column
__device__ __forceinline__ void massless_cols(const LCv& p, Sp& cL, Sp& cR) {
  cf e1, e2, z1, z2;
  if (p.pp >= p.pm) {
    const float r = rsqrtf(p.pp);
    e1 = -(r * conjf(p.pt));
    e2 = C(p.pp * r);
    z1 = C(p.pp * r);
    z2 = r * p.pt;
  } else {
    const float r = rsqrtf(p.pm);
    e1 = C(p.pm * r);
    e2 = -(r * p.pt);
    z1 = r * conjf(p.pt);
    z2 = C(p.pm * r);
  }
  cL = {e1, e2, C(0.f), C(0.f)};
  cR = {C(0.f), C(0.f), z1, z2};
}
__device__ __forceinline__ Sp row_of(const Sp& c) { return {conjf(c.r1), conjf(c.r2), conjf(c.l1), conjf(c.l2)}; }

// three-gluon vertex (g f^{abc} stripped to g) contracted with A (momentum kA incoming)
// and B (kB): the vector of the third leg (incoming kC = -kA - kB)
__device__ __forceinline__ CV v3(float g, const CV& A, const CV& kA, const CV& B, const CV& kB) {
  const CV kC = cv_scale(C(-1.f), cv_add(kA, kB));
  const CV kAB = cv_add(kA, cv_scale(C(-1.f), kB));
  const CV kBC = cv_add(kB, cv_scale(C(-1.f), kC));
  const CV kCA = cv_add(kC, cv_scale(C(-1.f), kA));
  CV r = cv_add(cv_scale(cvdot(A, B), kAB), cv_scale(cvdot(kBC, A), B));
  r = cv_add(r, cv_scale(cvdot(kCA, B), A));
  return cv_scale(C(g), r);
}

// The colour-summed square L^dagger K L = sum_k |conj(u_k) . L|^2 from the factor rows
// W (rank x N) in constant memory: rank x N complex products instead of N x N.
template <int N>
__device__ __forceinline__ float colour_quad(const cf* L, const float2* W, int rank) {
  float s = 0.f;
#pragma unroll 1
  for (int k = 0; k < rank; ++k) {
    cf acc = C(0.f);
    for (int mm = 0; mm < N; ++mm) {
      const float2 w = W[k * N + mm];
      acc = fma_c(C(w.x, w.y), L[mm], acc);
    }
    s += norm2(acc);
  }
  return s;
}

struct TTBBAmp2 { float gg, qq12, qq21; };

// Colour- and helicity-summed production |M|^2 with the Fierz-collapsed decays (l+ and
// mu- analysers, top tp and antitop tm light-cone momenta), the extra pair b3 (b) and
// b4 (bbar), for g g and for q qbar with the quark along +z (qq12) or along -z (qq21);
// g = g_s. The decay factors, W couplings and averages are applied by the caller.
static __device__ __noinline__ TTBBAmp2 ttbb_amp2(const LCv& l, const LCv& d, const LCv& tp,
                                                  const LCv& tm, const LCv& b3, const LCv& b4,
                                                  float m, float m2, float k1p, float k2m, float g) {
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
  const cf I1 = C(0.f, 1.f);
  const cf ig = C(0.f, g);
  // pair momenta
  LCv P12, P34;
  P12.pp = tp.pp + tm.pp; P12.pm = tp.pm + tm.pm; P12.pt = tp.pt + tm.pt;
  P34.pp = b3.pp + b4.pp; P34.pm = b3.pm + b4.pm; P34.pt = b3.pt + b4.pt;
  const float s12 = fmaf(P12.pp, P12.pm, -norm2(P12.pt));
  const float s34 = fmaf(P34.pp, P34.pm, -norm2(P34.pt));
  // top-line momenta (from the top side) and denominators, as in tth_amp2 with the pair
  const cf tht = tp.pt + P34.pt, mht = -(tm.pt + P34.pt);
  const float a_pp = tm.pp + P34.pp, b_pm = tm.pm + P34.pm;
  const LCv TA = lc(-a_pp, tp.pm, tp.pt);
  const float dTA = -(fmaf(a_pp, tp.pm, norm2(tp.pt)) + m2);
  const LCv TB = lc(tp.pp, -b_pm, tp.pt);
  const float dTB = -(fmaf(tp.pp, b_pm, norm2(tp.pt)) + m2);
  const LCv TC = lc(tp.pp + P34.pp, tp.pm + P34.pm, tht);
  const float dTC = fmaf(TC.pp, TC.pm, -norm2(tht)) - m2;
  const LCv TD = lc(-a_pp, -b_pm, mht);
  const float dTD = fmaf(a_pp, b_pm, -norm2(mht)) - m2;
  const LCv TE = lc(-tm.pp, tp.pm + P34.pm, tht);
  const float dTE = -(fmaf(tm.pp, tp.pm + P34.pm, norm2(tht)) + m2);
  const LCv TF = lc(tp.pp + P34.pp, -tm.pm, tht);
  const float dTF = -(fmaf(tp.pp + P34.pp, tm.pm, norm2(tht)) + m2);
  // b-line momenta (from the b side), massless
  const cf bht = b3.pt + P12.pt, bmt = -(b4.pt + P12.pt);
  const float c_pp = b4.pp + P12.pp, d_pm = b4.pm + P12.pm;
  const LCv BA = lc(-c_pp, b3.pm, b3.pt);
  const float dBA = -fmaf(c_pp, b3.pm, norm2(b3.pt));
  const LCv BB = lc(b3.pp, -d_pm, b3.pt);
  const float dBB = -fmaf(b3.pp, d_pm, norm2(b3.pt));
  const LCv BC = lc(b3.pp + P12.pp, b3.pm + P12.pm, bht);
  const float dBC = fmaf(BC.pp, BC.pm, -norm2(bht));
  const LCv BD = lc(-c_pp, -d_pm, bmt);
  const float dBD = fmaf(c_pp, d_pm, -norm2(bmt));
  const LCv BE = lc(-b4.pp, b3.pm + P12.pm, bht);
  const float dBE = -fmaf(b4.pp, b3.pm + P12.pm, norm2(bht));
  const LCv BF = lc(b3.pp + P12.pp, -b4.pm, bht);
  const float dBF = -fmaf(b3.pp + P12.pp, b4.pm, norm2(bht));
  // row x i (q/ + m)/den
  auto rprop = [&](const Sp& r, const LCv& q, float mm_, float den) {
    const Sp o = row_slash_m(r, q, mm_);
    const float s = 1.f / den;
    return Sp{s * mul_i(o.l1), s * mul_i(o.l2), s * mul_i(o.r1), s * mul_i(o.r2)};
  };
  // row x i g V/
  auto rvtx = [&](const Sp& r, const CV& V) {
    const Sp o = rowV(r, V);
    return Sp{ig * o.l1, ig * o.l2, ig * o.r1, ig * o.r2};
  };
  const CV K1 = {C(k1p), C(0.f), C(0.f), C(0.f)}, K2 = {C(0.f), C(k2m), C(0.f), C(0.f)};
  const CV K12 = cv_add(K1, K2), mP12 = cv_scale(C(-1.f), cv_of(P12)),
           mP34 = cv_scale(C(-1.f), cv_of(P34));
  const float sh = k1p * k2m;
  const CV EX = {C(0.f), C(0.f), C(1.f), C(1.f)}, EY = {C(0.f), C(0.f), C(0.f, 1.f), C(0.f, -1.f)};
  TTBBAmp2 res = {0.f, 0.f, 0.f};
  // the extra pair's massless spinors
  Sp c3L, c3R, c4L, c4R;
  massless_cols(b3, c3L, c3R);
  massless_cols(b4, c4L, c4R);
  const Sp r3[2] = {row_of(c3R), row_of(c3L)};   // rows of ubar(b3), both chiralities
  const Sp c4[2] = {c4L, c4R};
  // top pair gluon (after its propagator): (-i/s12) (i g) J = (g / s12) J
  const CV Gt = cv_scale(C(g / s12), current(U, Y));
#pragma unroll 1
  for (int hb = 0; hb < 4; ++hb) {
    const Sp& rb = r3[hb >> 1];
    const Sp& cb = c4[hb & 1];
    const CV Gb = cv_scale(C(g / s34), current(rb, cb));
    if (Gb.p.re == 0.f && Gb.p.im == 0.f && Gb.m.re == 0.f && Gb.m.im == 0.f &&
        Gb.t.re == 0.f && Gb.t.im == 0.f && Gb.tb.re == 0.f && Gb.tb.im == 0.f)
      continue;   // helicity-violating combination of the massless pair
    // ---------------- g g
#pragma unroll 1
    for (int pol = 0; pol < 4; ++pol) {
      const CV e1 = (pol >> 1) ? EY : EX, e2 = (pol & 1) ? EY : EX;
      const CV E[2] = {e1, e2};
      cf L[TTBB_NGG];
      int n = 0;
      // A: top line, orders of (e1, e2, Gb)
      {
        const CV V[3] = {e1, e2, Gb};
        const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
        const LCv* q1s[6] = {&TA, &TA, &TB, &TB, &TC, &TC};
        const float d1s[6] = {dTA, dTA, dTB, dTB, dTC, dTC};
        const LCv* q2s[6] = {&TD, &TE, &TD, &TF, &TE, &TF};
        const float d2s[6] = {dTD, dTE, dTD, dTF, dTE, dTF};
        for (int p = 0; p < 6; ++p) {
          Sp r = rvtx(U, V[perm[p][0]]);
          r = rprop(r, *q1s[p], m, d1s[p]);
          r = rvtx(r, V[perm[p][1]]);
          r = rprop(r, *q2s[p], m, d2s[p]);
          r = rvtx(r, V[perm[p][2]]);
          L[n++] = dot4(r, Y);
        }
        // B: b line, orders of (e1, e2, Gt)
        const CV W[3] = {e1, e2, Gt};
        const LCv* p1s[6] = {&BA, &BA, &BB, &BB, &BC, &BC};
        const float e1s[6] = {dBA, dBA, dBB, dBB, dBC, dBC};
        const LCv* p2s[6] = {&BD, &BE, &BD, &BF, &BE, &BF};
        const float e2s[6] = {dBD, dBE, dBD, dBF, dBE, dBF};
        for (int p = 0; p < 6; ++p) {
          Sp r = rvtx(rb, W[perm[p][0]]);
          r = rprop(r, *p1s[p], 0.f, e1s[p]);
          r = rvtx(r, W[perm[p][1]]);
          r = rprop(r, *p2s[p], 0.f, e2s[p]);
          r = rvtx(r, W[perm[p][2]]);
          L[n++] = dot4(r, cb);
        }
      }
      // C: e_x on the top line, e_y on the b line, joined by a gluon
      for (int x = 0; x < 2; ++x) {
        const int y = 1 - x;
        // momentum the joining gluon brings into the b line: P34 - k_y
        const LCv qin = y == 0 ? lc(-P12.pp, P34.pm, P34.pt) : lc(P34.pp, -P12.pm, P34.pt);
        const float sin_ = fmaf(qin.pp, qin.pm, -norm2(qin.pt));
        for (int bo = 0; bo < 2; ++bo) {
          CV J;
          if (bo == 0) {   // e_y first from the b row, then the open vertex
            Sp r = rvtx(rb, E[y]);
            r = y == 0 ? rprop(r, BA, 0.f, dBA) : rprop(r, BB, 0.f, dBB);
            J = current(r, cb);
          } else {         // open vertex first: b3 - qin = k_y - b4
            const LCv q = y == 0 ? lc(P12.pp + b3.pp, -b4.pm, -b4.pt) : lc(-b4.pp, P12.pm + b3.pm, -b4.pt);
            const float den = fmaf(q.pp, q.pm, -norm2(q.pt));
            Sp c = colV(E[y], cb);
            c = {ig * c.l1, ig * c.l2, ig * c.r1, ig * c.r2};
            c = col_prop(q, 0.f, den, c);
            c = {I1 * c.l1, I1 * c.l2, I1 * c.r1, I1 * c.r2};
            J = current(rb, c);
          }
          // open vertex i g, gluon propagator -i / qin^2: g / qin^2
          const CV G = cv_scale(C(g / sin_), J);
          for (int to = 0; to < 2; ++to) {
            Sp r;
            if (to == 0) {
              r = rvtx(U, E[x]);
              r = x == 0 ? rprop(r, TA, m, dTA) : rprop(r, TB, m, dTB);
              r = rvtx(r, G);
            } else {   // G first: p_t - (k_y - P34)
              r = rvtx(U, G);
              r = y == 0 ? rprop(r, TE, m, dTE) : rprop(r, TF, m, dTF);
              r = rvtx(r, E[x]);
            }
            L[n++] = dot4(r, Y);
          }
        }
      }
      // D: g g -> g* onto the top line with Gb, onto the b line with Gt
      const CV Js = cv_scale(C(0.f, -1.f / sh), v3(g, e1, K1, e2, K2));
      for (int to = 0; to < 2; ++to) {
        Sp r;
        if (to == 0) {
          r = rprop(rvtx(U, Js), TD, m, dTD);
          r = rvtx(r, Gb);
        } else {
          r = rprop(rvtx(U, Gb), TC, m, dTC);
          r = rvtx(r, Js);
        }
        L[n++] = dot4(r, Y);
      }
      for (int bo = 0; bo < 2; ++bo) {
        Sp r;
        if (bo == 0) {
          r = rprop(rvtx(rb, Js), BD, 0.f, dBD);
          r = rvtx(r, Gt);
        } else {
          r = rprop(rvtx(rb, Gt), BC, 0.f, dBC);
          r = rvtx(r, Js);
        }
        L[n++] = dot4(r, cb);
      }
      // E: V3(e_x, pair gluon) joining the line with e_y
      for (int x = 0; x < 2; ++x) {
        const int y = 1 - x;
        const CV Kx = x == 0 ? K1 : K2;
        {
          // k_x - P34 into the top line
          const LCv q = x == 0 ? lc(P12.pp, -P34.pm, -P34.pt) : lc(-P34.pp, P12.pm, -P34.pt);
          const float qq = fmaf(q.pp, q.pm, -norm2(q.pt));
          const CV J = cv_scale(C(0.f, -1.f / qq), v3(g, E[x], Kx, Gb, mP34));
          for (int to = 0; to < 2; ++to) {
            Sp r;
            if (to == 0) {
              r = rvtx(U, E[y]);
              r = y == 0 ? rprop(r, TA, m, dTA) : rprop(r, TB, m, dTB);
              r = rvtx(r, J);
            } else {
              r = rvtx(U, J);
              r = x == 0 ? rprop(r, TE, m, dTE) : rprop(r, TF, m, dTF);
              r = rvtx(r, E[y]);
            }
            L[n++] = dot4(r, Y);
          }
        }
        {
          const LCv q = x == 0 ? lc(P34.pp, -P12.pm, -P12.pt) : lc(-P12.pp, P34.pm, -P12.pt);
          const float qq = fmaf(q.pp, q.pm, -norm2(q.pt));
          const CV J = cv_scale(C(0.f, -1.f / qq), v3(g, E[x], Kx, Gt, mP12));
          for (int bo = 0; bo < 2; ++bo) {
            Sp r;
            if (bo == 0) {
              r = rvtx(rb, E[y]);
              r = y == 0 ? rprop(r, BA, 0.f, dBA) : rprop(r, BB, 0.f, dBB);
              r = rvtx(r, J);
            } else {
              r = rvtx(rb, J);
              r = x == 0 ? rprop(r, BE, 0.f, dBE) : rprop(r, BF, 0.f, dBF);
              r = rvtx(r, E[y]);
            }
            L[n++] = dot4(r, cb);
          }
        }
      }
      // F: four-gluon vertex (e1, e2, Gt, Gb)
      {
        const cf ig2 = C(0.f, -g * g);
        const cf e1e2 = cvdot(e1, e2), e1t = cvdot(e1, Gt), e1b = cvdot(e1, Gb);
        const cf e2t = cvdot(e2, Gt), e2b = cvdot(e2, Gb), tb = cvdot(Gt, Gb);
        L[n++] = ig2 * (e1t * e2b - e1b * e2t);
        L[n++] = ig2 * (e1e2 * tb - e1b * e2t);
        L[n++] = ig2 * (e1e2 * tb - e1t * e2b);
      }
      // G: two three-gluon vertices
      {
        L[n++] = cvdot(v3(g, Js, K12, Gt, mP12), Gb);
        const LCv q1 = lc(P34.pp, -P12.pm, -P12.pt);    // k1 - P12
        const float s1 = fmaf(q1.pp, q1.pm, -norm2(q1.pt));
        const CV X1 = cv_scale(C(0.f, -1.f / s1), v3(g, e1, K1, Gt, mP12));
        L[n++] = cvdot(v3(g, e2, K2, Gb, mP34), X1);
        const LCv q2 = lc(-P12.pp, P34.pm, -P12.pt);    // k2 - P12
        const float s2 = fmaf(q2.pp, q2.pm, -norm2(q2.pt));
        const CV X2 = cv_scale(C(0.f, -1.f / s2), v3(g, e2, K2, Gt, mP12));
        L[n++] = cvdot(v3(g, e1, K1, Gb, mP34), X2);
      }
      res.gg += colour_quad<TTBB_NGG>(L, c_ttbb_ugg, c_ttbb_rank[0]);
    }
    // ---------------- q qbar, the quark along +z (o = 0) or -z (o = 1)
#pragma unroll 1
    for (int o = 0; o < 2; ++o) {
      const LCv kq = o == 0 ? lc(k1p, 0.f, C(0.f)) : lc(0.f, k2m, C(0.f));
      const LCv kqb = o == 0 ? lc(0.f, k2m, C(0.f)) : lc(k1p, 0.f, C(0.f));
      Sp qL, qR, aL, aR;
      massless_cols(kq, qL, qR);
      massless_cols(kqb, aL, aR);
      float qsum = 0.f;
#pragma unroll 1
      for (int hq = 0; hq < 4; ++hq) {
        const Sp cq = (hq >> 1) ? qR : qL;                    // u(kq)
        const Sp rqbar = row_of((hq & 1) ? aR : aL);          // vbar(kqb)
        const CV Jq = cv_scale(C(g / sh), current(rqbar, cq));
        if (Jq.p.re == 0.f && Jq.p.im == 0.f && Jq.m.re == 0.f && Jq.m.im == 0.f &&
            Jq.t.re == 0.f && Jq.t.im == 0.f && Jq.tb.re == 0.f && Jq.tb.im == 0.f)
          continue;   // helicity-violating light pair: no coupling to any vector
        cf L[TTBB_NQQ];
        int n = 0;
        for (int to = 0; to < 2; ++to) {
          Sp r;
          if (to == 0) {
            r = rprop(rvtx(U, Jq), TD, m, dTD);
            r = rvtx(r, Gb);
          } else {
            r = rprop(rvtx(U, Gb), TC, m, dTC);
            r = rvtx(r, Jq);
          }
          L[n++] = dot4(r, Y);
        }
        for (int bo = 0; bo < 2; ++bo) {
          Sp r;
          if (bo == 0) {
            r = rprop(rvtx(rb, Jq), BD, 0.f, dBD);
            r = rvtx(r, Gt);
          } else {
            r = rprop(rvtx(rb, Gt), BC, 0.f, dBC);
            r = rvtx(r, Jq);
          }
          L[n++] = dot4(r, cb);
        }
        L[n++] = cvdot(v3(g, Jq, K12, Gt, mP12), Gb);
        // both pair gluons from the light line (antiquark row first): -kqb + P12 or + P34
        for (int lo = 0; lo < 2; ++lo) {
          const LCv& PA = lo == 0 ? P12 : P34;
          const LCv& PB = lo == 0 ? P34 : P12;
          const LCv q = o == 0 ? lc(PA.pp, -PB.pm, PA.pt) : lc(-PB.pp, PA.pm, PA.pt);
          const float den = fmaf(q.pp, q.pm, -norm2(q.pt));
          Sp r = rvtx(rqbar, lo == 0 ? Gt : Gb);
          r = rprop(r, q, 0.f, den);
          r = rvtx(r, lo == 0 ? Gb : Gt);
          L[n++] = dot4(r, cq);
        }
        qsum += colour_quad<TTBB_NQQ>(L, c_ttbb_uqq, c_ttbb_rank[1]);
      }
      if (o == 0) res.qq12 += qsum;
      else res.qq21 += qsum;
    }
  }
  return res;
}


template <int PDFM>
struct PhysTTBB_ {
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
           rec[4] > 0.f && T.jet_core > 0.f && T.jet_tail > 0.f;
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
    // b, bbar: E sin(theta) L / sqrt(2 pi) per jet with E per point; the extra pair's
    // jets: sin(theta) / sqrt(2 pi) (their f and m^2 Jacobians are per point); leptons
    // 1/E each; R / (m G) per W and top Breit-Wigner map; P.ttbb_c: (g_W^2/2)^4 x 64
    // (Fierz) for the two leptonic decays; x TTH_WEIGHT_SCALE.
    const double mgw = (double)P.mwgw, mgt = (double)P.mtgt;
    c.cst = (float)(sn[0] * sn[1] * sn[2] * sn[3] * Lb * Lbb / (4.0 * PI_D * PI_D) /
                    ((double)rec[0] * (double)rec[4]) / (mgw * mgw * mgt * mgt) *
                    (double)P.ttbb_c * TTH_WEIGHT_SCALE);
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
    // the extra pair: its mass is not resonant, m^2 log-uniform over its window
    // (Jacobian m^2 L_m), then f -> (E1, E2) as for the Higgs pair
    const float m2p = c.m_lo * __expf(x[7] * c.Lm);
    float e_big, e_small, Jf;
    if (!th_pair(c, m2p, x[6], e_big, e_small, Jf)) return 0.f;
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
        // the extra pair's jets as (b, bbar) and as (bbar, b)
        LCv Lj1, Lj2;
        Lj1.pp = E1 * c.h1lcp; Lj1.pm = E1 * c.h1lcm; Lj1.pt = C(E1 * c.h1nx, E1 * c.h1ny);
        Lj2.pp = E2 * c.h2lcp; Lj2.pm = E2 * c.h2lcm; Lj2.pt = C(E2 * c.h2nx, E2 * c.h2ny);
        PdfX f1, f2;
        pdf_pair<PDFM>(P, x1, x2, f1, f2);
        float init = 0.f;
#pragma unroll 1
        for (int po = 0; po < 2; ++po) {
          const TTBBAmp2 amp = ttbb_amp2(Llp, Llm, tp, tm, po == 0 ? Lj1 : Lj2, po == 0 ? Lj2 : Lj1,
                                         m, P.mt2, k1p, k2m, P.gs);
          init += (f1.g * f2.g) * amp.gg * (1.f / 256.f) +
                  2.f * (f1.q * f2.qb * amp.qq12 + f1.qb * f2.q * amp.qq21) * (1.f / 36.f);
        }
        acc += init * (4.f / shat) * (dec * (float)TTH_DEC_SCALE);
      }
      if (acc != 0.f) total += acc * dgauss_g(c, c.E1m, E1) * dgauss_g(c, c.E2m, E2);
    }
    if (total == 0.f) return 0.f;
    const float gb = dgauss_g(c, c.Ebm, Eb), gbb = dgauss_g(c, c.Ebbm, Ebb);
    // the pair-mass map's Jacobian m^2 L_m, the f map's and the (E1, E2) Jacobians
    return (c.cst * Eb * Ebb * gb * gbb * (wp.R * wm.R) * (tq.R * tbq.R) * (m2p * c.Lm) * Jf *
           total) * TTH_OUT_SCALE;
  }
};
using PhysTTBB = PhysTTBB_<PDF_ANY>;

}  // namespace mem

/* Physics map, Jacobians, PDFs and transfer functions of the oracle
 * (test infrastructure; see oracle.h). Direct FP64 restatement:
 *
 * - MEM density (Sec. 1, Eq. "mem_def"): sum over flavours of |M|^2 f1 f2/(|q1||q2|)
 *   times the n-body phase-space element (Sec. 1, phase-space equation); the
 *   momentum-conserving delta consumes dx1 dx2 through E and p_z (Jacobian 2/s);
 *   the transverse imbalance is removed by a transverse boost of the final state.
 * - Transfer-function convolution (Sec. 1): delta functions in all directions and
 *   in the ttbar lepton energy, Gaussian lepton energies, double-Gaussian jet
 *   energies, and a Gaussian on the missing transverse momentum for the neutrino.
 * - Jets and energy-integrated leptons carry E^2 sin(theta) dE (Sec. 3, after
 *   Eq. "integrand"), with E = |p| (massless).
 * - Propagator virtualities as integration variables (Sec. 3, the paragraph before
 *   Eq. "dilepsolv"): Breit-Wigner arctan maps for W and top masses; the neutrino
 *   p_z follows from the W mass constraint (both quadratic roots summed).
 */
#include <math.h>
#include <string.h>

#include "oracle.h"
#include "ora_dirac.h"

int ora_dims(int kind) { return kind == 0 ? 2 : kind == 1 ? 4 : kind == 2 ? 7 : kind == 3 ? 6 : 8; }  /* 4, 5: 8 */
int ora_nperm(int kind) { return kind == 2 ? 24 : kind == 3 ? 2 : (kind == 4 || kind == 5) ? 12 : 1; }

double ora_pdf(const ora_process* P, int type, double x) {
  if (!(x > 0.0 && x < 1.0)) return 0.0;
  return P->pdf_A[type] * pow(x, P->pdf_a[type]) * pow(1.0 - x, P->pdf_b[type]);
}

/* Bilinear interpolation in (ln x, ln Q) between the four nodes around the
 * point (Sec. 3 and its PDF listing: per-flavour (x, Q) grids evaluated by
 * bilinear interpolation; here the nodes include both ends of each range, so
 * the step is range/(N - 1)). Outside the table the edge cell's bilinear form
 * continues linearly; a negative result is set to 0. f = 0 unless 0 < x < 1. */
static double grid_pdf(const ora_process* P, int type, double x, double Q) {
  if (!(x > 0.0 && x < 1.0)) return 0.0;
  const int nx = P->grid_nx, nq = P->grid_nq;
  const double hx = (P->grid_lx[1] - P->grid_lx[0]) / (nx - 1);
  const double hq = (P->grid_lq[1] - P->grid_lq[0]) / (nq - 1);
  const double tx = (log(x) - P->grid_lx[0]) / hx;
  const double tq = (log(Q) - P->grid_lq[0]) / hq;
  int i = tx < 0.0 ? 0 : tx > nx - 2 ? nx - 2 : (int)floor(tx);
  int j = tq < 0.0 ? 0 : tq > nq - 2 ? nq - 2 : (int)floor(tq);
  const double a = tx - i, b = tq - j;
  const double* T = P->pdf_grid + (size_t)type * nq * nx;
  const double f = (1.0 - a) * (1.0 - b) * T[j * nx + i] + a * (1.0 - b) * T[j * nx + i + 1] +
                   (1.0 - a) * b * T[(j + 1) * nx + i] + a * b * T[(j + 1) * nx + i + 1];
  return f > 0.0 ? f : 0.0;
}

double ora_pdf_q(const ora_process* P, int type, double x, double Q) {
  return P->pdf_grid ? grid_pdf(P, type, x, Q) : ora_pdf(P, type, x);
}

static double gauss(double x, double mu, double sig) {
  double z = (x - mu) / sig;
  return exp(-0.5 * z * z) / (sqrt(2.0 * M_PI) * sig);
}

/* Double-Gaussian jet response: (1-w) N(x; E, c E) + w N(x; E, t E). */
static double dgauss(const ora_tf* T, double x, double E) {
  return (1.0 - T->jet_tail_w) * gauss(x, E, T->jet_core * E) +
         T->jet_tail_w * gauss(x, E, T->jet_tail * E);
}

typedef struct {
  double E, eta, phi, kind;
  double n[3];
  double sin_theta;
} obj_t;

static obj_t get_obj(const float* rec, int o) {
  obj_t a;
  a.E = rec[4 * o + 0];
  a.eta = rec[4 * o + 1];
  a.phi = rec[4 * o + 2];
  a.kind = rec[4 * o + 3];
  double ch = cosh(a.eta);
  a.n[0] = cos(a.phi) / ch;
  a.n[1] = sin(a.phi) / ch;
  a.n[2] = tanh(a.eta);
  a.sin_theta = 1.0 / ch;
  return a;
}

static rv4 massless(double E, const double* n) { return rv(E, E * n[0], E * n[1], E * n[2]); }

/* Breit-Wigner map of v in [0,1] onto q^2 in [lo, hi]:
 * q^2 = m^2 + m w tan(th), th uniform between atan((lo-m^2)/(m w)) and
 * atan((hi-m^2)/(m w)). Returns q^2, writes dq^2/dv. */
static double bw_map(double lo, double hi, double m, double w, double v, double* jac) {
  double tlo = atan((lo - m * m) / (m * w));
  double thi = atan((hi - m * m) / (m * w));
  double th = tlo + (thi - tlo) * v;
  double c = cos(th);
  *jac = (thi - tlo) * m * w / (c * c);
  return m * m + m * w * tan(th);
}

/* General Lorentz boost into the frame moving with velocity b. */
static rv4 boost(rv4 p, double bx, double by, double bz) {
  double b2 = bx * bx + by * by + bz * bz;
  if (b2 == 0.0) return p;
  double g = 1.0 / sqrt(1.0 - b2);
  double bp = bx * p.v[1] + by * p.v[2] + bz * p.v[3];
  double c = (g - 1.0) * bp / b2 - g * p.v[0];
  return rv(g * (p.v[0] - bp), p.v[1] + c * bx, p.v[2] + c * by, p.v[3] + c * bz);
}

/* Neutrino p_z from q^2 = (p_l + p_nu)^2 with massless lepton and neutrino and
 * known neutrino p_T. Squaring E_l E_nu - p_l.p_nu = q^2/2 gives
 *   pT_l^2 pz^2 - 2 a pz_l pz + (E_l^2 pT_nu^2 - a^2) = 0,  a = q^2/2 + pT_l.pT_nu.
 * Roots by the quadratic formula; jac = 1 / |d q^2 / d pz| with
 * d q^2/d pz = 2 (E_l pz / E_nu - pz_l). Roots that fail the unsquared
 * equation are dropped. */
static int nu_roots(rv4 pl, double nx, double ny, double q2, double* pz, double* jac) {
  double pTl2 = pl.v[1] * pl.v[1] + pl.v[2] * pl.v[2];
  double pTn2 = nx * nx + ny * ny;
  double a = 0.5 * q2 + pl.v[1] * nx + pl.v[2] * ny;
  double A = pTl2, B = -2.0 * a * pl.v[3], C = pl.v[0] * pl.v[0] * pTn2 - a * a;
  double disc = B * B - 4.0 * A * C;
  if (disc < 0.0 || A <= 0.0) return 0;
  double sq = sqrt(disc);
  double cand[2] = {(-B + sq) / (2.0 * A), (-B - sq) / (2.0 * A)};
  int n = 0;
  for (int r = 0; r < 2; ++r) {
    double En = sqrt(pTn2 + cand[r] * cand[r]);
    double q2r = 2.0 * (pl.v[0] * En - pl.v[1] * nx - pl.v[2] * ny - pl.v[3] * cand[r]);
    if (fabs(q2r - q2) > 1e-6 * (fabs(q2) + 1.0)) continue;
    double d = 2.0 * (pl.v[0] * cand[r] / En - pl.v[3]);
    pz[n] = cand[r];
    jac[n] = 1.0 / fabs(d);
    ++n;
  }
  return n;
}

typedef struct {
  int nfs;
  rv4 lab[8];
  double jac;   /* product of the physics-map Jacobians */
  double meas;  /* prod 1/((2pi)^3 2E) and E^2 sin(theta) measure factors */
  double tf;    /* product of transfer functions */
  double aux[8];
} state_t;

static const double TWO_PI = 2.0 * M_PI;
static double inv_ps(double E) { return 1.0 / (pow(TWO_PI, 3) * 2.0 * E); }

/* Lepton energy with a Gaussian TF: log-uniform over the +- k sigma window
 * [Em/(1+k r), Em/(1-k r)]. */
static double lepton_energy(const ora_tf* T, double Em, double x, double* jac) {
  double r = T->lep_rel, k = T->window_k;
  double lo = Em / (1.0 + k * r), hi = Em / (1.0 - k * r);
  double L = log(hi / lo);
  double E = lo * exp(x * L);
  *jac = E * L;
  return E;
}

static void jet_window(const ora_process* P, const ora_tf* T, double Em, double* lo,
                       double* hi) {
  *lo = Em / T->jet_lo_div;
  *hi = fmin(Em * T->jet_hi_mul, 0.5 * P->sqrt_s);
}

static void met_box(const ora_tf* T, const float* rec, double x1, double x2, double* nx,
                    double* ny, double* jac, double* tf) {
  double B = T->met_box_k * T->met_sigma;
  *nx = rec[24] + B * (2.0 * x1 - 1.0);
  *ny = rec[25] + B * (2.0 * x2 - 1.0);
  *jac = (2.0 * B) * (2.0 * B);
  *tf = gauss(rec[24], *nx, T->met_sigma) * gauss(rec[25], *ny, T->met_sigma);
}

/* Squared transverse mass of a massless lepton and a neutrino of given pT. */
static double mt2(rv4 pl, double nx, double ny) {
  double pTl = hypot(pl.v[1], pl.v[2]), pTn = hypot(nx, ny);
  return 2.0 * (pTl * pTn - pl.v[1] * nx - pl.v[2] * ny);
}

static int states_dy(const ora_process* P, const ora_tf* T, const float* rec,
                     const double* x, state_t* st) {
  obj_t o[2] = {get_obj(rec, 0), get_obj(rec, 1)}; /* mu-, mu+ */
  st->nfs = 2;
  st->jac = 1.0;
  st->meas = 1.0;
  st->tf = 1.0;
  for (int i = 0; i < 2; ++i) {
    double J;
    double E = lepton_energy(T, o[i].E, x[i], &J);
    st->jac *= J;
    st->lab[i] = massless(E, o[i].n);
    st->meas *= E * E * o[i].sin_theta * inv_ps(E);
    st->tf *= gauss(o[i].E, E, T->lep_rel * E);
    st->aux[i] = E;
  }
  return 1;
}

static int states_w(const ora_process* P, const ora_tf* T, const float* rec, const double* x,
                    state_t* st) {
  obj_t e = get_obj(rec, 0);
  double Je;
  double Ee = lepton_energy(T, e.E, x[0], &Je);
  rv4 pe = massless(Ee, e.n);
  double nx, ny, Jbox, tfm;
  met_box(T, rec, x[1], x[2], &nx, &ny, &Jbox, &tfm);
  double s = P->sqrt_s * P->sqrt_s;
  double lo = mt2(pe, nx, ny), hi = s;
  if (!(lo < hi)) return 0;
  double t = x[3], dq2;
  double q2 = bw_map(lo, hi, P->mw, P->ww, t * t, &dq2);
  double Jq = dq2 * 2.0 * t;
  double pz[2], jpz[2];
  int n = nu_roots(pe, nx, ny, q2, pz, jpz);
  for (int r = 0; r < n; ++r) {
    double En = sqrt(nx * nx + ny * ny + pz[r] * pz[r]);
    state_t* S = &st[r];
    S->nfs = 2;
    S->lab[0] = pe;
    S->lab[1] = rv(En, nx, ny, pz[r]);
    S->jac = Je * Jbox * Jq * jpz[r];
    S->meas = Ee * Ee * e.sin_theta * inv_ps(Ee) * inv_ps(En);
    S->tf = gauss(e.E, Ee, T->lep_rel * Ee) * tfm;
    rv4 w = rv_add(S->lab[0], S->lab[1]);
    S->aux[0] = q2;
    S->aux[1] = rv_dot(w, w);
    S->aux[2] = Ee;
    S->aux[3] = pz[r];
  }
  return n;
}

static int states_tt(const ora_process* P, const ora_tf* T, const float* rec, int perm,
                     const double* x, state_t* st) {
  static const int perms[24][4] = {
      {0, 1, 2, 3}, {0, 1, 3, 2}, {0, 2, 1, 3}, {0, 2, 3, 1}, {0, 3, 1, 2}, {0, 3, 2, 1},
      {1, 0, 2, 3}, {1, 0, 3, 2}, {1, 2, 0, 3}, {1, 2, 3, 0}, {1, 3, 0, 2}, {1, 3, 2, 0},
      {2, 0, 1, 3}, {2, 0, 3, 1}, {2, 1, 0, 3}, {2, 1, 3, 0}, {2, 3, 0, 1}, {2, 3, 1, 0},
      {3, 0, 1, 2}, {3, 0, 2, 1}, {3, 1, 0, 2}, {3, 1, 2, 0}, {3, 2, 0, 1}, {3, 2, 1, 0}};
  obj_t lep = get_obj(rec, 0);
  obj_t jb = get_obj(rec, 1 + perms[perm][0]);
  obj_t jbb = get_obj(rec, 1 + perms[perm][1]);
  obj_t jd = get_obj(rec, 1 + perms[perm][2]);
  obj_t ju = get_obj(rec, 1 + perms[perm][3]);
  double s = P->sqrt_s * P->sqrt_s;
  double lo, hi, dq2;
  /* d-quark energy: log-uniform over its jet window */
  jet_window(P, T, jd.E, &lo, &hi);
  double L = log(hi / lo);
  double Ed = lo * exp(x[0] * L);
  double J0 = Ed * L;
  rv4 pd = massless(Ed, jd.n);
  /* hadronic W mass -> ubar energy, q^2 range from the ubar jet window */
  double omc = 1.0 - (jd.n[0] * ju.n[0] + jd.n[1] * ju.n[1] + jd.n[2] * ju.n[2]);
  jet_window(P, T, ju.E, &lo, &hi);
  double q2wh = bw_map(2.0 * Ed * lo * omc, 2.0 * Ed * hi * omc, P->mw, P->ww, x[1], &dq2);
  double Eu = q2wh / (2.0 * Ed * omc);
  double J1 = dq2 / (2.0 * Ed * omc);
  rv4 pu = massless(Eu, ju.n);
  rv4 pwh = rv_add(pd, pu);
  /* antitop mass -> bbar energy */
  double K = pwh.v[0] - (jbb.n[0] * pwh.v[1] + jbb.n[1] * pwh.v[2] + jbb.n[2] * pwh.v[3]);
  jet_window(P, T, jbb.E, &lo, &hi);
  double q2tb = bw_map(q2wh + 2.0 * lo * K, q2wh + 2.0 * hi * K, P->mt, P->wt, x[2], &dq2);
  double Ebb = (q2tb - q2wh) / (2.0 * K);
  double J2 = dq2 / (2.0 * K);
  rv4 pbb = massless(Ebb, jbb.n);
  /* neutrino transverse momentum */
  double nx, ny, Jbox, tfm;
  met_box(T, rec, x[3], x[4], &nx, &ny, &Jbox, &tfm);
  /* leptonic W mass -> neutrino pz (two roots) */
  rv4 pl = massless(lep.E, lep.n);
  double wlo = mt2(pl, nx, ny);
  if (!(wlo < s)) return 0;
  double t = x[5];
  double q2wl = bw_map(wlo, s, P->mw, P->ww, t * t, &dq2);
  double J5 = dq2 * 2.0 * t;
  double pz[2], jpz[2];
  int n = nu_roots(pl, nx, ny, q2wl, pz, jpz);
  for (int r = 0; r < n; ++r) {
    state_t* S = &st[r];
    double En = sqrt(nx * nx + ny * ny + pz[r] * pz[r]);
    rv4 pn = rv(En, nx, ny, pz[r]);
    rv4 pwl = rv_add(pl, pn);
    /* top mass -> b energy */
    double Kb = pwl.v[0] - (jb.n[0] * pwl.v[1] + jb.n[1] * pwl.v[2] + jb.n[2] * pwl.v[3]);
    jet_window(P, T, jb.E, &lo, &hi);
    double q2t = bw_map(q2wl + 2.0 * lo * Kb, q2wl + 2.0 * hi * Kb, P->mt, P->wt, x[6], &dq2);
    double Eb = (q2t - q2wl) / (2.0 * Kb);
    double J6 = dq2 / (2.0 * Kb);
    rv4 pb = massless(Eb, jb.n);
    S->nfs = 6;
    S->lab[0] = pb;
    S->lab[1] = pl;
    S->lab[2] = pn;
    S->lab[3] = pbb;
    S->lab[4] = pd;
    S->lab[5] = pu;
    S->jac = J0 * J1 * J2 * Jbox * J5 * jpz[r] * J6;
    double Ej[4] = {Eb, Ebb, Ed, Eu};
    const obj_t* oj[4] = {&jb, &jbb, &jd, &ju};
    S->meas = inv_ps(pl.v[0]) * inv_ps(En);
    S->tf = tfm;
    for (int k = 0; k < 4; ++k) {
      S->meas *= Ej[k] * Ej[k] * oj[k]->sin_theta * inv_ps(Ej[k]);
      S->tf *= dgauss(T, oj[k]->E, Ej[k]);
    }
    S->aux[0] = q2wh;
    S->aux[1] = q2tb;
    S->aux[2] = q2wl;
    S->aux[3] = q2t;
  }
  return n;
}

/* Dilepton ttbar (the final state of Sec. 3-4 without the Higgs): t -> b l+ nu,
 * tbar -> bbar mu- nubar; leptons measured exactly (delta TFs), b-jet energies
 * with the double-Gaussian TF. Variables: x0 -> E_b and x1 -> E_bbar (log-uniform
 * over their jet windows), x2 -> q2_W+ and x3 -> q2_W- (Breit-Wigner maps over
 * [0, s]), x4 -> q2_t over [q2_W+ + (b + l+)^2, s] and x5 -> q2_tbar over
 * [q2_W- + (bbar + mu-)^2, s] (Breit-Wigner; the lower ends are where 2 b.nu = 0).
 * The missing pT at each point is the visible imbalance -(l+ + mu- + b + bbar)_T
 * (Sec. 4, hadron level), so the final state has zero total pT; the neutrinos
 * follow from Eq. "dilepsolv" (ora_dilep_nu), one state per solution, each with
 * its Jacobian. perm 0: object 2 is the b jet, object 3 the bbar; perm 1 the reverse. */
static int states_ttdl(const ora_process* P, const ora_tf* T, const float* rec, int perm,
                       const double* x, state_t* st) {
  obj_t lp = get_obj(rec, 0), lm = get_obj(rec, 1);
  obj_t jb = get_obj(rec, perm == 0 ? 2 : 3), jbb = get_obj(rec, perm == 0 ? 3 : 2);
  const double s = P->sqrt_s * P->sqrt_s;
  double lo, hi;
  jet_window(P, T, jb.E, &lo, &hi);
  double L = log(hi / lo);
  const double Eb = lo * exp(x[0] * L), J0 = Eb * L;
  jet_window(P, T, jbb.E, &lo, &hi);
  L = log(hi / lo);
  const double Ebb = lo * exp(x[1] * L), J1 = Ebb * L;
  rv4 pb = massless(Eb, jb.n), pbb = massless(Ebb, jbb.n);
  rv4 plp = massless(lp.E, lp.n), plm = massless(lm.E, lm.n);
  double j2, j3, j4, j5;
  const double q2wp = bw_map(0.0, s, P->mw, P->ww, x[2], &j2);
  const double q2wm = bw_map(0.0, s, P->mw, P->ww, x[3], &j3);
  const double lo_t = q2wp + 2.0 * rv_dot(pb, plp), lo_tb = q2wm + 2.0 * rv_dot(pbb, plm);
  if (!(lo_t < s && lo_tb < s)) return 0;
  const double q2t = bw_map(lo_t, s, P->mt, P->wt, x[4], &j4);
  const double q2tb = bw_map(lo_tb, s, P->mt, P->wt, x[5], &j5);
  const double metx = -(plp.v[1] + plm.v[1] + pb.v[1] + pbb.v[1]);
  const double mety = -(plp.v[2] + plm.v[2] + pb.v[2] + pbb.v[2]);
  double nu[4 * ORA_MAXSOL], nub[4 * ORA_MAXSOL], jnu[ORA_MAXSOL];
  const int n = ora_dilep_nu(pb.v, pbb.v, plp.v, plm.v, metx, mety, q2wp, q2wm, q2t, q2tb, nu,
                             nub, jnu);
  for (int r = 0; r < n; ++r) {
    state_t* S = &st[r];
    S->nfs = 6;
    S->lab[0] = pb;
    S->lab[1] = plp;
    S->lab[2] = rv(nu[4 * r], nu[4 * r + 1], nu[4 * r + 2], nu[4 * r + 3]);
    S->lab[3] = pbb;
    S->lab[4] = plm;
    S->lab[5] = rv(nub[4 * r], nub[4 * r + 1], nub[4 * r + 2], nub[4 * r + 3]);
    S->jac = J0 * J1 * j2 * j3 * j4 * j5 * jnu[r];
    S->meas = 1.0;
    for (int i = 0; i < 6; ++i) S->meas *= inv_ps(S->lab[i].v[0]);
    S->meas *= Eb * Eb * jb.sin_theta * Ebb * Ebb * jbb.sin_theta;
    S->tf = dgauss(T, jb.E, Eb) * dgauss(T, jbb.E, Ebb);
    S->aux[0] = q2wp;
    S->aux[1] = q2wm;
    S->aux[2] = q2t;
    S->aux[3] = q2tb;
  }
  return n;
}

/* Dilepton ttH (Sec. 3-4, Eq. "integrand" with Eq. "mhsolve"): t -> b l+ nu,
 * tbar -> bbar mu- nubar, H -> b1 b2; leptons and jet directions exact, the four
 * b-jet energies with the double-Gaussian TF. perm (0..11) picks the jets (objects
 * 2..5) of the b and the bbar -- the (perm / 3)-th jet and the (perm % 3)-th of the
 * other three -- and gives the remaining two to the Higgs pair in object order (the
 * two energy solutions below cover both energy orderings of the pair, so the pair is
 * unordered). Variables: x0..x5 as in dilepton ttbar; x7 -> m_H^2 = 2 E1 E2 (1 - cos
 * theta_12) (Breit-Wigner map over [2 (1 - cos) lo1 lo2, 2 (1 - cos) hi1 hi2], the values
 * the two jet windows allow); with K = E1 E2 the energy E1 lies in [A, B] = [max(lo1,
 * K/hi2), min(hi1, K/lo2)] and f = E1 + E2 = E1 + K/E1 in [f_min, f_max], its image (f_min
 * = 2 sqrt(K) when sqrt(K) is inside); x6 -> f = f_min + (f_max - f_min) x6^2 (the square
 * removes the 1/sqrt end-point singularity below). Given f and K, E1,2 = (f +-
 * sqrt(f^2 - 4K)) / 2, both orderings, each with 1 / |d(f, m_H^2)/d(E1, E2)| =
 * 1 / (2 (1 - cos theta_12) |E1 - E2|); at least one ordering lies inside both jet
 * windows by construction, one that leaves a window has no weight. Then the missing pT is the visible imbalance and the neutrinos follow from Eq. "dilepsolv" as for dilepton ttbar.
 * Dilepton ttbb (kind 5, the background) uses the same variables (Sec. 4 applies the
 * transformations to both processes) with the extra b bbar pair in the role of the Higgs
 * pair; its mass is not resonant, so m^2 is mapped log-uniformly over the same window. */
static void tth_perm(int perm, int* jb, int* jbb, int* j1, int* j2) {
  int rest[3], n = 0;
  const int ib = perm / 3;
  for (int j = 0; j < 4; ++j)
    if (j != ib) rest[n++] = j;
  *jb = 2 + ib;
  *jbb = 2 + rest[perm % 3];
  int h[2], m = 0;
  for (int k = 0; k < 3; ++k)
    if (k != perm % 3) h[m++] = rest[k];
  *j1 = 2 + h[0];
  *j2 = 2 + h[1];
}

static int states_tthdl(const ora_process* P, const ora_tf* T, const float* rec, int perm,
                        const double* x, state_t* st) {
  if (perm < 0 || perm > 11) return 0;
  int ob, obb, o1, o2;
  tth_perm(perm, &ob, &obb, &o1, &o2);
  obj_t lp = get_obj(rec, 0), lm = get_obj(rec, 1);
  obj_t jb = get_obj(rec, ob), jbb = get_obj(rec, obb), h1 = get_obj(rec, o1), h2 = get_obj(rec, o2);
  const double s = P->sqrt_s * P->sqrt_s;
  double lo, hi;
  jet_window(P, T, jb.E, &lo, &hi);
  double L = log(hi / lo);
  const double Eb = lo * exp(x[0] * L), J0 = Eb * L;
  jet_window(P, T, jbb.E, &lo, &hi);
  L = log(hi / lo);
  const double Ebb = lo * exp(x[1] * L), J1 = Ebb * L;
  rv4 pb = massless(Eb, jb.n), pbb = massless(Ebb, jbb.n);
  rv4 plp = massless(lp.E, lp.n), plm = massless(lm.E, lm.n);
  double j2, j3, j4, j5;
  const double q2wp = bw_map(0.0, s, P->mw, P->ww, x[2], &j2);
  const double q2wm = bw_map(0.0, s, P->mw, P->ww, x[3], &j3);
  const double lo_t = q2wp + 2.0 * rv_dot(pb, plp), lo_tb = q2wm + 2.0 * rv_dot(pbb, plm);
  if (!(lo_t < s && lo_tb < s)) return 0;
  const double q2t = bw_map(lo_t, s, P->mt, P->wt, x[4], &j4);
  const double q2tb = bw_map(lo_tb, s, P->mt, P->wt, x[5], &j5);
  /* the Higgs pair: m^2 = 2 E1 E2 (1 - cos theta_12) first, over the range the two jet
   * windows allow, then f = E1 + E2 over the values its energies reach inside them */
  double lo1, hi1, lo2, hi2;
  jet_window(P, T, h1.E, &lo1, &hi1);
  jet_window(P, T, h2.E, &lo2, &hi2);
  const double dx = h1.n[0] - h2.n[0], dy = h1.n[1] - h2.n[1], dz = h1.n[2] - h2.n[2];
  const double omc = 0.5 * (dx * dx + dy * dy + dz * dz); /* 1 - cos theta_12 */
  if (!(omc > 0.0)) return 0;
  const double mlo = 2.0 * omc * lo1 * lo2, mhi = 2.0 * omc * hi1 * hi2;
  double J7, m2;
  if (P->kind == 4) {
    m2 = bw_map(mlo, mhi, P->mh, P->wh, x[7], &J7);
  } else { /* the extra pair's mass is not resonant: m^2 log-uniform over its window */
    const double Lm = log(mhi / mlo);
    m2 = mlo * exp(x[7] * Lm);
    J7 = m2 * Lm;
  }
  const double K = m2 / (2.0 * omc); /* E1 E2 */
  const double A = fmax(lo1, K / hi2), B = fmin(hi1, K / lo2); /* E1 inside both windows */
  if (!(A < B)) return 0;
  const double r = sqrt(K), fA = A + K / A, fB = B + K / B;
  const double fmn = (A <= r && r <= B) ? 2.0 * r : fmin(fA, fB), fmx = fmax(fA, fB);
  /* f = fmn + (fmx - fmn) v^2: the pre-map cancels the 1/sqrt(f - 2 sqrt(K)) end-point
   * singularity of the (E1, E2) Jacobian when f can reach 2 sqrt(K) */
  const double v = x[6];
  const double f = fmn + (fmx - fmn) * v * v, J6 = 2.0 * v * (fmx - fmn);
  const double disc = f * f - 4.0 * K;
  if (!(disc > 0.0)) return 0;
  const double sq = sqrt(disc);
  const double JH = 1.0 / (2.0 * omc * sq);
  int n = 0;
  for (int o = 0; o < 2; ++o) {
    const double E1 = 0.5 * (f + (o == 0 ? sq : -sq)), E2 = f - E1;
    if (!(E1 >= lo1 && E1 <= hi1 && E2 >= lo2 && E2 <= hi2)) continue;
    rv4 p1 = massless(E1, h1.n), p2 = massless(E2, h2.n);
    const double metx = -(plp.v[1] + plm.v[1] + pb.v[1] + pbb.v[1] + p1.v[1] + p2.v[1]);
    const double mety = -(plp.v[2] + plm.v[2] + pb.v[2] + pbb.v[2] + p1.v[2] + p2.v[2]);
    double nu[4 * 4], nub[4 * 4], jnu[4];
    const int nn = ora_dilep_nu(pb.v, pbb.v, plp.v, plm.v, metx, mety, q2wp, q2wm, q2t, q2tb, nu,
                                nub, jnu);
    for (int r = 0; r < nn && n < ORA_MAXSOL; ++r) {
      state_t* S = &st[n++];
      S->nfs = 8;
      S->lab[0] = pb;
      S->lab[1] = plp;
      S->lab[2] = rv(nu[4 * r], nu[4 * r + 1], nu[4 * r + 2], nu[4 * r + 3]);
      S->lab[3] = pbb;
      S->lab[4] = plm;
      S->lab[5] = rv(nub[4 * r], nub[4 * r + 1], nub[4 * r + 2], nub[4 * r + 3]);
      S->lab[6] = p1;
      S->lab[7] = p2;
      S->jac = J0 * J1 * j2 * j3 * j4 * j5 * J6 * J7 * JH * jnu[r];
      S->meas = 1.0;
      for (int i = 0; i < 8; ++i) S->meas *= inv_ps(S->lab[i].v[0]);
      S->meas *= Eb * Eb * jb.sin_theta * Ebb * Ebb * jbb.sin_theta * E1 * E1 * h1.sin_theta *
                 E2 * E2 * h2.sin_theta;
      S->tf = dgauss(T, jb.E, Eb) * dgauss(T, jbb.E, Ebb) * dgauss(T, h1.E, E1) *
              dgauss(T, h2.E, E2);
      S->aux[0] = q2wp;
      S->aux[1] = q2wm;
      S->aux[2] = q2t;
      S->aux[3] = q2tb;
    }
  }
  return n;
}

static int build_states(const ora_process* P, const ora_tf* T, const float* rec, int perm,
                        const double* x, state_t* st) {
  memset(st, 0, ORA_MAXSOL * sizeof(state_t));
  switch (P->kind) {
    case 0: return states_dy(P, T, rec, x, st);
    case 1: return states_w(P, T, rec, x, st);
    case 2: return states_tt(P, T, rec, perm, x, st);
    case 3: return states_ttdl(P, T, rec, perm, x, st);
    case 4:
    case 5: return states_tthdl(P, T, rec, perm, x, st);
  }
  return 0;
}

/* Transverse boost of the final state to zero total pT, parton momenta and
 * momentum fractions x1 = (E + pz)/sqrt(s), x2 = (E - pz)/sqrt(s). */
static void to_parton_frame(const ora_process* P, const state_t* S, rv4* boo, rv4* k1, rv4* k2,
                            double* x1, double* x2) {
  rv4 tot = rv(0, 0, 0, 0);
  for (int i = 0; i < S->nfs; ++i) tot = rv_add(tot, S->lab[i]);
  double bx = tot.v[1] / tot.v[0], by = tot.v[2] / tot.v[0];
  for (int i = 0; i < S->nfs; ++i) boo[i] = boost(S->lab[i], bx, by, 0.0);
  rv4 T = boost(tot, bx, by, 0.0);
  double rs = P->sqrt_s;
  *x1 = (T.v[0] + T.v[3]) / rs;
  *x2 = (T.v[0] - T.v[3]) / rs;
  *k1 = rv(0.5 * *x1 * rs, 0, 0, 0.5 * *x1 * rs);
  *k2 = rv(0.5 * *x2 * rs, 0, 0, -0.5 * *x2 * rs);
}

/* PDF-weighted, flavour- and orientation-summed |M|^2 (Eq. "mem_def"). */
static double flavour_sum(const ora_process* P, const rv4* b, rv4 k1, rv4 k2, double x1,
                          double x2, const float* rec) {
  double Q = sqrt(x1 * x2) * P->sqrt_s; /* factorisation scale: the partonic mass */
  double fq1 = ora_pdf_q(P, 0, x1, Q), fqb1 = ora_pdf_q(P, 1, x1, Q), fg1 = ora_pdf_q(P, 2, x1, Q);
  double fq2 = ora_pdf_q(P, 0, x2, Q), fqb2 = ora_pdf_q(P, 1, x2, Q), fg2 = ora_pdf_q(P, 2, x2, Q);
  double sum = 0.0;
  if (P->kind == 0) {
    for (int fl = 0; fl < 2; ++fl) {
      sum += fq1 * fqb2 * ora_msq_dy(P, fl, k1.v, k2.v, b[0].v, b[1].v);
      sum += fqb1 * fq2 * ora_msq_dy(P, fl, k2.v, k1.v, b[0].v, b[1].v);
    }
  } else if (P->kind == 1) {
    int charge = rec[3] == 4.0f ? +1 : -1;
    sum += fq1 * fqb2 * ora_msq_w(P, charge, k1.v, k2.v, b[0].v, b[1].v);
    sum += fqb1 * fq2 * ora_msq_w(P, charge, k2.v, k1.v, b[0].v, b[1].v);
  } else if (P->kind == 4) {   /* dilepton ttH */
    sum += fg1 * fg2 *
           ora_msq_tth(P, 0, k1.v, k2.v, b[0].v, b[1].v, b[2].v, b[3].v, b[4].v, b[5].v, b[6].v,
                       b[7].v);
    for (int fl = 0; fl < 2; ++fl) {
      sum += fq1 * fqb2 *
             ora_msq_tth(P, 1, k1.v, k2.v, b[0].v, b[1].v, b[2].v, b[3].v, b[4].v, b[5].v,
                         b[6].v, b[7].v);
      sum += fqb1 * fq2 *
             ora_msq_tth(P, 1, k2.v, k1.v, b[0].v, b[1].v, b[2].v, b[3].v, b[4].v, b[5].v,
                         b[6].v, b[7].v);
    }
  } else if (P->kind == 5) {   /* dilepton ttbb: the extra pair's two jets as (b, bbar) and (bbar, b) */
    for (int o = 0; o < 2; ++o) {
      const rv4 x3 = o == 0 ? b[6] : b[7], x4 = o == 0 ? b[7] : b[6];
      sum += fg1 * fg2 *
             ora_msq_ttbb(P, 0, k1.v, k2.v, b[0].v, b[1].v, b[2].v, b[3].v, b[4].v, b[5].v, x3.v,
                          x4.v);
      for (int fl = 0; fl < 2; ++fl) {
        sum += fq1 * fqb2 *
               ora_msq_ttbb(P, 1, k1.v, k2.v, b[0].v, b[1].v, b[2].v, b[3].v, b[4].v, b[5].v,
                            x3.v, x4.v);
        sum += fqb1 * fq2 *
               ora_msq_ttbb(P, 1, k2.v, k1.v, b[0].v, b[1].v, b[2].v, b[3].v, b[4].v, b[5].v,
                            x3.v, x4.v);
      }
    }
  } else {   /* ttbar (kind 2) and dilepton ttbar (kind 3) */
    sum += fg1 * fg2 *
           ora_msq_ttbar(P, 0, k1.v, k2.v, b[0].v, b[1].v, b[2].v, b[3].v, b[4].v, b[5].v);
    for (int fl = 0; fl < 2; ++fl) { /* u ubar and d dbar */
      sum += fq1 * fqb2 *
             ora_msq_ttbar(P, 1, k1.v, k2.v, b[0].v, b[1].v, b[2].v, b[3].v, b[4].v, b[5].v);
      sum += fqb1 * fq2 *
             ora_msq_ttbar(P, 1, k2.v, k1.v, b[0].v, b[1].v, b[2].v, b[3].v, b[4].v, b[5].v);
    }
  }
  /* W- -> mu- nubar is one channel where W- -> q qbar' counts 3 colours x 2 generations */
  if (P->kind == 3) sum /= 6.0;
  return sum;
}

/* Weight of one final state: PDF-weighted |M|^2, flux 1/(|q1||q2|), (2 pi)^4 and the
 * 2/s of the consumed dx1 dx2, times the state's measure, TF and Jacobian factors.
 * aux (optional): x1, x2, s-hat, PDF-weighted |M|^2. */
static double state_weight(const ora_process* P, const state_t* S, const float* rec,
                           double* aux) {
  rv4 b[8], k1, k2;
  double x1, x2;
  to_parton_frame(P, S, b, &k1, &k2, &x1, &x2);
  if (!(x1 > 0.0 && x1 < 1.0 && x2 > 0.0 && x2 < 1.0)) return 0.0;
  double s = P->sqrt_s * P->sqrt_s;
  double msq = flavour_sum(P, b, k1, k2, x1, x2, rec);
  double flux = 1.0 / (k1.v[0] * k2.v[0]); /* 1/(|q1||q2|) */
  if (aux) {
    aux[0] = x1;
    aux[1] = x2;
    aux[2] = x1 * x2 * s;
    aux[3] = msq;
  }
  return msq * flux * pow(TWO_PI, 4) * (2.0 / s) * S->meas * S->tf * S->jac;
}

/* PDF-weighted, flavour-summed |M|^2 at given parton-frame momenta (fs: the six
 * final-state momenta in the process's lab order, k12: q1 then q2). */
double ora_flavour_msq(const ora_process* P, const double* fs, const double* k12, double x1,
                       double x2, const float* rec) {
  rv4 b[8];
  for (int i = 0; i < 8; ++i) b[i] = rv(fs[4 * i], fs[4 * i + 1], fs[4 * i + 2], fs[4 * i + 3]);
  rv4 k1 = rv(k12[0], k12[1], k12[2], k12[3]), k2 = rv(k12[4], k12[5], k12[6], k12[7]);
  return flavour_sum(P, b, k1, k2, x1, x2, rec);
}

double ora_integrand(const ora_process* P, const ora_tf* T, const float* rec, int perm,
                     const double* x) {
  state_t st[ORA_MAXSOL];
  int n = build_states(P, T, rec, perm, x, st);
  double total = 0.0;
  for (int r = 0; r < n; ++r) total += state_weight(P, &st[r], rec, NULL);
  return total;
}

int ora_integrand_roots(const ora_process* P, const ora_tf* T, const float* rec, int perm,
                        const double* x, double* w_root) {
  state_t st[ORA_MAXSOL];
  int n = build_states(P, T, rec, perm, x, st);
  for (int r = 0; r < n; ++r) w_root[r] = state_weight(P, &st[r], rec, NULL);
  return n;
}

/* Density at given lab-frame final-state momenta with delta-function transfer
 * functions and no change of variables (Sec. 1, Eq. "mem_def" with the n-body
 * phase-space element): PDF-weighted, flavour-summed |M|^2, flux 1/(|q1||q2|),
 * (2 pi)^4, the 2/s of the consumed dx1 dx2 and prod_i 1/((2 pi)^3 2 E_i) at the lab
 * energies; the transverse imbalance is removed by the transverse boost of
 * to_parton_frame. lab: nfs x (E, px, py, pz) in the process's lab order; rec
 * supplies the lepton charge (W). aux as for state_weight. */
double ora_density(const ora_process* P, int nfs, const double* lab, const float* rec,
                   double* aux) {
  if (nfs < 1 || nfs > 8) return 0.0;
  state_t S;
  memset(&S, 0, sizeof(S));
  S.nfs = nfs;
  S.meas = 1.0;
  S.tf = 1.0;
  S.jac = 1.0;
  for (int i = 0; i < nfs; ++i) {
    S.lab[i] = rv(lab[4 * i], lab[4 * i + 1], lab[4 * i + 2], lab[4 * i + 3]);
    S.meas *= inv_ps(lab[4 * i]);
  }
  return state_weight(P, &S, rec, aux);
}

/* Parton-level ttbar weight (Sec. 4, parton level): every final-state momentum is
 * known, so all transfer functions are delta functions and nothing is integrated.
 * The record holds l+, the two b quarks, d, ubar and the neutrino as objects 0..5;
 * bperm = 0 takes object 1 as the b and object 2 as the bbar, bperm = 1 the reverse.
 * Weight = the integrand's density at these momenta: PDF-weighted |M|^2, flux,
 * (2 pi)^4 2/s and prod_i 1/((2 pi)^3 2 E_i) over the six final-state particles. */
double ora_parton_ttbar(const ora_process* P, const float* rec, int bperm, double* aux) {
  if (P->kind != 2 || bperm < 0 || bperm > 1) return 0.0;
  const int slot[6] = {1 + bperm, 0, 5, 2 - bperm, 3, 4}; /* b, l+, nu, bbar, d, ubar */
  state_t S;
  memset(&S, 0, sizeof(S));
  S.nfs = 6;
  S.meas = 1.0;
  S.tf = 1.0;
  S.jac = 1.0;
  for (int i = 0; i < 6; ++i) {
    obj_t o = get_obj(rec, slot[i]);
    S.lab[i] = massless(o.E, o.n);
    S.meas *= inv_ps(o.E);
  }
  return state_weight(P, &S, rec, aux);
}

int ora_kinematics(const ora_process* P, const ora_tf* T, const float* rec, int perm,
                   const double* x, int root, double* fs, double* fs_lab, double* k12,
                   double* aux) {
  state_t st[ORA_MAXSOL];
  int n = build_states(P, T, rec, perm, x, st);
  if (root >= n) return n;
  rv4 b[8], k1, k2;
  double x1, x2;
  to_parton_frame(P, &st[root], b, &k1, &k2, &x1, &x2);
  for (int i = 0; i < st[root].nfs; ++i)
    for (int m = 0; m < 4; ++m) {
      fs[4 * i + m] = b[i].v[m];
      fs_lab[4 * i + m] = st[root].lab[i].v[m];
    }
  for (int m = 0; m < 4; ++m) {
    k12[m] = k1.v[m];
    k12[4 + m] = k2.v[m];
  }
  for (int i = 0; i < 4; ++i) aux[i] = st[root].aux[i];
  aux[4] = x1;
  aux[5] = x2;
  aux[6] = st[root].jac;
  aux[7] = st[root].tf;
  return n;
}

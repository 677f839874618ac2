/* FP64 CPU oracle for the matrix-element-method integral.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this library.
 * The product path (the CUDA library) never routes through it, and the two
 * share no code, headers or tables.
 *
 * What it computes (Sec. 1, Eq. "mem_def", the transfer-function convolution
 * for p_hat, and Eq. "integrand" of Sec. 3): for each event X and jet
 * permutation,
 *   p_hat(X) = (1/N_perm) sum_perm  int du  sum_roots F(Y(u)) J(u)
 * with F = sum_flavour f_a(x1) f_b(x2) |M|^2 / (|q1||q2|) * (2pi)^4 (2/s)
 *          * prod_i 1/((2pi)^3 2E_i) * prod_{energy-integrated i} E_i^2 sin(theta_i)
 *          * prod T(X|Y)
 * and the plain Monte Carlo estimator with its standard error (Sec. 2,
 * Eq. "sum" and the error formula that follows it), on a VEGAS-adapted map
 * (Sec. 2, Lepage's algorithm).
 *
 * Everything is written in the most direct form: 4x4 complex Dirac matrices,
 * explicit spinor sums, textbook quadratic roots, explicit Lorentz boosts.
 */
#ifndef MEM_ORACLE_H
#define MEM_ORACLE_H
#include <stdint.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t kind; /* 0 Drell-Yan, 1 W -> e nu, 2 semileptonic ttbar, 3 dilepton ttbar,
                 * 4 dilepton ttH (H -> b bbar), 5 dilepton ttbb */
  int32_t pad;
  double sqrt_s;
  double mz, wz, mw, ww, mt, wt;
  double alpha, sw2, alpha_s;
  double pdf_A[3], pdf_a[3], pdf_b[3]; /* quark, antiquark, gluon */
  /* Optional tabulated PDFs (Sec. 3: per-flavour grids in (x, Q), bilinear
   * interpolation). NULL: the parametric f(x) = A x^a (1-x)^b above. Else
   * pdf_grid[(t * grid_nq + j) * grid_nx + i] = f_t(x_i, Q_j) for t = quark,
   * antiquark, gluon on the uniform nodes ln x_i = grid_lx[0] + i h_x,
   * h_x = (grid_lx[1] - grid_lx[0]) / (grid_nx - 1), likewise ln Q_j; the
   * factorisation scale is Q = sqrt(x1 x2 s). */
  const double* pdf_grid;
  int32_t grid_nx, grid_nq;
  double grid_lx[2], grid_lq[2];
  double mh, wh, mb; /* Higgs mass and width, b-quark mass in the b Yukawa (ttH) */
} ora_process;

typedef struct {
  double lep_rel;     /* Gaussian sigma/E for lepton energies */
  double window_k;    /* single-Gaussian integration window: +- k sigma */
  double jet_core;    /* double Gaussian: core sigma/E */
  double jet_tail;    /* tail sigma/E */
  double jet_tail_w;  /* tail weight */
  double jet_lo_div;  /* jet window [E/lo_div, min(E*hi_mul, sqrt_s/2)] */
  double jet_hi_mul;
  double met_sigma;   /* MET Gaussian sigma per component */
  double met_box_k;   /* neutrino px,py box: MET +- k sigma */
} ora_tf;

#define ORA_NG 128      /* VEGAS bins per dimension */
#define ORA_MAXD 8
#define ORA_REC 32
#define ORA_MAXSOL 8    /* kinematic solutions per point (dilepton ttH: 2 Higgs-pair x 4 neutrino) */

int ora_dims(int kind);
int ora_nperm(int kind);

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Uniform in (0,1) from a 32-bit word: ((x >> 9) + 0.5) * 2^-23 (exact in FP32). */
double ora_u01(uint32_t x);
/* Unit-cube point for (event_id, perm, point index) from the integration stream. */
void ora_point_u(uint64_t seed, uint64_t event_id, int perm, uint64_t idx, int d, double* u);
/* The same from stream `tag` (2 = base draws of the learned sampler). */
void ora_point_u_tag(uint64_t seed, uint64_t event_id, int perm, uint64_t idx, int d, int tag,
                     double* u);

/* Integrand on the unit cube (physics map + Jacobians, no VEGAS map). */
double ora_integrand(const ora_process* P, const ora_tf* T, const float* rec, int perm,
                     const double* x);

/* Kinematics at one point for tests: writes boosted momenta of the final
 * state (n_fs x 4, in the process's particle order) and the partons k1, k2.
 * fs_lab receives the same momenta before the boost (lab frame).
 * Returns the number of root branches (0 if the point has no solution).
 * `root` picks the branch. Extra diagnostics in aux (process dependent). */
/* Density at lab-frame final-state momenta (nfs x 4: E, px, py, pz) with
 * delta-function TFs and no change of variables: flavour-summed PDF x |M|^2,
 * flux, (2 pi)^4 2/s, prod 1/((2 pi)^3 2E); aux (optional, 4): x1, x2, s-hat,
 * PDF-weighted |M|^2. rec supplies the lepton charge for W. */
double ora_density(const ora_process* P, int nfs, const double* lab, const float* rec,
                   double* aux);

/* Parton-level ttbar weight (Sec. 4): delta TFs for all six final-state partons of a
 * parton-level record (objects l+, b-quark, b-quark, d, ubar, neutrino); bperm 0/1
 * assigns objects 1/2 to (b, bbar) or (bbar, b). aux (NULL or 4 doubles): x1, x2,
 * s-hat, PDF-weighted |M|^2. */
double ora_parton_ttbar(const ora_process* P, const float* rec, int bperm, double* aux);
/* The above for n records on n_threads threads: w_out (NULL or 2n) per assignment,
 * prob_out (n) their mean. */
void ora_parton_batch(const ora_process* P, const float* recs, int64_t n, int n_threads,
                      double* prob_out, double* w_out);

/* The integrand's contribution of each kinematic root (neutrino p_z solution) at
 * point x; returns the number of roots (0..2). Their sum is ora_integrand. */
/* g g (channel 0) or q qbar (channel 1) -> t tbar H with on-shell tops, summed over
 * all spins and colours, averaged over the initial ones (Sec. 3's signal process). */
double ora_msq_tth_production(const ora_process* P, int channel, const double* k1,
                              const double* k2, const double* pt, const double* ptb,
                              const double* pH);
/* The same with the decays t -> b l+ nu, tbar -> bbar mu- nubar, H -> b1 b2 and
 * Breit-Wigner t, tbar, W+, W-, H propagators. */
double ora_msq_tth(const ora_process* P, int channel, const double* k1, const double* k2,
                   const double* pb, const double* pl, const double* pn, const double* pbb,
                   const double* pm, const double* pnb, const double* ph1, const double* ph2);
/* g g (channel 0) or q qbar (channel 1) -> t tbar b bbar with on-shell tops and
 * massless b quarks, all spins and colours summed, initial ones averaged (the ttbb
 * background of Sec. 3-4). */
double ora_msq_ttbb_production(const ora_process* P, int channel, const double* k1,
                               const double* k2, const double* p1, const double* p2,
                               const double* p3, const double* p4);
double ora_ttbb_gauge_probe(const ora_process* P, const double* k1, const double* k2,
                            const double* p1, const double* p2, const double* p3,
                            const double* p4, int which, int hel);
/* The same with the decays t -> b l+ nu, tbar -> bbar mu- nubar (Breit-Wigner t, tbar,
 * W+, W- propagators); (p3, p4) the extra b, bbar. */
double ora_msq_ttbb(const ora_process* P, int channel, const double* k1, const double* k2,
                    const double* pb, const double* pl, const double* pn, const double* pbb,
                    const double* pm, const double* pnb, const double* p3, const double* p4);
void ora_su3_check(double* out);
void ora_ttbb_colour_matrices(double* kgg, double* kqq);
void ora_ttbb_qq_ward_probe(const ora_process* P, const double* k1, const double* k2,
                            const double* p1, const double* p2, const double* p3,
                            const double* p4, double* out);
double ora_tth_gauge_probe(const ora_process* P, const double* k1, const double* k2,
                           const double* pt, const double* ptb, const double* pH, int which,
                           int hel);
double ora_flavour_msq(const ora_process* P, const double* fs, const double* k12, double x1,
                       double x2, const float* rec);
int ora_integrand_roots(const ora_process* P, const ora_tf* T, const float* rec, int perm,
                        const double* x, double* w_root);
int ora_kinematics(const ora_process* P, const ora_tf* T, const float* rec, int perm,
                   const double* x, int root, double* fs, double* fs_lab, double* k12,
                   double* aux);

/* Spin/colour averaged |M|^2 at given momenta (4-vectors E,px,py,pz). */
double ora_msq_dy(const ora_process* P, int flavour /*0 u, 1 d*/, const double* kq,
                  const double* kqb, const double* pl_minus, const double* pl_plus);
double ora_msq_w(const ora_process* P, int charge, const double* kq, const double* kqb,
                 const double* pl, const double* pn);
/* channel 0: g(k1) g(k2); channel 1: q(k1) qbar(k2). Final state b l+ nu bbar d ubar. */
double ora_msq_ttbar(const ora_process* P, int channel, const double* k1, const double* k2,
                     const double* pb, const double* pl, const double* pn, const double* pbb,
                     const double* pd, const double* pu);
/* Production only, on-shell tops, summed over top spins (for closed-form pins). */
double ora_msq_ttbar_production(const ora_process* P, int channel, const double* k1,
                                const double* k2, const double* pt, const double* ptb);
/* Gauge check: |A1|^2+|A2|^2 for on-shell tops, with gluon `which` polarisation
 * replaced by its momentum and the other gluon of helicity index `hel`. */
double ora_ttbar_gauge_probe(const ora_process* P, const double* k1, const double* k2,
                             const double* pt, const double* ptb, int which, int hel);
/* Decay-chain pins. Top at rest (p_t = (m,0,0,0)): for basis spin s (0 up, 1 down
 * along z), out[s] = sum over b, nu, l spins of |row . u_t(s)|^2 where row is the
 * top-side row spinor used by ora_msq_ttbar. Antitop similarly with v_tbar(s). */
void ora_top_decay_probe(const ora_process* P, const double* pb, const double* pl,
                         const double* pn, double* out2);
void ora_antitop_decay_probe(const ora_process* P, const double* pbb, const double* pd,
                             const double* pu, double* out2);

/* Parametric PDF f(x) = A x^a (1-x)^b, zero outside (0,1). type 0 q, 1 qbar, 2 g. */
double ora_pdf(const ora_process* P, int type, double x);
/* PDF of type t (0 quark, 1 antiquark, 2 gluon) at x and factorisation scale Q:
 * the grid's bilinear interpolation if one is attached, else ora_pdf. */
double ora_pdf_q(const ora_process* P, int type, double x, double Q);

/* VEGAS */
void ora_grid_uniform(int d, double* grid /* d x (NG+1) */);
double ora_vegas_map(int d, const double* grid, const double* u, double* x, int* bins);
void ora_vegas_refine(int d, const double* hist /* d x NG */, const double* grid_in,
                      double alpha, double* grid_out);

/* Weights at consecutive points (with grid; NULL grid = uniform). */
void ora_eval_points(const ora_process* P, const ora_tf* T, const float* rec,
                     uint64_t event_id, int perm, uint64_t seed, uint64_t point0, int64_t n,
                     const double* grid, double* w_out);

typedef struct {
  int32_t n_adapt_iters;   /* VEGAS adaptation iterations (excluded from the estimate) */
  int32_t n_threads;       /* worker threads over items */
  uint64_t adapt_points;   /* points per adaptation iteration; 0 = min(2^14, n/8) */
  double alpha;            /* grid compression exponent */
  const double* grid_in;   /* optional starting grid shared by all items (d x (NG+1)) */
  uint64_t event_id_base;  /* id of event 0 in the Philox counter */
  int32_t strat_points;    /* 0: plain sampling after adaptation; k >= 2: stratified
                              sampling with k points in each of n_s^d hypercubes */
  int32_t pad;
} ora_opts;

/* Dilepton ttbar: the neutrino and antineutrino momenta (E, px, py, pz) for given
 * b, bbar, l+, l- momenta (massless), missing pT and the virtualities q2_W+, q2_W-,
 * q2_t, q2_tbar (Sec. 3, Eq. "dilepsolv"); up to 4 solutions in nu_out, nub_out
 * (4 x 4 doubles each) with jac_out[i] = 1 / |det d(q2_W+, q2_t, q2_W-, q2_tbar) /
 * d(nu_x, nu_y, nu_z, nubar_z)|. Returns the number of solutions. */
int ora_dilep_nu(const double* pb, const double* pbb, const double* plp, const double* plm,
                 double metx, double mety, double q2wp, double q2wm, double q2t, double q2tb,
                 double* nu_out, double* nub_out, double* jac_out);

/* Event discriminant D = log10(p_S / p_B) and its first-order error from the
 * errors of the two estimates; returns 1 (NaN outputs) unless both p > 0. */
int ora_discriminant(double p_s, double e_s, double p_b, double e_b, double* D, double* err);

/* Hypercubes per dimension of the stratified phase: the largest n_s >= 1 with
 * k n_s^d <= n (0 if n < k). */
uint64_t ora_strat_side(uint64_t n, int d, int k);

/* Integrate n_events records with n_points per item (item = event x perm).
 * prob/err per event; item_mean/item_err/grid_out optional (per item). */
int ora_integrate(const ora_process* P, const ora_tf* T, const float* recs, int64_t n_events,
                  uint64_t seed, uint64_t n_points, const ora_opts* opt, double* prob,
                  double* err, uint64_t* n_used, double* item_mean, double* item_err,
                  double* grid_out);

#ifdef __cplusplus
}
#endif
#endif

/* Oracle-internal Dirac algebra (test infrastructure; see oracle.h) in the Dirac
 * representation:
 *   gamma^0 = diag(1, -1) in 2x2 blocks, gamma^k = [[0, s_k], [-s_k, 0]],
 *   gamma^5 = [[0, 1], [1, 0]], P_L = (1 - gamma^5)/2, P_R = (1 + gamma^5)/2.
 * Plain 4x4 complex matrices and 4-component spinors. Test oracle only. */
#ifndef ORA_DIRAC_H
#define ORA_DIRAC_H
#include <complex.h>

typedef double complex cplx;
typedef struct { double v[4]; } rv4;     /* real 4-vector (E, px, py, pz) */
typedef struct { cplx v[4]; } cv4;       /* complex 4-vector */
typedef struct { cplx m[4][4]; } dmat;   /* 4x4 complex matrix */
typedef struct { cplx s[4]; } spin;      /* column spinor or row spinor */

rv4 rv(double e, double x, double y, double z);
rv4 rv_add(rv4 a, rv4 b);
rv4 rv_sub(rv4 a, rv4 b);
rv4 rv_scale(rv4 a, double s);
double rv_dot(rv4 a, rv4 b);
cv4 cv_from_rv(rv4 a);
cplx cv_dot(cv4 a, cv4 b);         /* bilinear, metric (+,-,-,-) */
cv4 cv_lin(cplx a, cv4 x, cplx b, cv4 y);

dmat d_zero(void);
dmat d_unit(void);
dmat d_gamma(int mu);
dmat d_gamma5(void);
dmat d_PL(void);
dmat d_PR(void);
dmat d_add(dmat a, dmat b);
dmat d_scale(dmat a, cplx s);
dmat d_mul(dmat a, dmat b);
dmat d_slash(cv4 a);                /* a_mu gamma^mu */
dmat d_slash_r(rv4 a);
spin d_mv(dmat a, spin x);          /* matrix x column */
spin d_vm(spin row, dmat a);        /* row x matrix */
cplx d_rc(spin row, spin col);      /* row . col */
spin d_bar(spin u);                 /* u^dagger gamma^0 (a row) */

/* Basis of solutions of the massless Dirac equation for momentum p:
 * u_s = sqrt(E) (chi_s, (sigma.p_hat) chi_s), chi_0 = (1,0), chi_1 = (0,1).
 * sum_s u_s ubar_s = pslash; the same set spans the massless v spinors. */
spin d_massless(rv4 p, int s);
/* Massive spinors of momentum p and mass m, basis chi_s:
 * u = (sqrt(E+m) chi, (sigma.p) chi / sqrt(E+m)),  sum u ubar = pslash + m
 * v = ((sigma.p) chi / sqrt(E+m), sqrt(E+m) chi),  sum v vbar = pslash - m */
spin d_massive_u(rv4 p, double m, int s);
spin d_massive_v(rv4 p, double m, int s);
/* Current J^mu = row gamma^mu P col for mu = 0..3 (P given). */
cv4 d_current(spin row, dmat P, spin col);
#endif

/* Monte Carlo integration driver of the oracle (test infrastructure; see oracle.h).
 *
 * Per item (event x jet permutation): n_adapt_iters VEGAS iterations of
 * adapt_points points each refine the grid and are excluded from the estimate;
 * the remaining points run on the frozen grid and give the plain MC mean
 * S_N = mean(f) with error sqrt(sum (f - mean)^2 / (N - 1)) / sqrt(N) (Sec. 2,
 * Eq. "sum" and the error estimate after it, read with the square root).
 * Event result: average over permutations (Sec. 4 averages over jet
 * assignments), errors added in quadrature. Points are counted over all
 * iterations. Sums use Neumaier's compensated summation.
 *
 * Stratified sampling (Sec. 4: the VEGAS integrator used "stratified sampling"
 * together with its adaptive map; Lepage's vegas): with strat_points = k the
 * frozen-grid phase divides the map's input cube (0,1)^d into M = n_s^d equal
 * hypercubes, n_s the largest integer with k n_s^d <= the phase's budget, and
 * places k points uniformly in each. The estimate is the mean over hypercubes of
 * the per-cube means; its variance is the sum over hypercubes of the per-cube
 * sample variance / k, divided by M^2. Point j of hypercube c has Philox index
 * (phase start) + c k + j; the hypercube's coordinates are the base-n_s digits
 * of c, dimension 0 the least significant.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

typedef struct {
  double s, c;
} nsum_t;

static void nadd(nsum_t* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static double nval(const nsum_t* a) { return a->s + a->c; }

void ora_eval_points(const ora_process* P, const ora_tf* T, const float* rec,
                     uint64_t event_id, int perm, uint64_t seed, uint64_t point0, int64_t n,
                     const double* grid, double* w_out) {
  int d = ora_dims(P->kind);
  double gbuf[ORA_MAXD * (ORA_NG + 1)];
  if (!grid) {
    ora_grid_uniform(d, gbuf);
    grid = gbuf;
  }
  for (int64_t i = 0; i < n; ++i) {
    double u[ORA_MAXD], x[ORA_MAXD];
    ora_point_u(seed, event_id, perm, point0 + (uint64_t)i, d, u);
    double J = ora_vegas_map(d, grid, u, x, NULL);
    w_out[i] = ora_integrand(P, T, rec, perm, x) * J;
  }
}

typedef struct {
  const ora_process* P;
  const ora_tf* T;
  const float* recs;
  int64_t n_items;
  uint64_t seed, n_points;
  const ora_opts* opt;
  double* item_mean;
  double* item_var;
  uint64_t* item_used;
  double* grid_out;
  int64_t next;
  pthread_mutex_t lock;
} job_t;

static void run_item(job_t* J, int64_t item) {
  const ora_process* P = J->P;
  int d = ora_dims(P->kind), np = ora_nperm(P->kind);
  int64_t ev = item / np;
  int perm = (int)(item % np);
  const float* rec = J->recs + ev * ORA_REC;
  uint64_t eid = J->opt->event_id_base + (uint64_t)ev;
  double grid[ORA_MAXD * (ORA_NG + 1)], grid2[ORA_MAXD * (ORA_NG + 1)];
  if (J->opt->grid_in) memcpy(grid, J->opt->grid_in, sizeof(double) * d * (ORA_NG + 1));
  else ora_grid_uniform(d, grid);
  uint64_t n = J->n_points;
  uint64_t na = J->opt->adapt_points;
  if (na == 0) na = n / 8 < 16384 ? n / 8 : 16384;
  int iters = J->opt->n_adapt_iters;
  uint64_t idx = 0;
  double* hist = (double*)malloc(sizeof(double) * d * ORA_NG);
  for (int it = 0; it < iters; ++it) {
    memset(hist, 0, sizeof(double) * d * ORA_NG);
    for (uint64_t k = 0; k < na; ++k, ++idx) {
      double u[ORA_MAXD], x[ORA_MAXD];
      int bins[ORA_MAXD];
      ora_point_u(J->seed, eid, perm, idx, d, u);
      double jac = ora_vegas_map(d, grid, u, x, bins);
      double w = ora_integrand(P, J->T, rec, perm, x) * jac;
      for (int j = 0; j < d; ++j) hist[j * ORA_NG + bins[j]] += w * w;
    }
    ora_vegas_refine(d, hist, grid, J->opt->alpha, grid2);
    memcpy(grid, grid2, sizeof(double) * d * (ORA_NG + 1));
  }
  free(hist);
  uint64_t nm = n - idx;
  const int k = J->opt->strat_points;
  if (k >= 2) {
    const uint64_t ns = ora_strat_side(nm, d, k);
    uint64_t M = 1;
    for (int j = 0; j < d; ++j) M *= ns;
    nsum_t sm = {0, 0}, sv = {0, 0};
    for (uint64_t c = 0; c < M; ++c) {
      double cell[ORA_MAXD], wk[64];
      uint64_t rest = c;
      for (int j = 0; j < d; ++j) {
        cell[j] = (double)(rest % ns);
        rest /= ns;
      }
      double mean = 0.0;
      for (int i = 0; i < k; ++i) {
        double u[ORA_MAXD], y[ORA_MAXD], x[ORA_MAXD];
        ora_point_u(J->seed, eid, perm, idx + c * (uint64_t)k + (uint64_t)i, d, u);
        for (int j = 0; j < d; ++j) y[j] = (cell[j] + u[j]) / (double)ns;
        double jac = ora_vegas_map(d, grid, y, x, NULL);
        wk[i] = ora_integrand(P, J->T, rec, perm, x) * jac;
        mean += wk[i];
      }
      mean /= k;
      double ss = 0.0;
      for (int i = 0; i < k; ++i) ss += (wk[i] - mean) * (wk[i] - mean);
      nadd(&sm, mean);
      nadd(&sv, ss / (double)(k - 1) / (double)k);
    }
    J->item_mean[item] = nval(&sm) / (double)M;
    J->item_var[item] = nval(&sv) / ((double)M * (double)M);
    J->item_used[item] = idx + (uint64_t)k * M;
    if (J->grid_out) memcpy(J->grid_out + item * d * (ORA_NG + 1), grid, sizeof(double) * d * (ORA_NG + 1));
    return;
  }
  nsum_t s1 = {0, 0}, s2 = {0, 0};
  for (uint64_t k = 0; k < nm; ++k, ++idx) {
    double u[ORA_MAXD], x[ORA_MAXD];
    ora_point_u(J->seed, eid, perm, idx, d, u);
    double jac = ora_vegas_map(d, grid, u, x, NULL);
    double w = ora_integrand(P, J->T, rec, perm, x) * jac;
    nadd(&s1, w);
    nadd(&s2, w * w);
  }
  double mean = nval(&s1) / (double)nm;
  double var = (nval(&s2) / (double)nm - mean * mean) / (double)(nm - 1);
  if (var < 0.0) var = 0.0;
  J->item_mean[item] = mean;
  J->item_var[item] = var;
  J->item_used[item] = n;
  if (J->grid_out) memcpy(J->grid_out + item * d * (ORA_NG + 1), grid, sizeof(double) * d * (ORA_NG + 1));
}

static void* worker(void* arg) {
  job_t* J = (job_t*)arg;
  for (;;) {
    pthread_mutex_lock(&J->lock);
    int64_t item = J->next++;
    pthread_mutex_unlock(&J->lock);
    if (item >= J->n_items) break;
    run_item(J, item);
  }
  return NULL;
}

int ora_integrate(const ora_process* P, const ora_tf* T, const float* recs, int64_t n_events,
                  uint64_t seed, uint64_t n_points, const ora_opts* opt, double* prob,
                  double* err, uint64_t* n_used, double* item_mean, double* item_err,
                  double* grid_out) {
  int np = ora_nperm(P->kind);
  int64_t n_items = n_events * np;
  uint64_t na = opt->adapt_points ? opt->adapt_points : (n_points / 8 < 16384 ? n_points / 8 : 16384);
  if (n_points < (uint64_t)opt->n_adapt_iters * na + 2) return 1;
  if (opt->strat_points == 1 || opt->strat_points < 0 || opt->strat_points > 64) return 1;
  if (opt->strat_points >= 2 &&
      n_points - (uint64_t)opt->n_adapt_iters * na < (uint64_t)opt->strat_points)
    return 1;
  job_t J;
  J.P = P;
  J.T = T;
  J.recs = recs;
  J.n_items = n_items;
  J.seed = seed;
  J.n_points = n_points;
  J.opt = opt;
  J.item_mean = (double*)malloc(sizeof(double) * n_items);
  J.item_var = (double*)malloc(sizeof(double) * n_items);
  J.item_used = (uint64_t*)malloc(sizeof(uint64_t) * n_items);
  J.grid_out = grid_out;
  J.next = 0;
  pthread_mutex_init(&J.lock, NULL);
  int nt = opt->n_threads > 0 ? opt->n_threads : 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nt);
  for (int t = 0; t < nt; ++t) pthread_create(&th[t], NULL, worker, &J);
  for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
  free(th);
  pthread_mutex_destroy(&J.lock);
  for (int64_t e = 0; e < n_events; ++e) {
    nsum_t m = {0, 0}, v = {0, 0};
    uint64_t used = 0;
    for (int p = 0; p < np; ++p) {
      nadd(&m, J.item_mean[e * np + p]);
      nadd(&v, J.item_var[e * np + p]);
      used += J.item_used[e * np + p];
    }
    prob[e] = nval(&m) / np;
    err[e] = sqrt(nval(&v)) / np;
    if (n_used) n_used[e] = used;
  }
  if (item_mean) memcpy(item_mean, J.item_mean, sizeof(double) * n_items);
  if (item_err)
    for (int64_t i = 0; i < n_items; ++i) item_err[i] = sqrt(J.item_var[i]);
  free(J.item_mean);
  free(J.item_var);
  free(J.item_used);
  return 0;
}

uint64_t ora_strat_side(uint64_t n, int d, int k) {
  uint64_t s = 0;
  for (;;) { /* increase while k (s+1)^d <= n */
    uint64_t p = (uint64_t)k;
    for (int j = 0; j < d && p <= n; ++j) p *= s + 1;
    if (p > n) return s;
    ++s;
  }
}

/* Parton-level ttbar weights of n records on n_threads threads (static blocks of
 * events): w_out[2 i + bperm] per b-quark assignment, prob_out[i] = their mean
 * (Sec. 4, parton level: the average over the b-quark assignments). */
typedef struct {
  const ora_process* P;
  const float* recs;
  int64_t lo, hi;
  double *prob, *w;
} parton_job_t;

static void* parton_worker(void* arg) {
  parton_job_t* J = (parton_job_t*)arg;
  for (int64_t i = J->lo; i < J->hi; ++i) {
    double w0 = ora_parton_ttbar(J->P, J->recs + i * ORA_REC, 0, NULL);
    double w1 = ora_parton_ttbar(J->P, J->recs + i * ORA_REC, 1, NULL);
    if (J->w) {
      J->w[2 * i] = w0;
      J->w[2 * i + 1] = w1;
    }
    J->prob[i] = 0.5 * (w0 + w1);
  }
  return NULL;
}

void ora_parton_batch(const ora_process* P, const float* recs, int64_t n, int n_threads,
                      double* prob_out, double* w_out) {
  int nt = n_threads > 0 ? n_threads : 1;
  if (nt > n) nt = n > 0 ? (int)n : 1;
  parton_job_t* jobs = (parton_job_t*)malloc(sizeof(parton_job_t) * nt);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nt);
  for (int t = 0; t < nt; ++t) {
    jobs[t].P = P;
    jobs[t].recs = recs;
    jobs[t].lo = n * t / nt;
    jobs[t].hi = n * (t + 1) / nt;
    jobs[t].prob = prob_out;
    jobs[t].w = w_out;
    pthread_create(&th[t], NULL, parton_worker, &jobs[t]);
  }
  for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}

/* Event discriminant (Sec. 3, the equation after the PDF paragraph): D = log10 of the
 * ratio of the signal and background probability densities, with the error of
 * independent estimates propagated to first order:
 *   sigma_D = sqrt((sigma_S / p_S)^2 + (sigma_B / p_B)^2) / ln(10).
 * Returns 0, or 1 (D and its error set to NaN) unless both densities are > 0. */
int ora_discriminant(double p_s, double e_s, double p_b, double e_b, double* D, double* err) {
  if (!(p_s > 0.0 && p_b > 0.0)) {
    *D = NAN;
    *err = NAN;
    return 1;
  }
  *D = log10(p_s / p_b);
  *err = sqrt((e_s / p_s) * (e_s / p_s) + (e_b / p_b) * (e_b / p_b)) / log(10.0);
  return 0;
}

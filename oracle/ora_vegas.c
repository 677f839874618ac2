/* VEGAS importance grid of the oracle (test infrastructure; see oracle.h).
 * The paper integrates with Lepage's VEGAS (Sec. 2; Sec. 4 uses the 2014
 * Cython/Python implementation). Grid and refinement follow Lepage, J. Comput.
 * Phys. 27 (1978) 192: a separable piecewise-linear map per dimension with NG
 * bins, bin importances from the accumulated squared weights, three-point
 * smoothing, compression ((1-r)/ln(1/r))^alpha, and re-binning to equal
 * importance per new bin. */
#include <math.h>
#include <string.h>

#include "oracle.h"

void ora_grid_uniform(int d, double* grid) {
  for (int j = 0; j < d; ++j)
    for (int i = 0; i <= ORA_NG; ++i) grid[j * (ORA_NG + 1) + i] = (double)i / ORA_NG;
}

/* y in (0,1)^d -> x; returns the Jacobian prod_j NG (x_{i+1} - x_i). */
double ora_vegas_map(int d, const double* grid, const double* u, double* x, int* bins) {
  double J = 1.0;
  for (int j = 0; j < d; ++j) {
    const double* g = grid + j * (ORA_NG + 1);
    double t = u[j] * ORA_NG;
    int i = (int)floor(t);
    if (i >= ORA_NG) i = ORA_NG - 1;
    double w = g[i + 1] - g[i];
    x[j] = g[i] + (t - i) * w;
    J *= ORA_NG * w;
    if (bins) bins[j] = i;
  }
  return J;
}

void ora_vegas_refine(int d, const double* hist, const double* grid_in, double alpha,
                      double* grid_out) {
  for (int j = 0; j < d; ++j) {
    const double* h = hist + j * ORA_NG;
    const double* g = grid_in + j * (ORA_NG + 1);
    double* go = grid_out + j * (ORA_NG + 1);
    double sm[ORA_NG];
    /* smoothing with the unsmoothed neighbours */
    sm[0] = 0.5 * (h[0] + h[1]);
    for (int i = 1; i < ORA_NG - 1; ++i) sm[i] = (h[i - 1] + h[i] + h[i + 1]) / 3.0;
    sm[ORA_NG - 1] = 0.5 * (h[ORA_NG - 2] + h[ORA_NG - 1]);
    double tot = 0.0;
    for (int i = 0; i < ORA_NG; ++i) tot += sm[i];
    if (!(tot > 0.0)) {
      memcpy(go, g, sizeof(double) * (ORA_NG + 1));
      continue;
    }
    double w[ORA_NG], wsum = 0.0;
    for (int i = 0; i < ORA_NG; ++i) {
      double r = sm[i] / tot;
      if (r <= 0.0) w[i] = 0.0;
      else if (r >= 1.0) w[i] = 1.0;
      else w[i] = pow((1.0 - r) / log(1.0 / r), alpha);
      wsum += w[i];
    }
    double per = wsum / ORA_NG;
    go[0] = g[0];
    go[ORA_NG] = g[ORA_NG];
    int i = 0;
    double acc = 0.0; /* importance of old bins before bin i */
    for (int k = 1; k < ORA_NG; ++k) {
      double target = k * per;
      while (i < ORA_NG - 1 && acc + w[i] < target) {
        acc += w[i];
        ++i;
      }
      double frac = w[i] > 0.0 ? (target - acc) / w[i] : 0.0;
      if (frac < 0.0) frac = 0.0;
      if (frac > 1.0) frac = 1.0;
      go[k] = g[i] + frac * (g[i + 1] - g[i]);
    }
  }
}

"""Pins of the oracle's stratified sampling of the frozen-grid phase (Sec. 4: the
VEGAS integrator samples with stratification as well as its adaptive map).

* The side rule: n_s is the largest integer with k n_s^d <= n, and the points
  used are the adaptation plus k n_s^d.
* With one hypercube (n_s = 1) the estimator is the plain mean on the same
  points, and its error the plain standard error.
* Drell-Yan: the stratified estimate agrees with converged Gauss-Legendre
  quadrature within 3 sigma, with an error below 0.75 of plain sampling's at the
  same budget (after the VEGAS map the integrand is flattened, so the gain from
  stratification is moderate: ~0.5 here).
* The reported error matches the scatter over independent seeds (W).
"""
import math

import numpy as np
import pytest


def test_side_rule(ora):
    for n, d, k in [(1000, 2, 2), (2 ** 20, 4, 2), (16, 3, 2), (15, 3, 2), (5000, 7, 4), (3, 2, 2)]:
        s = ora.strat_side(n, d, k)
        assert k * s ** d <= n < k * (s + 1) ** d


def test_single_cube_is_plain(ora, synth):
    P = ora.process(1, synth.DEFAULT_PROCESS)
    T = ora.tf(synth.DEFAULT_TF[1])
    rec = synth.gen_w(1, 61)
    # budget after adaptation = 31: n_s = 1 for d = 4, k = 16 (16 * 2^4 > 31)
    a = ora.integrate(P, T, rec, seed=4, n_points=2 * 64 + 31, n_adapt_iters=2, adapt_points=64,
                      strat_points=16)
    b = ora.integrate(P, T, rec, seed=4, n_points=2 * 64 + 16, n_adapt_iters=2, adapt_points=64)
    assert a["n_used"][0] == 2 * 64 + 16
    assert a["prob"][0] == pytest.approx(b["prob"][0], rel=1e-13, abs=0)
    assert a["err"][0] == pytest.approx(b["err"][0], rel=1e-9, abs=0)


def gl_unit(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1), 0.5 * w


def test_dy_stratified_vs_quadrature(ora, synth):
    P = ora.process(0, synth.DEFAULT_PROCESS)
    T = ora.tf(synth.DEFAULT_TF[0])
    recs = synth.gen_dy(2, 41)
    n = 1 << 13
    strat = ora.integrate(P, T, recs, seed=5, n_points=n, n_adapt_iters=3, adapt_points=1024,
                          strat_points=2)
    plain = ora.integrate(P, T, recs, seed=5, n_points=n, n_adapt_iters=3, adapt_points=1024)
    xg, wg = gl_unit(120)
    for e, rec in enumerate(recs):
        quad = sum(wa * wb * ora.integrand(P, T, rec, 0, [a, b])
                   for a, wa in zip(xg, wg) for b, wb in zip(xg, wg))
        assert abs(strat["prob"][e] - quad) < 3 * strat["err"][e]
        assert strat["err"][e] < 0.75 * plain["err"][e]
        s = ora.strat_side(n - 3 * 1024, 2, 2)
        assert strat["n_used"][e] == 3 * 1024 + 2 * s * s


def test_error_matches_seed_scatter(ora, synth):
    P = ora.process(1, synth.DEFAULT_PROCESS)
    T = ora.tf(synth.DEFAULT_TF[1])
    rec = synth.gen_w(1, 42)
    vals, errs = [], []
    for seed in range(16):
        r = ora.integrate(P, T, rec, seed=2000 + seed, n_points=1 << 13, n_adapt_iters=2,
                          strat_points=2)
        vals.append(r["prob"][0])
        errs.append(r["err"][0])
    ratio = np.std(vals, ddof=1) / np.mean(errs)
    assert 0.6 < ratio < 1.5

"""Pins of the oracle's Monte Carlo integral (Sec. 2, Eq. "sum" and its error
estimate; Sec. 1, the p_hat integral).

* Drell-Yan: the MC estimate agrees with brute-force two-dimensional
  Gauss-Legendre quadrature of the same integrand within 3 sigma, and the
  quadrature is converged.
* The reported MC error matches the scatter of independent seeds.
* The ttbar event result is the average over the 24 jet permutations.
"""
import math

import numpy as np
import pytest


def gl_unit(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1), 0.5 * w


def test_dy_mc_vs_quadrature(ora, synth):
    P = ora.process(0, synth.DEFAULT_PROCESS)
    T = ora.tf(synth.DEFAULT_TF[0])
    recs = synth.gen_dy(2, 41)
    res = ora.integrate(P, T, recs, seed=5, n_points=1 << 15)
    for e, rec in enumerate(recs):
        quads = []
        for n in (100, 140):
            xg, wg = gl_unit(n)
            quads.append(sum(wa * wb * ora.integrand(P, T, rec, 0, [a, b])
                             for a, wa in zip(xg, wg) for b, wb in zip(xg, wg)))
        assert quads[1] == pytest.approx(quads[0], rel=1e-7, abs=0)
        assert abs(res["prob"][e] - quads[1]) < 3 * res["err"][e]
        assert res["err"][e] < 0.02 * quads[1]


def test_error_estimate_matches_seed_scatter(ora, synth):
    P = ora.process(1, synth.DEFAULT_PROCESS)
    T = ora.tf(synth.DEFAULT_TF[1])
    rec = synth.gen_w(1, 42)
    vals, errs = [], []
    for seed in range(12):
        r = ora.integrate(P, T, rec, seed=1000 + seed, n_points=1 << 13, n_adapt_iters=2)
        vals.append(r["prob"][0])
        errs.append(r["err"][0])
    vals, errs = np.array(vals), np.array(errs)
    ratio = vals.std(ddof=1) / errs.mean()
    assert 0.4 < ratio < 2.0
    assert np.all(r["n_used"] == 1 << 13)


def test_ttbar_average_over_permutations(ora, synth):
    P = ora.process(2, synth.DEFAULT_PROCESS)
    T = ora.tf(synth.DEFAULT_TF[2])
    rec = synth.gen_ttbar(1, 43)
    r = ora.integrate(P, T, rec, seed=3, n_points=256, n_adapt_iters=1, adapt_points=64,
                      want_items=True)
    assert r["prob"][0] == pytest.approx(r["item_mean"].mean(), rel=1e-13, abs=0)
    assert r["err"][0] == pytest.approx(math.sqrt((r["item_err"] ** 2).sum()) / 24, rel=1e-13, abs=0)
    assert r["n_used"][0] == 256 * 24
    # the permutation the generator used is among the ones with the largest weight
    truth = int(rec[0, 28])
    order = np.argsort(-r["item_mean"])
    assert truth in order[:8]

"""Pins of the oracle's VEGAS grid (Sec. 2: importance sampling with Lepage's
VEGAS; grid and refinement as in Lepage, J. Comput. Phys. 27 (1978) 192).

* The map is the identity with Jacobian 1 on the uniform grid, and for any grid
  the Jacobian averages to exactly 1 over the unit cube (it is a bijection).
* Refinement keeps a uniform importance histogram a fixed point, keeps edges
  monotone with fixed end points, and moves bins into a peak.
* On a separable peaked function with an analytic integral the adapted grid
  reduces the variance by a large factor and the estimate agrees with the
  exact value.
"""
import math

import numpy as np
import pytest

NG = 128


def test_uniform_grid_is_identity(ora):
    g = ora.grid_uniform(3)
    rng = np.random.default_rng(0)
    for _ in range(20):
        u = rng.uniform(size=3)
        x, J, bins = ora.vegas_map(g, u)
        assert np.allclose(x, u, rtol=0, atol=1e-15) and J == pytest.approx(1.0, rel=1e-14, abs=0)
        assert bins == [int(v * NG) for v in u]


def _random_grid(rng, d):
    g = np.zeros((d, NG + 1))
    for j in range(d):
        w = rng.gamma(0.3, size=NG) + 1e-6
        g[j, 1:] = np.cumsum(w) / w.sum()
    g[:, -1] = 1.0
    return g


def test_jacobian_averages_to_one(ora):
    rng = np.random.default_rng(1)
    g = _random_grid(rng, 2)
    # J is constant on each bin: midpoints of a 128 x 128 lattice integrate it exactly
    us = (np.arange(NG) + 0.5) / NG
    tot = 0.0
    for a in us:
        for b in us:
            tot += ora.vegas_map(g, [a, b])[1]
    assert tot / NG ** 2 == pytest.approx(1.0, rel=1e-12, abs=0)
    # x(u) is increasing and continuous across bin edges
    uu = np.linspace(1e-6, 1 - 1e-6, 5001)
    xs = np.array([ora.vegas_map(g, [v, 0.5])[0][0] for v in uu])
    assert np.all(np.diff(xs) >= 0)


def test_refine_fixed_point_and_shape(ora):
    g = ora.grid_uniform(2)
    flat = np.ones((2, NG))
    g2 = ora.vegas_refine(flat, g)
    assert np.allclose(g2, g, rtol=0, atol=1e-14)
    rng = np.random.default_rng(2)
    gr = _random_grid(rng, 2)
    h = rng.uniform(0, 1, size=(2, NG)) ** 4
    out = ora.vegas_refine(h, gr)
    assert np.all(np.diff(out, axis=1) > 0)
    assert np.all(out[:, 0] == 0.0) and np.all(out[:, -1] == 1.0)
    # a peaked histogram pulls many new edges into the peak region
    h = np.full((1, NG), 1e-3)
    h[0, 60:68] = 100.0
    out = ora.vegas_refine(h, ora.grid_uniform(1))
    inside = np.sum((out[0] > 60 / NG) & (out[0] < 68 / NG))
    assert inside > 40


def test_vegas_on_separable_peak(ora):
    """f(x) = prod_j N(x_j; 0.3, 0.02) on [0,1]^3, exact integral known from erf."""
    d, mu, sig = 3, 0.3, 0.02
    exact = ((math.erf((1 - mu) / (sig * math.sqrt(2))) + math.erf(mu / (sig * math.sqrt(2)))) / 2) ** d

    def f(x):
        return np.prod(np.exp(-0.5 * ((x - mu) / sig) ** 2) / (sig * math.sqrt(2 * math.pi)))

    rng = np.random.default_rng(3)
    grid = ora.grid_uniform(d)

    def run(grid, n, hist=False):
        ws = np.zeros(n)
        hh = np.zeros((d, NG))
        for i in range(n):
            u = rng.uniform(size=d)
            x, J, bins = ora.vegas_map(grid, u)
            w = f(x) * J
            ws[i] = w
            if hist:
                for j in range(d):
                    hh[j, bins[j]] += w * w
        return ws, hh

    w0, _ = run(grid, 4000)
    var0 = w0.var()
    for _ in range(6):
        _, hh = run(grid, 4000, hist=True)
        grid = ora.vegas_refine(hh, grid, 1.5)
    w1, _ = run(grid, 8000)
    assert w1.var() < var0 / 20
    est, err = w1.mean(), w1.std(ddof=1) / math.sqrt(len(w1))
    assert abs(est - exact) < 4 * err

"""Pins of the oracle's dilepton ttbar neutrino solution (Sec. 3, Eq. "dilepsolv":
the two neutrino momenta from the W+-, W--, t- and tbar-virtualities and the
missing transverse momentum).

* Generator truth: with the virtualities and MET of the generated partons, one
  solution is the generated (nu, nubar) to 1e-8.
* Every solution satisfies all eight equations (four virtualities, two MET
  components, two mass shells) with positive energies; there are 0, 2 or 4.
* The Jacobian 1 / |det d(q^2) / d(nu_x, nu_y, nu_z, nubar_z)| of every solution
  against central finite differences of the forward map (virtualities as
  functions of the free neutrino components; independent of the solver).
* Change of variables: for a Gaussian f of the four free neutrino components
  centred on the truth, the integral over the four virtualities of
  sum_solutions f(nu(q^2)) J (estimated by importance sampling through the forward
  map) equals the closed form (2 pi sigma^2)^2 within the Monte Carlo error, and
  every sampled neutrino configuration is among the solutions of its own
  virtualities -- so no solution that carries weight is lost. (The Jacobian's
  value cancels in this estimator; the finite-difference pin fixes it.)
"""
import math

import numpy as np
import pytest


def dot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def virtualities(b, bb, lp, lm, nu, nub):
    return (dot(lp + nu, lp + nu), dot(lm + nub, lm + nub), dot(b + lp + nu, b + lp + nu),
            dot(bb + lm + nub, bb + lm + nub))


@pytest.fixture(scope="module")
def truth(synth):
    return synth.gen_ttbar_dilep(64, 321, truth=True)[1]


def test_truth_recovered(ora, truth):
    for ev in truth:
        b, bb, lp, lm, nu, nub = ev
        q2wp, q2wm, q2t, q2tb = virtualities(b, bb, lp, lm, nu, nub)
        sols = ora.dilep_nu(b, bb, lp, lm, (nu + nub)[1:3], q2wp, q2wm, q2t, q2tb)
        err = min(np.max(np.abs(s[0] - nu)) / nu[0] + np.max(np.abs(s[1] - nub)) / nub[0]
                  for s in sols)
        assert err < 1e-8


def test_all_solutions_satisfy_the_constraints(ora, truth):
    counts = set()
    for ev in truth:
        b, bb, lp, lm, nu, nub = ev
        q2 = virtualities(b, bb, lp, lm, nu, nub)
        met = (nu + nub)[1:3]
        sols = ora.dilep_nu(b, bb, lp, lm, met, *q2)
        counts.add(len(sols))
        for n1, n2, jac in sols:
            assert n1[0] > 0 and n2[0] > 0 and jac > 0
            assert abs(dot(n1, n1)) < 1e-8 * n1[0] ** 2 and abs(dot(n2, n2)) < 1e-8 * n2[0] ** 2
            got = virtualities(b, bb, lp, lm, n1, n2)
            for g, w in zip(got, q2):
                assert g == pytest.approx(w, rel=1e-8, abs=0)
            assert np.allclose(n1[1:3] + n2[1:3], met, rtol=0, atol=1e-8 * n1[0])
    assert counts <= {0, 2, 4} and 4 in counts and 2 in counts


def _forward(b, bb, lp, lm, met, f):
    """(q2_W+, q2_t, q2_W-, q2_tbar) of the free components f = (nu_x, nu_y, nu_z,
    nubar_z), the antineutrino's transverse momentum being MET - nu_T."""
    n1 = np.array([0.0, f[0], f[1], f[2]])
    n1[0] = np.linalg.norm(n1[1:])
    n2 = np.array([0.0, met[0] - f[0], met[1] - f[1], f[3]])
    n2[0] = np.linalg.norm(n2[1:])
    q = virtualities(b, bb, lp, lm, n1, n2)
    return np.array([q[0], q[2], q[1], q[3]])


def test_jacobian_by_finite_differences(ora, truth):
    """Every solution's Jacobian against central differences of the forward map
    (the virtualities as functions of the free neutrino components), which does
    not involve the solver."""
    checked = 0
    for ev in truth[:16]:
        b, bb, lp, lm, nu, nub = ev
        met = (nu + nub)[1:3]
        for n1, n2, jac in ora.dilep_nu(b, bb, lp, lm, met, *virtualities(b, bb, lp, lm, nu, nub)):
            f0 = np.array([n1[1], n1[2], n1[3], n2[3]])
            M = np.zeros((4, 4))
            for j in range(4):
                h = 1e-4 * max(1.0, abs(f0[j]))
                fp, fm = f0.copy(), f0.copy()
                fp[j] += h
                fm[j] -= h
                M[:, j] = (_forward(b, bb, lp, lm, met, fp) - _forward(b, bb, lp, lm, met, fm)) / (2 * h)
            # central differences: O(h^2) ~ 1e-8 truncation per entry
            assert abs(np.linalg.det(M)) * jac == pytest.approx(1.0, rel=1e-5, abs=0)
            checked += 1
    assert checked >= 32


def test_change_of_variables_integral(ora, truth):
    """Importance sampling of the virtualities through the forward map: draw the free
    neutrino components nu' from a normal density phi (width 1.5 sigma), map them to
    q^2; the density of q^2 is then sum over all preimages of phi J, which are the
    solver's solutions (nu' must be one of them). The mean of
    sum_sol f J / sum_sol phi J estimates the integral of sum_sol f J over q^2,
    which must equal the integral of f over the neutrino components."""
    b, bb, lp, lm, nu, nub = truth[3]
    met = (nu + nub)[1:3]
    sigma, sw = 8.0, 12.0
    centre = np.array([nu[1], nu[2], nu[3], nub[3]])
    rng = np.random.default_rng(11)
    n = 4000
    vals = np.zeros(n)
    for i in range(n):
        f1 = centre + sw * rng.standard_normal(4)
        q = _forward(b, bb, lp, lm, met, f1)          # (W+, t, W-, tbar)
        sols = ora.dilep_nu(b, bb, lp, lm, met, q[0], q[2], q[1], q[3])
        frees = [np.array([s1[1], s1[2], s1[3], s2[3]]) for s1, s2, _ in sols]
        assert min(np.max(np.abs(fr - f1)) for fr in frees) < 1e-6 * (1 + np.max(np.abs(f1)))
        num = den = 0.0
        for fr, (_, _, jac) in zip(frees, sols):
            d2 = float((fr - centre) @ (fr - centre))
            num += math.exp(-0.5 * d2 / sigma ** 2) * jac
            den += math.exp(-0.5 * d2 / sw ** 2) / ((2 * math.pi) ** 2 * sw ** 4) * jac
        vals[i] = num / den
    est, err = vals.mean(), vals.std() / math.sqrt(n)
    want = (2 * math.pi * sigma ** 2) ** 2
    assert err < 0.02 * want
    assert abs(est - want) < 4 * err

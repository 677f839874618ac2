"""Pins of the oracle's event discriminant (Sec. 3: D = log10(p_S / p_B), the
quantity whose distribution the paper shows for signal and background).

* Closed forms: D(p, p) = 0, D(10 p, p) = 1, antisymmetry under S <-> B.
* The error is the first-order propagation of the two estimates' errors: it
  matches the spread of log10(p_S / p_B) over Gaussian fluctuations of p_S, p_B
  with small relative errors.
* Non-positive densities give NaN and a non-zero status.
* On integrals: Drell-Yan events favour the Z mass they were generated with
  over one 10 GeV heavier.
"""
import math

import numpy as np
import pytest


def test_closed_forms(ora):
    assert ora.discriminant(3.0e-20, 1e-22, 3.0e-20, 1e-22)[0] == 0.0
    assert ora.discriminant(5.0e-19, 0, 5.0e-20, 0)[0] == pytest.approx(1.0, rel=1e-15, abs=0)
    a = ora.discriminant(2.0e-30, 1e-32, 7.0e-31, 3e-33)
    b = ora.discriminant(7.0e-31, 3e-33, 2.0e-30, 1e-32)
    assert a[0] == pytest.approx(-b[0], rel=1e-15, abs=0) and a[1] == b[1]
    assert a[0] == pytest.approx(math.log10(2.0 / 0.7), rel=1e-15, abs=0)


def test_error_propagation(ora):
    rng = np.random.default_rng(3)
    ps, es, pb, eb = 4.0e-25, 4.0e-28, 1.5e-25, 3.0e-28     # 0.1 % and 0.2 %
    D, err, rc = ora.discriminant(ps, es, pb, eb)
    samples = np.log10(rng.normal(ps, es, 200000) / rng.normal(pb, eb, 200000))
    assert rc == 0
    assert np.std(samples) == pytest.approx(err, rel=0.01, abs=0)
    assert abs(np.mean(samples) - D) < 5 * err / math.sqrt(200000) + 1e-7


def test_nonpositive(ora):
    for ps, pb in [(0.0, 1.0), (1.0, 0.0), (-1.0, 1.0)]:
        D, e, rc = ora.discriminant(ps, 0.1, pb, 0.1)
        assert rc == 1 and math.isnan(D) and math.isnan(e)


def test_mass_hypotheses(ora, synth):
    """Drell-Yan events generated on the Z peak (m_Z = 91.19 GeV) favour it over a
    hypothesis with the Z 10 GeV heavier: D > 0 on most events, and the sum of D
    (the log-likelihood ratio of the sample) is large."""
    recs = synth.gen_dy(12, 77)
    T = ora.tf(synth.DEFAULT_TF[0])
    Ps = ora.process(0, synth.DEFAULT_PROCESS)
    Pb = ora.process(0, dict(synth.DEFAULT_PROCESS, mz=101.19))
    rs = ora.integrate(Ps, T, recs, seed=1, n_points=1 << 13)
    rb = ora.integrate(Pb, T, recs, seed=1, n_points=1 << 13)
    D = np.array([ora.discriminant(a, b, c, d)[0]
                  for a, b, c, d in zip(rs["prob"], rs["err"], rb["prob"], rb["err"])])
    assert np.mean(D > 0) >= 0.75
    assert D.sum() > 5.0

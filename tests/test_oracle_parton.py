"""Pins of the oracle's parton-level ttbar weight (Sec. 4, parton level: delta
transfer functions for every final-state particle, averaged over the b-quark
assignments).

* x1, x2 and s-hat against their closed forms from the event's total momentum
  (a transverse boost keeps p_z and the invariant mass).
* The generator-truth b assignment carries the larger weight in almost every
  event (the wrong one puts both tops off their Breit-Wigner peaks).
* Invariance under a common azimuthal rotation; relabelling the two b-quark
  objects swaps the two assignment weights and leaves their mean unchanged.
* With flat parton densities, w x prod_i 2 E_i is invariant under a common
  longitudinal boost (x1 x2 s, the flux 1/(|q1||q2|) and |M|^2 are invariant).
* Consistency with the hadron-level integrand: at a point of the ttbar
  integral, the integrand equals, summed over the neutrino roots, the parton
  weight of the mapped final state times the transfer functions, the map
  Jacobian and the jets' E^2 sin(theta) measure factors.
"""
import math

import numpy as np
import pytest


def _mom(rec):
    """(6, 4) lab four-momenta (E, px, py, pz) of the six massless objects, FP64."""
    E = rec[0:24:4].astype(float)
    eta = rec[1:24:4].astype(float)
    phi = rec[2:24:4].astype(float)
    pt = E / np.cosh(eta)
    return np.stack([E, pt * np.cos(phi), pt * np.sin(phi), E * np.tanh(eta)], axis=1)


def _record(p_list, kinds):
    """Parton-level record from FP64 four-momenta (E, px, py, pz)."""
    r = np.zeros(32, dtype=np.float32)
    for o, (p, k) in enumerate(zip(p_list, kinds)):
        pt = math.hypot(p[1], p[2])
        r[4 * o: 4 * o + 4] = (p[0], math.asinh(p[3] / pt), math.atan2(p[2], p[1]), k)
    r[24], r[25] = p_list[5][1], p_list[5][2]
    r[26], r[27], r[29] = 6, 2, 1
    return r


@pytest.fixture(scope="module")
def events(synth):
    return synth.gen_ttbar_parton(64, 901)


def test_momentum_fractions_closed_form(ora, synth, events):
    P = ora.process(2, synth.DEFAULT_PROCESS)
    rs = synth.SQRT_S
    for rec in events[:16]:
        tot = _mom(rec).sum(axis=0)
        m2 = tot[0] ** 2 - tot[1] ** 2 - tot[2] ** 2 - tot[3] ** 2
        ep = math.sqrt(m2 + tot[3] ** 2)
        for a in (0, 1):
            _, aux = ora.parton_ttbar(P, rec, a)
            assert aux[0] == pytest.approx((ep + tot[3]) / rs, rel=1e-10, abs=0)
            assert aux[1] == pytest.approx((ep - tot[3]) / rs, rel=1e-10, abs=0)
            assert aux[2] == pytest.approx(m2, rel=1e-10, abs=0)


def test_truth_assignment_dominates(ora, synth, events):
    P = ora.process(2, synth.DEFAULT_PROCESS)
    prob, w = ora.parton_batch(P, events, n_threads=4)
    truth = events[:, 28].astype(int)
    idx = np.arange(len(events))
    assert np.mean(w[idx, truth] > 100.0 * w[idx, 1 - truth]) > 0.95
    assert np.allclose(prob, 0.5 * w.sum(axis=1), rtol=1e-15, atol=0)
    assert np.all(prob > 0)


def test_azimuthal_rotation(ora, synth, events):
    P = ora.process(2, synth.DEFAULT_PROCESS)
    for rec in events[:8]:
        r2 = _record([_rot(p, 0.7) for p in _mom(rec)], rec[3:24:4])
        for a in (0, 1):
            w1, _ = ora.parton_ttbar(P, rec, a)
            w2, _ = ora.parton_ttbar(P, r2, a)
            assert w2 == pytest.approx(w1, rel=2e-4, abs=0)


def _rot(p, a):
    c, s = math.cos(a), math.sin(a)
    return np.array([p[0], c * p[1] - s * p[2], s * p[1] + c * p[2], p[3]])


def test_bquark_relabelling(ora, synth, events):
    P = ora.process(2, synth.DEFAULT_PROCESS)
    for rec in events[:8]:
        sw = rec.copy()
        sw[4:8], sw[8:12] = rec[8:12], rec[4:8]
        w0, _ = ora.parton_ttbar(P, rec, 0)
        w1, _ = ora.parton_ttbar(P, rec, 1)
        assert ora.parton_ttbar(P, sw, 0)[0] == w1
        assert ora.parton_ttbar(P, sw, 1)[0] == w0


def test_longitudinal_boost_with_flat_densities(ora, synth, events):
    flat = dict(synth.DEFAULT_PROCESS, pdf_A=(1.0, 1.0, 1.0), pdf_a=(0.0, 0.0, 0.0),
                pdf_b=(0.0, 0.0, 0.0))
    P = ora.process(2, flat)
    for rec in events[:8]:
        for dy in (-0.4, 0.3):
            moms = _mom(rec)
            ch, sh = math.cosh(dy), math.sinh(dy)
            boosted = [np.array([ch * p[0] + sh * p[3], p[1], p[2], sh * p[0] + ch * p[3]])
                       for p in moms]
            r2 = _record(boosted, rec[3:24:4])
            e1 = np.prod(2.0 * rec[0:24:4].astype(float))
            e2 = np.prod(2.0 * r2[0:24:4].astype(float))
            for a in (0, 1):
                w1, x1 = ora.parton_ttbar(P, rec, a)
                w2, x2 = ora.parton_ttbar(P, r2, a)
                assert x2[0] == pytest.approx(x1[0] * math.exp(dy), rel=1e-5, abs=0)
                assert w2 * e2 == pytest.approx(w1 * e1, rel=2e-4, abs=0)


def test_consistent_with_hadron_level_integrand(ora, synth):
    P = ora.process(2, synth.DEFAULT_PROCESS)
    T = ora.tf(synth.DEFAULT_TF[2])
    recs = synth.gen_ttbar(4, 77)
    rng = np.random.default_rng(5)
    checked = 0
    for rec in recs:
        perm = int(rec[28])
        for _ in range(6):
            x = rng.uniform(0.05, 0.95, 7)
            total = ora.integrand(P, T, rec, perm, x)
            acc = 0.0
            n = ora.kinematics(P, T, rec, perm, x, 0)["n"]
            for root in range(n):
                k = ora.kinematics(P, T, rec, perm, x, root)
                b, l, nu, bb, d, u = k["lab"]
                r2 = _record([l, b, bb, d, u, nu], [4, 5, 5, 5, 5, 6])
                w, aux = ora.parton_ttbar(P, r2, 0)
                jets = r2[4:20].reshape(4, 4)
                meas = np.prod(jets[:, 0].astype(float) ** 2 / np.cosh(jets[:, 1].astype(float)))
                acc += w * meas * k["aux"][6] * k["aux"][7]
            if total > 0:
                assert acc == pytest.approx(total, rel=2e-4, abs=0)
                checked += 1
    assert checked >= 12

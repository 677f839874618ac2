"""Pins of the oracle's change of variables (Sec. 3: propagator virtualities as
integration variables; neutrino from the W mass constraint; jets with
E^2 sin(theta) dE) and of its transfer-function normalisation (Sec. 1).

* Momentum conservation q1 + q2 = sum of final-state momenta at every point.
* Every virtuality that the map sets (W, top, antitop masses) is the invariant
  mass of the momenta it produces.
* The Jacobian the oracle multiplies in equals |det d(physical variables)/dx|
  computed by central finite differences of the map itself.
* Parton-level limit (Sec. 4, first analysis level: delta-function TFs): with
  a vanishing lepton resolution the Drell-Yan integral approaches the
  delta-TF evaluation at the measured momenta as O(r^2). This restates the
  density's prefactor, so it checks the limit only; the prefactor itself is
  pinned in test_oracle_normalisation.py.
"""
import math

import numpy as np
import pytest


def dot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


@pytest.fixture(scope="module")
def events(synth):
    return {0: synth.gen_dy(4, 11), 1: synth.gen_w(4, 12), 2: synth.gen_ttbar(3, 13)}


def _setup(ora, synth, kind, tf_over=None):
    tf = dict(synth.DEFAULT_TF[kind])
    if tf_over:
        tf.update(tf_over)
    return ora.process(kind, synth.DEFAULT_PROCESS), ora.tf(tf)


def physical_vars(kind, lab):
    """Integration variables in the lab frame, in map order."""
    if kind == 0:
        return np.array([lab[0][0], lab[1][0]])
    if kind == 1:
        return np.array([lab[0][0], lab[1][1], lab[1][2], lab[1][3]])
    # ttbar lab order: b, l+, nu, bbar, d, ubar
    return np.array([lab[4][0], lab[5][0], lab[3][0], lab[2][1], lab[2][2], lab[2][3], lab[0][0]])


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_conservation_and_masses(ora, synth, events, kind):
    P, T = _setup(ora, synth, kind)
    d = ora.dims(kind)
    rng = np.random.default_rng(20 + kind)
    checked = 0
    for rec in events[kind]:
        for _ in range(40):
            x = rng.uniform(0.02, 0.98, size=d)
            perm = int(rng.integers(0, ora.nperm(kind)))
            k = ora.kinematics(P, T, rec, perm, x, 0)
            for r in range(k["n"]):
                k = ora.kinematics(P, T, rec, perm, x, r)
                fs, k12, aux = k["fs"], k["k12"], k["aux"]
                nfs = 2 if kind < 2 else 6
                tot = fs[:nfs].sum(axis=0)
                scale = tot[0]
                assert np.allclose(k12[0] + k12[1], tot, rtol=0, atol=1e-12 * scale)
                assert abs(tot[1]) < 1e-12 * scale and abs(tot[2]) < 1e-12 * scale
                for p in fs[:nfs]:  # massless final state
                    assert abs(dot(p, p)) < 1e-10 * p[0] ** 2
                if kind == 1:
                    w = fs[0] + fs[1]
                    assert dot(w, w) == pytest.approx(aux[0], rel=1e-10, abs=0)
                if kind == 2:
                    b, l, n, bb, dq, ub = fs[:6]
                    assert dot(dq + ub, dq + ub) == pytest.approx(aux[0], rel=1e-10, abs=0)
                    assert dot(bb + dq + ub, bb + dq + ub) == pytest.approx(aux[1], rel=1e-10, abs=0)
                    assert dot(l + n, l + n) == pytest.approx(aux[2], rel=1e-10, abs=0)
                    assert dot(b + l + n, b + l + n) == pytest.approx(aux[3], rel=1e-10, abs=0)
                checked += 1
    assert checked > 50


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_jacobian_is_determinant_of_the_map(ora, synth, events, kind):
    P, T = _setup(ora, synth, kind)
    d = ora.dims(kind)
    rng = np.random.default_rng(30 + kind)
    n_ok = 0
    for rec in events[kind]:
        for _ in range(12):
            x = rng.uniform(0.05, 0.95, size=d)
            perm = int(rng.integers(0, ora.nperm(kind)))
            k0 = ora.kinematics(P, T, rec, perm, x, 0)
            for r in range(k0["n"]):
                k = ora.kinematics(P, T, rec, perm, x, r)
                jac = k["aux"][6]
                M = np.zeros((d, d))
                ok = True
                for j in range(d):
                    h = 1e-6
                    xp, xm = x.copy(), x.copy()
                    xp[j] += h
                    xm[j] -= h
                    kp = ora.kinematics(P, T, rec, perm, xp, r)
                    km = ora.kinematics(P, T, rec, perm, xm, r)
                    if kp["n"] != k0["n"] or km["n"] != k0["n"]:
                        ok = False
                        break
                    M[:, j] = (physical_vars(kind, kp["lab"]) - physical_vars(kind, km["lab"])) / (2 * h)
                if not ok:
                    continue
                assert abs(np.linalg.det(M)) == pytest.approx(jac, rel=2e-5, abs=0)
                n_ok += 1
    assert n_ok >= 10


def test_parton_level_limit_dy(ora, synth, events):
    """Vanishing resolution: int f dx -> the delta-TF evaluation at the measured
    momenta, times the Gaussian mass inside the +-5 sigma window per lepton. At
    relative resolution r the deviation is O(r^2) (the resonance is smeared over
    sigma_q2 ~ r m^2): it must shrink fourfold when r halves, and the Richardson
    extrapolation to r = 0 must vanish."""
    p = synth.DEFAULT_PROCESS
    s = p["sqrt_s"] ** 2
    xg, wg = np.polynomial.legendre.leggauss(48)
    xg = 0.5 * (xg + 1)
    wg = 0.5 * wg
    for rec in events[0][:2]:
        # delta-TF value at the measured momenta
        mom = []
        meas = 1.0
        for o in range(2):
            E, eta, phi = (float(v) for v in rec[4 * o: 4 * o + 3])
            n = np.array([math.cos(phi) / math.cosh(eta), math.sin(phi) / math.cosh(eta), math.tanh(eta)])
            mom.append(np.array([E, *(E * n)]))
            meas *= E * E / math.cosh(eta) / ((2 * math.pi) ** 3 * 2 * E)
        tot = mom[0] + mom[1]
        M2 = dot(tot, tot)
        Ep = math.sqrt(M2 + tot[3] ** 2)      # energy after the transverse boost
        x1, x2 = (Ep + tot[3]) / p["sqrt_s"], (Ep - tot[3]) / p["sqrt_s"]
        # boosted lepton momenta: boost with velocity (px/E, py/E, 0)
        bx, by = tot[1] / tot[0], tot[2] / tot[0]
        g = 1 / math.sqrt(1 - bx * bx - by * by)

        def bst(q):
            bp = bx * q[1] + by * q[2]
            c = (g - 1) * bp / (bx * bx + by * by) - g * q[0]
            return np.array([g * (q[0] - bp), q[1] + c * bx, q[2] + c * by, q[3]])
        lm, lp = bst(mom[0]), bst(mom[1])
        rs = p["sqrt_s"]
        k1 = np.array([x1 * rs / 2, 0, 0, x1 * rs / 2])
        k2 = np.array([x2 * rs / 2, 0, 0, -x2 * rs / 2])
        P0, _ = _setup(ora, synth, 0)
        fsum = 0.0
        for fl in (0, 1):
            fsum += ora.pdf(P0, 0, x1) * ora.pdf(P0, 1, x2) * ora.msq_dy(P0, fl, k1, k2, lm, lp)
            fsum += ora.pdf(P0, 1, x1) * ora.pdf(P0, 0, x2) * ora.msq_dy(P0, fl, k2, k1, lm, lp)
        want = fsum / (k1[0] * k2[0]) * (2 * math.pi) ** 4 * (2 / s) * meas
        window = math.erf(5 / math.sqrt(2)) ** 2
        dev = []
        for r in (2e-4, 1e-4):
            P, T = _setup(ora, synth, 0, {"lep_rel": r})
            quad = sum(wa * wb * ora.integrand(P, T, rec, 0, [a, b])
                       for a, wa in zip(xg, wg) for b, wb in zip(xg, wg))
            dev.append(quad / (want * window) - 1.0)
        assert abs(dev[1]) < 1e-4
        assert 3.0 < dev[0] / dev[1] < 5.0
        assert abs((4.0 * dev[1] - dev[0]) / 3.0) < 2e-6

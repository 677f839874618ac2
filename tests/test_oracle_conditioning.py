"""The oracle's measure of a point's conditioning, which the dilepton GPU parity rules
(parity_rules.check_conditioned) turn into per-point tolerances: s = sum over the
unit-cube coordinates of |w(u + 2^-24 e_k) / w(u) - 1|.

* Where the maps are smooth (W -> e nu) s is small: the weight's logarithmic
  derivative times 2^-24, a few 1e-6.
* Next to a neutrino branch point of the dilepton system (Sec. 3, Eq. "dilepsolv"),
  where two solutions merge at distance delta (in a unit-cube coordinate), the
  Jacobian 1/|det| grows like delta^-1/2, so d ln w / du ~ 1 / (2 delta) and s grows like
  1 / delta: s delta stays constant as the branch point is approached (measured from
  delta = 1e-3 to 1e-5), at about 2^-24 / 2.
"""
import numpy as np
import pytest

from parity_rules import sensitivity


@pytest.fixture(scope="module")
def env():
    from oracle import oracle as O
    from paper_1407_7595_gb300 import synth
    return O, synth


def test_smooth_maps_are_well_conditioned(env):
    O, synth = env
    kind = 1
    recs = synth.gen_events(kind, 2, 901)
    P = O.process(kind, synth.DEFAULT_PROCESS)
    T = O.tf(synth.DEFAULT_TF[kind])
    ss = []
    for e in range(2):
        w = O.eval_points(P, T, recs[e], e, 0, 5, 0, 256)
        for i in np.flatnonzero(w)[:60]:
            ss.append(sensitivity(O, P, T, recs[e], e, 0, 5, int(i), 4))
    assert len(ss) >= 100
    assert max(ss) < 2e-5


def _weight_sensitivity(O, P, T, rec, perm, v):
    w0 = O.integrand(P, T, rec, perm, v)
    assert w0 != 0
    s = 0.0
    for k in range(len(v)):
        vv = v.copy()
        vv[k] += 2.0 ** -24 if v[k] < 0.5 else -(2.0 ** -24)
        s += abs(O.integrand(P, T, rec, perm, vv) / w0 - 1.0)
    return s


def test_conditioning_diverges_at_a_neutrino_branch_point(env):
    O, synth = env
    kind = 3
    recs = synth.gen_events(kind, 4, 7100)
    P = O.process(kind, synth.DEFAULT_PROCESS)
    T = O.tf(synth.DEFAULT_TF[kind])
    rng = np.random.default_rng(4)
    found = 0
    for _ in range(200):
        e, perm = int(rng.integers(0, 4)), int(rng.integers(0, 2))
        u = rng.uniform(0.05, 0.95, 6)

        def nsol(t):
            v = u.copy()
            v[4] = t   # the top virtuality's coordinate
            return O.kinematics(P, T, recs[e], perm, v, 0)["n"]

        ts = np.linspace(0.01, 0.99, 60)
        ns = [nsol(t) for t in ts]
        for a, b, na, nb in zip(ts[:-1], ts[1:], ns[:-1], ns[1:]):
            if na == nb or max(na, nb) == 0:
                continue
            lo, hi = a, b
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                if nsol(mid) == na:
                    lo = mid
                else:
                    hi = mid
            side, sgn = (lo, -1.0) if na > nb else (hi, 1.0)   # the side with the solutions
            s = []
            for dist in (1e-3, 1e-5):
                v = u.copy()
                v[4] = side + sgn * dist
                s.append(_weight_sensitivity(O, P, T, recs[e], perm, v))
            # s ~ 1 / delta: a hundredfold from delta = 1e-3 to 1e-5
            assert 30.0 < s[1] / s[0] < 300.0, s
            # and s delta ~ 2^-24 / 2 (within the spread of the other coordinates' terms)
            assert 0.3 * 3e-8 < s[1] * 1e-5 < 30.0 * 3e-8, s
            found += 1
            break
        if found >= 3:
            break
    assert found >= 3

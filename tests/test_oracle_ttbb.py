"""Pins of the oracle's g g / q qbar -> t tbar b bbar amplitude (the ttbb background of
Sec. 3-4), written diagram by diagram from the QCD Feynman rules with explicit colour
sums.

* SU(3): the generators give C_F = 4/3, C_A = 3, Tr(t^a t^b) = delta/2, and the
  colour sums 16/3 and -2/3 of the two orderings t^a t^b, t^b t^a (the numbers the
  semileptonic ttbar amplitude uses).
* Gauge invariance (g g): replacing one gluon's polarisation by its momentum, the other
  gluon physical, the colour- and spin-summed square vanishes -- to 1e-7 of the physical
  value, where flipping the sign of any one diagram class gives O(1e4) (checked by hand
  when the pin was written); this fixes the relative signs and factors of the 36 diagrams
  and their colour tensors.
* Current conservation (q qbar): the g* -> t tbar b bbar part contracted with the g*
  momentum vanishes.
* Bose symmetry (g g) and Lorentz invariance (a boost along and a rotation about the
  beam axis, which keep the transverse gluon polarisations valid).
"""
import math

import numpy as np
import pytest

from test_oracle_tth import _boost, _two_body


def dot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def _kinematics(rng, rs, m):
    k1, k2 = np.array([rs / 2, 0, 0, rs / 2]), np.array([rs / 2, 0, 0, -rs / 2])
    M1 = rng.uniform(2 * m + 10, rs - 60)
    M2 = rng.uniform(20, rs - M1 - 5)
    A, B = _two_body(rng, rs, M1, M2)
    t, tb = _two_body(rng, M1, m, m)
    b, bb = _two_body(rng, M2, 0.0, 0.0)
    bA, bB = A[1:] / A[0], B[1:] / B[0]
    return k1, k2, _boost(t, bA), _boost(tb, bA), _boost(b, bB), _boost(bb, bB)


@pytest.fixture(scope="module")
def P(ora, synth):
    return ora.process(2, synth.DEFAULT_PROCESS)


def test_su3(ora):
    s_ab, s_ba, cf, ca, tr_dev = ora.su3_check()
    assert s_ab == pytest.approx(16 / 3, rel=1e-14, abs=0)
    assert s_ba == pytest.approx(-2 / 3, rel=1e-13, abs=0)
    assert cf == pytest.approx(4 / 3, rel=1e-14, abs=0)
    assert ca == pytest.approx(3.0, rel=1e-14, abs=0)
    assert tr_dev < 1e-15


def test_ttbb_gauge_invariance(ora, synth, P):
    m = synth.DEFAULT_PROCESS["mt"]
    rng = np.random.default_rng(61)
    for rs in (700.0, 1500.0, 3000.0):
        k1, k2, p1, p2, p3, p4 = _kinematics(rng, rs, m)
        assert np.allclose(k1 + k2, p1 + p2 + p3 + p4, rtol=0, atol=1e-10 * rs)
        ref = ora.msq_ttbb_production(P, 0, k1, k2, p1, p2, p3, p4) * 256
        assert ref > 0
        for which in (0, 1):
            for hel in (0, 1):
                assert abs(ora.ttbb_gauge_probe(P, k1, k2, p1, p2, p3, p4, which, hel)) < 1e-7 * ref


def test_ttbb_qq_current_conservation(ora, synth, P):
    m = synth.DEFAULT_PROCESS["mt"]
    rng = np.random.default_rng(62)
    for rs in (700.0, 2000.0):
        k1, k2, p1, p2, p3, p4 = _kinematics(rng, rs, m)
        ward, scale = ora.ttbb_qq_ward_probe(P, k1, k2, p1, p2, p3, p4)
        assert scale > 0 and abs(ward) < 1e-12 * scale


def test_ttbb_bose_and_lorentz(ora, synth, P):
    m = synth.DEFAULT_PROCESS["mt"]
    rng = np.random.default_rng(63)
    for _ in range(2):
        k1, k2, p1, p2, p3, p4 = _kinematics(rng, 1200.0, m)
        for channel in (0, 1):
            ref = ora.msq_ttbb_production(P, channel, k1, k2, p1, p2, p3, p4)
            assert ref > 0
            if channel == 0:
                assert ora.msq_ttbb_production(P, 0, k2, k1, p1, p2, p3, p4) == pytest.approx(ref, rel=1e-11, abs=0)
            bz = np.array([0.0, 0.0, rng.uniform(-0.7, 0.7)])
            a = rng.uniform(0, 2 * math.pi)
            R = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])

            def tr(p):
                q = _boost(p, bz)
                return np.array([q[0], *(R @ q[1:])])
            got = ora.msq_ttbb_production(P, channel, *[tr(v) for v in (k1, k2, p1, p2, p3, p4)])
            assert got == pytest.approx(ref, rel=1e-9, abs=0)


def _decay3(rng, M, m12):
    a, w = _two_body(rng, M, 0.0, m12)
    b, c = _two_body(rng, m12, 0.0, 0.0)
    beta = w[1:] / w[0]
    return a, _boost(b, beta), _boost(c, beta)


@pytest.mark.parametrize("channel", [0, 1])
def test_ttbb_full_chain_factorises(ora, synth, P, channel):
    """With on-shell tops the full 2 -> 8 |M|^2 (t and W propagator denominators
    removed), averaged over parity-reflected decays in each top rest frame, equals
    |M|^2(ttbb production, top spins summed) x (g_W^2/2)^4 c_t c_tbar, c_t = 8 (p_t.p_l+)
    (p_b.p_nu), c_tbar = 8 (p_tbar.p_mu-)(p_bbar.p_nubar) (the reflection removes the
    top-spin correlations; the W- decays to one lepton channel)."""
    prm = synth.DEFAULT_PROCESS
    m, mw, ww, wt = prm["mt"], prm["mw"], prm["ww"], prm["wt"]
    gw2 = 4 * math.pi * prm["alpha"] / prm["sw2"]
    rng = np.random.default_rng(64 + channel)
    k1, k2, pt, ptb, p3, p4 = _kinematics(rng, 900.0, m)
    b0, l0, n0 = _decay3(rng, m, 79.0)
    bb0, m0, nb0 = _decay3(rng, m, 82.0)
    acc = 0.0
    for par_t in (1, -1):
        for par_tb in (1, -1):
            bt, btb = pt[1:] / pt[0], ptb[1:] / ptb[0]
            pb, pl, pn = (_boost(np.array([v[0], *(par_t * v[1:])]), bt) for v in (b0, l0, n0))
            pbb, pm, pnb = (_boost(np.array([v[0], *(par_tb * v[1:])]), btb) for v in (bb0, m0, nb0))
            w1, w2 = pl + pn, pm + pnb
            dens = (wt * m) ** 4 * ((dot(w1, w1) - mw * mw) ** 2 + (mw * ww) ** 2) * \
                ((dot(w2, w2) - mw * mw) ** 2 + (mw * ww) ** 2)
            acc += ora.msq_ttbb(P, channel, k1, k2, pb, pl, pn, pbb, pm, pnb, p3, p4) * dens
            ct = 8 * dot(pt, pl) * dot(pb, pn)
            ctb = 8 * dot(ptb, pm) * dot(pbb, pnb)
    prod = ora.msq_ttbb_production(P, channel, k1, k2, pt, ptb, p3, p4)
    assert acc / 4 == pytest.approx(prod * (gw2 / 2) ** 4 * ct * ctb, rel=1e-9, abs=0)


# ---------------------------------------------------------------------------
# The dilepton ttbb integrand (process kind 5): the variables of dilepton ttH with the
# extra b bbar pair in the Higgs pair's place and its mass mapped log-uniformly.
# ---------------------------------------------------------------------------
from test_oracle_tth import _phys8, _states, _find_point, _which_object  # noqa: E402

KIND_TTBB = 5


@pytest.fixture(scope="module")
def ttbb_setup(ora, synth):
    recs = synth.gen_tth_dilep(3, 97).copy()
    recs[:, 27] = KIND_TTBB     # two leptons and four b jets: the same record layout
    return (ora.process(KIND_TTBB, synth.DEFAULT_PROCESS), ora.tf(synth.DEFAULT_TF[4]), recs)


def test_ttbb_integrand_map(ora, synth, ttbb_setup):
    """8 variables, 12 assignments; at every state momentum conservation, zero total
    pT, the virtualities of the produced momenta, and the full map's Jacobian against
    central differences in (E_b, E_bbar, nu, nubar_z, E_b1, E_b2)."""
    P, T, recs = ttbb_setup
    assert ora.dims(KIND_TTBB) == 8 and ora.nperm(KIND_TTBB) == 12
    rng = np.random.default_rng(65)
    n_ok = 0
    for rec in recs:
        for _ in range(80):
            x = rng.uniform(0.05, 0.95, size=8)
            perm = int(rng.integers(0, 12))
            for k in _states(ora, P, T, rec, perm, x):
                fs, lab, k12, aux = k["fs"], k["lab"], k["k12"], k["aux"]
                tot = fs.sum(axis=0)
                assert np.allclose(k12[0] + k12[1], tot, rtol=0, atol=1e-12 * tot[0])
                ltot = lab.sum(axis=0)
                assert abs(ltot[1]) < 1e-10 * ltot[0] and abs(ltot[2]) < 1e-10 * ltot[0]
                b, lp, nu, bb, lm, nub, h1, h2 = lab
                want = (dot(lp + nu, lp + nu), dot(lm + nub, lm + nub),
                        dot(b + lp + nu, b + lp + nu), dot(bb + lm + nub, bb + lm + nub))
                for g, w in zip(aux[:4], want):
                    assert g == pytest.approx(w, rel=1e-9, abs=0)
                f0 = _phys8(lab)
                M = np.zeros((8, 8))
                ok = True
                for j in range(8):
                    cols = []
                    for sgn in (1, -1):
                        xs = x.copy()
                        xs[j] += sgn * 1e-6
                        cand = [_phys8(q["lab"]) for q in _states(ora, P, T, rec, perm, xs)]
                        if not cand:
                            ok = False
                            break
                        d = sorted((np.max(np.abs(c - f0)), i) for i, c in enumerate(cand))
                        if len(d) > 1 and d[1][0] < 10 * d[0][0]:
                            ok = False
                            break
                        cols.append(cand[d[0][1]])
                    if not ok:
                        break
                    M[:, j] = (cols[0] - cols[1]) / 2e-6
                if ok:
                    assert abs(np.linalg.det(M)) == pytest.approx(aux[6], rel=2e-5, abs=0)
                    n_ok += 1
    assert n_ok >= 5


def test_ttbb_flavour_sum_both_pair_orientations(ora, synth, ttbb_setup):
    """The extra pair's two jets enter as (b, bbar) and as (bbar, b): the flavour-summed
    |M|^2 at a state equals the sum over both orientations of the ttbb amplitudes."""
    P, T, recs = ttbb_setup
    rng = np.random.default_rng(66)
    rec = recs[0]
    x = _find_point(ora, P, T, rec, 0, rng)
    assert x is not None
    k = _states(ora, P, T, rec, 0, x)[0]
    fs, k12 = k["fs"], k["k12"]
    x1, x2 = k["aux"][4], k["aux"][5]
    got = ora.flavour_msq(P, fs, k12, x1, x2, rec)
    Q = math.sqrt(x1 * x2) * synth.DEFAULT_PROCESS["sqrt_s"]
    f = {t: (ora.pdf_q(P, t, x1, Q), ora.pdf_q(P, t, x2, Q)) for t in (0, 1, 2)}
    want = 0.0
    for a, bq in ((fs[6], fs[7]), (fs[7], fs[6])):
        mom = (fs[0], fs[1], fs[2], fs[3], fs[4], fs[5], a, bq)
        want += f[2][0] * f[2][1] * ora.msq_ttbb(P, 0, k12[0], k12[1], *mom)
        want += 2 * f[0][0] * f[1][1] * ora.msq_ttbb(P, 1, k12[0], k12[1], *mom)
        want += 2 * f[1][0] * f[0][1] * ora.msq_ttbb(P, 1, k12[1], k12[0], *mom)
    assert got == pytest.approx(want, rel=1e-12, abs=0)



def test_ttbb_pair_exchange_symmetry_with_massless_tops(ora, synth):
    """With m_t = 0 the two quark pairs differ only by their labels: |M|^2 is symmetric
    under exchanging (t, tbar) with (b, bbar), in both channels. This ties the top-line
    diagrams to the b-line ones (classes A/B, the two halves of D and E) and the two
    orders of the pair gluons on the light line."""
    P = ora.process(2, dict(synth.DEFAULT_PROCESS, mt=0.0))
    rng = np.random.default_rng(67)
    for rs in (500.0, 1500.0):
        k1, k2, p1, p2, p3, p4 = _kinematics(rng, rs, 0.0)
        for channel in (0, 1):
            a = ora.msq_ttbb_production(P, channel, k1, k2, p1, p2, p3, p4)
            b = ora.msq_ttbb_production(P, channel, k1, k2, p3, p4, p1, p2)
            assert a > 0 and b == pytest.approx(a, rel=1e-12, abs=0)

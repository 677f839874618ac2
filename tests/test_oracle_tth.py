"""Pins of the oracle's g g / q qbar -> t tbar H production amplitude (Sec. 3's
signal process; the Higgs-top Yukawa y_t = m_t / v).

* Gauge invariance: each colour-ordered g g amplitude vanishes when one gluon's
  polarisation is replaced by its momentum (the other gluon physical).
* Soft-Higgs limit: as the Higgs momentum goes to zero, |M(ttH)|^2 ->
  y_t^2 m_t^2 (1/(p_t.p_H) + 1/(p_tbar.p_H))^2 |M(tt)|^2 -- the scalar emission off the
  two external top lines, whose numerators reduce to 2 m_t (u-bar(p)(p/ + m) =
  2 m u-bar(p)); the deviation is O(p_H), so it shrinks tenfold when p_H does. This
  fixes the Higgs vertex, its placement in every diagram and the relative sign of
  the emissions off the top and the antitop.
* Bose symmetry (g g: exchanging the gluons) and Lorentz invariance (a boost along
  and a rotation about the beam axis, which keep the gluon polarisations valid).
"""
import math

import numpy as np
import pytest


def dot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


@pytest.fixture(scope="module")
def params(synth):
    return dict(synth.DEFAULT_PROCESS)


def _boost(p, beta):
    """Boost p by velocity beta (3-vector)."""
    b2 = float(beta @ beta)
    if b2 == 0.0:
        return p.copy()
    g = 1.0 / math.sqrt(1.0 - b2)
    bp = float(beta @ p[1:])
    out = np.empty(4)
    out[0] = g * (p[0] + bp)
    out[1:] = p[1:] + ((g - 1.0) * bp / b2 + g * p[0]) * beta
    return out


def _two_body(rng, M, m1, m2):
    """Momenta of a two-body decay at rest, isotropic."""
    p = math.sqrt((M * M - (m1 + m2) ** 2) * (M * M - (m1 - m2) ** 2)) / (2 * M)
    c = rng.uniform(-1, 1)
    s = math.sqrt(1 - c * c)
    ph = rng.uniform(0, 2 * math.pi)
    n = np.array([s * math.cos(ph), s * math.sin(ph), c])
    return (np.array([math.sqrt(p * p + m1 * m1), *(p * n)]),
            np.array([math.sqrt(p * p + m2 * m2), *(-p * n)]))


def _tth_kinematics(rng, rs, m, pH):
    """Beams along z in the partonic rest frame; the Higgs momentum pH given; the
    t tbar pair recoils and decays isotropically in its own rest frame."""
    k1, k2 = np.array([rs / 2, 0, 0, rs / 2]), np.array([rs / 2, 0, 0, -rs / 2])
    Q = k1 + k2 - pH
    MQ = math.sqrt(dot(Q, Q))
    t, tb = _two_body(rng, MQ, m, m)
    beta = Q[1:] / Q[0]
    return k1, k2, _boost(t, beta), _boost(tb, beta)


def _random_higgs(rng, rs, mh):
    E = rng.uniform(mh + 5.0, 0.3 * rs)
    p = math.sqrt(E * E - mh * mh)
    c = rng.uniform(-1, 1)
    s = math.sqrt(1 - c * c)
    ph = rng.uniform(0, 2 * math.pi)
    return np.array([E, p * s * math.cos(ph), p * s * math.sin(ph), p * c])


def test_tth_gauge_invariance(ora, params):
    P = ora.process(2, params)
    rng = np.random.default_rng(41)
    for rs in (600.0, 2000.0):
        pH = _random_higgs(rng, rs, 125.0)
        k1, k2, pt, ptb = _tth_kinematics(rng, rs, params["mt"], pH)
        assert np.allclose(k1 + k2, pt + ptb + pH, rtol=0, atol=1e-10 * rs)
        ref = ora.msq_tth_production(P, 0, k1, k2, pt, ptb, pH)
        gs4y2 = (4 * math.pi * params["alpha_s"]) ** 2 * (params["mt"] / (2 * params["mw"] / math.sqrt(4 * math.pi * params["alpha"] / params["sw2"]))) ** 2
        ref_ordered = ref / gs4y2 * 256      # undo couplings and the 1/(4 x 64) average
        assert ref > 0
        for which in (0, 1):
            for hel in (0, 1):
                assert ora.tth_gauge_probe(P, k1, k2, pt, ptb, pH, which, hel) < 1e-20 * ref_ordered


@pytest.mark.parametrize("channel", [0, 1])
def test_tth_soft_higgs_limit(ora, params, channel):
    P = ora.process(2, params)
    m = params["mt"]
    y = m / (2 * params["mw"] / math.sqrt(4 * math.pi * params["alpha"] / params["sw2"]))
    rng = np.random.default_rng(42 + channel)
    rs = 900.0
    for _ in range(3):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        c = rng.uniform(-1, 1)
        ph = rng.uniform(0, 2 * math.pi)
        # t tbar at lambda = 0, direction fixed; the same direction in the pair's rest frame
        dev = []
        for lam in (1e-3, 1e-4):
            pH = lam * rs * np.array([1.0, *n])
            k1, k2 = np.array([rs / 2, 0, 0, rs / 2]), np.array([rs / 2, 0, 0, -rs / 2])
            Q = k1 + k2 - pH
            MQ = math.sqrt(dot(Q, Q))
            p = math.sqrt(MQ * MQ / 4 - m * m)
            s_ = math.sqrt(1 - c * c)
            d = np.array([s_ * math.cos(ph), s_ * math.sin(ph), c])
            beta = Q[1:] / Q[0]
            pt = _boost(np.array([MQ / 2, *(p * d)]), beta)
            ptb = _boost(np.array([MQ / 2, *(-p * d)]), beta)
            p0 = math.sqrt(rs * rs / 4 - m * m)
            pt0 = np.array([rs / 2, *(p0 * d)])
            ptb0 = np.array([rs / 2, *(-p0 * d)])
            tt = ora.msq_ttbar_production(P, channel, k1, k2, pt0, ptb0)
            eik = y * y * m * m * (1 / dot(pt, pH) + 1 / dot(ptb, pH)) ** 2
            tth = ora.msq_tth_production(P, channel, k1, k2, pt, ptb, pH)
            dev.append(tth / (eik * tt) - 1.0)
        assert abs(dev[0]) < 2e-2
        assert abs(dev[1]) < 0.2 * abs(dev[0]) + 1e-6   # O(p_H): tenfold smaller


def test_tth_bose_and_lorentz(ora, params):
    P = ora.process(2, params)
    rng = np.random.default_rng(44)
    rs = 1200.0
    for _ in range(3):
        pH = _random_higgs(rng, rs, 125.0)
        k1, k2, pt, ptb = _tth_kinematics(rng, rs, params["mt"], pH)
        for channel in (0, 1):
            ref = ora.msq_tth_production(P, channel, k1, k2, pt, ptb, pH)
            if channel == 0:
                assert ora.msq_tth_production(P, 0, k2, k1, pt, ptb, pH) == pytest.approx(ref, rel=1e-11, abs=0)
            # boost along z and rotation about z
            bz = np.array([0.0, 0.0, rng.uniform(-0.7, 0.7)])
            a = rng.uniform(0, 2 * math.pi)
            R = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])

            def tr(p):
                q = _boost(p, bz)
                return np.array([q[0], *(R @ q[1:])])
            got = ora.msq_tth_production(P, channel, tr(k1), tr(k2), tr(pt), tr(ptb), tr(pH))
            assert got == pytest.approx(ref, rel=1e-10, abs=0)


def _decay3(rng, M, m12):
    """Massless three-body configuration at rest: M -> a + (b c), (b c) of mass m12."""
    a, w = _two_body(rng, M, 0.0, m12)
    b, c = _two_body(rng, m12, 0.0, 0.0)
    beta = w[1:] / w[0]
    return a, _boost(b, beta), _boost(c, beta)


@pytest.mark.parametrize("channel", [0, 1])
def test_tth_full_chain_factorises(ora, params, channel):
    """With on-shell tops the full 2 -> 8 |M|^2 (propagator denominators removed),
    averaged over parity-reflected decays in each top rest frame, equals
    |M|^2(ttH production, top spins summed) x (g_W^2/2)^4 c_t c_tbar x 3 y_b^2 4 p_b1.p_b2
    with c_t = 8 (p_t.p_l+)(p_b.p_nu), c_tbar = 8 (p_tbar.p_mu-)(p_bbar.p_nubar): the
    top decays as in semileptonic ttbar (the reflection removes their spin
    correlation), the W- decaying to one lepton channel, and the scalar Higgs decay
    factorising exactly (sum over spins of |ubar(b1) v(b2)|^2 = 4 p_b1.p_b2, 3 colours)."""
    P = ora.process(2, params)
    m, mw, ww, wt = params["mt"], params["mw"], params["ww"], params["wt"]
    mh, wh = params["mh"], params["wh"]
    gw2 = 4 * math.pi * params["alpha"] / params["sw2"]
    yb = params["mb"] / (2 * mw / math.sqrt(gw2))
    rng = np.random.default_rng(46 + channel)
    for rs in (700.0, 1500.0):
        pH = _random_higgs(rng, rs, mh + 0.003)
        k1, k2, pt, ptb = _tth_kinematics(rng, rs, m, pH)
        h1, h2 = _two_body(rng, math.sqrt(dot(pH, pH)), 0.0, 0.0)
        bH = pH[1:] / pH[0]
        h1, h2 = _boost(h1, bH), _boost(h2, bH)
        b0, l0, n0 = _decay3(rng, m, 79.0)
        bb0, m0, nb0 = _decay3(rng, m, 82.0)
        acc = 0.0
        for par_t in (1, -1):
            for par_tb in (1, -1):
                bt, btb = pt[1:] / pt[0], ptb[1:] / ptb[0]
                pb, pl, pn = (_boost(np.array([v[0], *(par_t * v[1:])]), bt) for v in (b0, l0, n0))
                pbb, pm, pnb = (_boost(np.array([v[0], *(par_tb * v[1:])]), btb) for v in (bb0, m0, nb0))
                w1, w2 = pl + pn, pm + pnb
                qh = h1 + h2
                dens = (wt * m) ** 4 * \
                    ((dot(w1, w1) - mw * mw) ** 2 + (mw * ww) ** 2) * \
                    ((dot(w2, w2) - mw * mw) ** 2 + (mw * ww) ** 2) * \
                    ((dot(qh, qh) - mh * mh) ** 2 + (mh * wh) ** 2)
                acc += ora.msq_tth(P, channel, k1, k2, pb, pl, pn, pbb, pm, pnb, h1, h2) * dens
                ct = 8 * dot(pt, pl) * dot(pb, pn)
                ctb = 8 * dot(ptb, pm) * dot(pbb, pnb)
        prod = ora.msq_tth_production(P, channel, k1, k2, pt, ptb, pH)
        want = prod * (gw2 / 2) ** 4 * ct * ctb * 3 * yb * yb * 4 * dot(h1, h2)
        assert acc / 4 == pytest.approx(want, rel=1e-9, abs=0)


# ---------------------------------------------------------------------------
# The dilepton ttH integrand (process kind 4): Eq. "integrand" with the neutrinos
# from Eq. "dilepsolv" and the Higgs pair's (f, m_H^2) variables of Eq. "mhsolve".
# ---------------------------------------------------------------------------
KIND_TTH = 4


def _tth_setup(ora, synth):
    return (ora.process(KIND_TTH, synth.DEFAULT_PROCESS),
            ora.tf(synth.DEFAULT_TF[KIND_TTH]))


@pytest.fixture(scope="module")
def tth_events(synth):
    return synth.gen_tth_dilep(4, 91)


def _dir(p):
    return p[1:] / np.linalg.norm(p[1:])


def _obj_dir(rec, o):
    eta, phi = float(rec[4 * o + 1]), float(rec[4 * o + 2])
    return np.array([math.cos(phi) / math.cosh(eta), math.sin(phi) / math.cosh(eta), math.tanh(eta)])


def _which_object(rec, p):
    d = _dir(p)
    best = min(range(2, 6), key=lambda o: np.linalg.norm(_obj_dir(rec, o) - d))
    assert np.linalg.norm(_obj_dir(rec, best) - d) < 1e-6
    return best


def _states(ora, P, T, rec, perm, x):
    n = ora.kinematics(P, T, rec, perm, x, 0)["n"]
    return [ora.kinematics(P, T, rec, perm, x, r) for r in range(n)]


def _find_point(ora, P, T, rec, perm, rng, tries=4000):
    for _ in range(tries):
        x = rng.uniform(0.02, 0.98, size=8)
        if ora.kinematics(P, T, rec, perm, x, 0)["n"] > 0:
            return x
    return None


def test_tth_dims_and_assignments(ora, synth, tth_events):
    """8 variables and 12 jet assignments: every ordered (b, bbar) pair of the four
    jets once, the other two jets going to the Higgs pair; the generator's truth
    index follows the same convention."""
    P, T = _tth_setup(ora, synth)
    assert ora.dims(KIND_TTH) == 8 and ora.nperm(KIND_TTH) == 12
    rng = np.random.default_rng(50)
    rec = tth_events[0]
    pairs = set()
    for perm in range(12):
        x = _find_point(ora, P, T, rec, perm, rng)
        assert x is not None
        lab = _states(ora, P, T, rec, perm, x)[0]["lab"]
        ob, obb, o1, o2 = (_which_object(rec, lab[i]) for i in (0, 3, 6, 7))
        assert len({ob, obb, o1, o2}) == 4
        assert synth.tth_perm_index(ob - 2, obb - 2) == perm
        pairs.add((ob, obb))
    assert len(pairs) == 12


def test_tth_conservation_and_virtualities(ora, synth, tth_events):
    P, T = _tth_setup(ora, synth)
    rng = np.random.default_rng(51)
    checked = 0
    for rec in tth_events:
        for _ in range(150):
            x = rng.uniform(0.02, 0.98, size=8)
            perm = int(rng.integers(0, 12))
            for k in _states(ora, P, T, rec, perm, x):
                fs, lab, k12, aux = k["fs"], k["lab"], k["k12"], k["aux"]
                assert fs.shape == (8, 4)
                tot = fs.sum(axis=0)
                assert np.allclose(k12[0] + k12[1], tot, rtol=0, atol=1e-12 * tot[0])
                ltot = lab.sum(axis=0)
                assert abs(ltot[1]) < 1e-10 * ltot[0] and abs(ltot[2]) < 1e-10 * ltot[0]
                for p in lab:
                    assert abs(dot(p, p)) < 1e-10 * p[0] ** 2
                b, lp, nu, bb, lm, nub, h1, h2 = lab
                want = (dot(lp + nu, lp + nu), dot(lm + nub, lm + nub),
                        dot(b + lp + nu, b + lp + nu), dot(bb + lm + nub, bb + lm + nub))
                for g, w in zip(aux[:4], want):
                    assert g == pytest.approx(w, rel=1e-9, abs=0)
                # the Higgs-pair energies lie inside their jet windows
                tf = synth.DEFAULT_TF[KIND_TTH]
                for p in (h1, h2):
                    Em = float(rec[4 * _which_object(rec, p)])
                    assert Em / tf["jet_lo_div"] * (1 - 1e-12) <= p[0] <= Em * tf["jet_hi_mul"] * (1 + 1e-12)
                checked += 1
    assert checked > 40


def _phys8(lab):
    """(E_b, E_bbar, nu_x, nu_y, nu_z, nubar_z, E_b1, E_b2)."""
    return np.array([lab[0][0], lab[3][0], lab[2][1], lab[2][2], lab[2][3], lab[5][3],
                     lab[6][0], lab[7][0]])


def test_tth_jacobian_is_determinant_of_the_map(ora, synth, tth_events):
    """Every state's Jacobian equals |det d(E_b, E_bbar, nu_x, nu_y, nu_z, nubar_z, E_b1,
    E_b2)/dx| by central differences of the map (the state at x +- h is the one
    nearest in those variables): this fixes the (f, m_H^2) transform and its
    two-solution Jacobian together with the neutrino part."""
    P, T = _tth_setup(ora, synth)
    rng = np.random.default_rng(52)
    n_ok = 0
    for rec in tth_events:
        for _ in range(60):
            x = rng.uniform(0.05, 0.95, size=8)
            perm = int(rng.integers(0, 12))
            for k in _states(ora, P, T, rec, perm, x):
                f0 = _phys8(k["lab"])
                M = np.zeros((8, 8))
                ok = True
                for j in range(8):
                    # h = 1e-5: the narrow Higgs Breit-Wigner makes the map steep, so smaller
                    # steps lose digits to cancellation (truncation at 1e-5 is ~1e-7)
                    h = 1e-5
                    cols = []
                    for sgn in (1, -1):
                        xs = x.copy()
                        xs[j] += sgn * h
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
                    M[:, j] = (cols[0] - cols[1]) / (2 * h)
                if not ok:
                    continue
                assert abs(np.linalg.det(M)) == pytest.approx(k["aux"][6], rel=2e-5, abs=0)
                n_ok += 1
    assert n_ok >= 10

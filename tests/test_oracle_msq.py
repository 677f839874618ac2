"""Pins of the oracle's tree-level |M|^2 (the |M_i|^2 of Sec. 1, Eq. "mem_def").

The oracle builds every amplitude from 4x4 Dirac matrices and explicit spinor
sums. These tests hold it against results fixed by physics and mathematics,
each computed here by an independent route:
  * analytic helicity-amplitude forms for q qbar -> (photon, Z) -> l l and
    u dbar -> W -> e nu (textbook electroweak structure),
  * closed-form total partonic cross sections (photon-only Drell-Yan, W),
  * Lorentz invariance,
  * the closed forms for q qbar -> Q Qbar and g g -> Q Qbar with massive quarks
    (Combridge 1979; Ellis-Stirling-Webber, QCD and Collider Physics),
  * gauge invariance of the colour-ordered g g -> t tbar amplitudes,
  * the polarised top-decay matrix element (charged lepton / down-type quark
    as the full spin analyser) and the exact factorisation of the full
    six-fermion |M|^2 into production x decay after parity-averaging each decay.
"""
import math

import numpy as np
import pytest

DEF = None


@pytest.fixture(scope="module")
def params(synth):
    return dict(synth.DEFAULT_PROCESS)


def dot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def rot_boost(rng, general=True):
    """Random proper orthochronous Lorentz transformation (as a 4x4 matrix).
    general=False keeps the z axis: rotation about z and a boost along z."""
    def rot(axis, ang):
        c, s = math.cos(ang), math.sin(ang)
        R = np.eye(4)
        i, j = {"x": (2, 3), "y": (3, 1), "z": (1, 2)}[axis]
        R[i, i], R[i, j], R[j, i], R[j, j] = c, -s, s, c
        return R

    def boost(axis, eta):
        B = np.eye(4)
        k = {"x": 1, "y": 2, "z": 3}[axis]
        B[0, 0] = B[k, k] = math.cosh(eta)
        B[0, k] = B[k, 0] = math.sinh(eta)
        return B
    if not general:
        return rot("z", rng.uniform(0, 6.28)) @ boost("z", rng.uniform(-1.5, 1.5))
    L = np.eye(4)
    for ax in ("x", "y", "z"):
        L = rot(ax, rng.uniform(0, 6.28)) @ boost(ax, rng.uniform(-1, 1)) @ L
    return L


def two_to_two(rs, c, phi=0.7):
    E = rs / 2
    s = math.sqrt(1 - c * c)
    k1 = np.array([E, 0, 0, E])
    k2 = np.array([E, 0, 0, -E])
    p3 = np.array([E, E * s * math.cos(phi), E * s * math.sin(phi), E * c])
    p4 = np.array([E, -p3[1], -p3[2], -p3[3]])
    return k1, k2, p3, p4


def dy_helicity(P, flavour, kq, kqb, plm, plp):
    """Sum over chiralities a (quark) and b (lepton) of 4|A_ab|^2 u^2 (a = b) or
    4|A_ab|^2 t^2 (a != b), with t = (kq - p_l-)^2, u = (kq - p_l+)^2, averaged
    over 4 spins and with colour factor 1/3."""
    e2 = 4 * math.pi * P["alpha"]
    sw2 = P["sw2"]
    gz = math.sqrt(e2 / (sw2 * (1 - sw2)))
    Qq, T3q = (2 / 3, 0.5) if flavour == 0 else (-1 / 3, -0.5)
    Ql, T3l = -1.0, -0.5
    gq = [gz * (T3q - Qq * sw2), gz * (-Qq * sw2)]
    gl = [gz * (T3l - Ql * sw2), gz * (-Ql * sw2)]
    s = dot(kq + kqb, kq + kqb)
    t = dot(kq - plm, kq - plm)
    u = dot(kq - plp, kq - plp)
    Dz = s - P["mz"] ** 2 + 1j * P["mz"] * P["wz"]
    tot = 0.0
    for a in range(2):
        for b in range(2):
            A = e2 * Qq * Ql / s + gq[a] * gl[b] / Dz
            tot += 4 * abs(A) ** 2 * (u * u if a == b else t * t)
    return tot / 12.0


def test_dy_vs_helicity_form(ora, params):
    P = ora.process(0, params)
    rng = np.random.default_rng(1)
    for rs in (40.0, 91.0, 91.19, 150.0, 700.0):
        for _ in range(4):
            c = rng.uniform(-1, 1)
            k1, k2, pm, pp = two_to_two(rs, c, rng.uniform(0, 6.28))
            for fl in (0, 1):
                want = dy_helicity(params, fl, k1, k2, pm, pp)
                got = ora.msq_dy(P, fl, k1, k2, pm, pp)
                assert got == pytest.approx(want, rel=1e-12, abs=0)
                # quark from the other beam
                got2 = ora.msq_dy(P, fl, k2, k1, pm, pp)
                assert got2 == pytest.approx(dy_helicity(params, fl, k2, k1, pm, pp), rel=1e-12, abs=0)


def test_dy_forward_backward_sign(ora, params):
    """Above the Z pole the l- prefers the quark direction (A_FB > 0 for u ubar)."""
    P = ora.process(0, params)
    k1, k2, pm_f, pp_f = two_to_two(200.0, 0.8)
    _, _, pm_b, pp_b = two_to_two(200.0, -0.8)
    assert ora.msq_dy(P, 0, k1, k2, pm_f, pp_f) > ora.msq_dy(P, 0, k1, k2, pm_b, pp_b)


def test_dy_photon_only_cross_section(ora, params):
    """sigma(q qbar -> photon -> l l) = 4 pi alpha^2 Q_q^2 / (9 s): integrate the
    oracle's |M|^2 over the two-body phase space (Gauss-Legendre in cos theta)."""
    p = dict(params)
    p["mz"] = 1e7  # decouple the Z
    P = ora.process(0, p)
    rs = 30.0
    s = rs * rs
    xg, wg = np.polynomial.legendre.leggauss(32)
    for fl, Q in ((0, 2 / 3), (1, -1 / 3)):
        avg = sum(w * ora.msq_dy(P, fl, *two_to_two(rs, c)) for c, w in zip(xg, wg)) / 2.0
        sigma = avg / (8 * math.pi) / (2 * s)   # int dPhi_2 = 1/(8 pi); flux 1/(2s)
        assert sigma == pytest.approx(4 * math.pi * p["alpha"] ** 2 * Q * Q / (9 * s), rel=1e-9, abs=0)


def test_w_vs_closed_forms(ora, params):
    P = ora.process(1, params)
    g2 = 4 * math.pi * params["alpha"] / params["sw2"]
    mw, ww = params["mw"], params["ww"]
    rng = np.random.default_rng(2)
    for rs in (60.0, 80.4, 120.0):
        s = rs * rs
        D2 = (s - mw * mw) ** 2 + (mw * ww) ** 2
        for _ in range(3):
            k1, k2, p3, p4 = two_to_two(rs, rng.uniform(-1, 1), rng.uniform(0, 6.28))
            # W+: u(k1) dbar(k2) -> e+(p3) nu(p4); |M|^2 = g^4 u^2/(12 D2), u = (k_u - p_e+)^2
            u = dot(k1 - p3, k1 - p3)
            assert ora.msq_w(P, +1, k1, k2, p3, p4) == pytest.approx(g2 * g2 * u * u / (12 * D2),
                                                                     rel=1e-12, abs=0)
            # W-: d(k1) ubar(k2) -> e-(p3) nubar(p4); |M|^2 = g^4 (k_d - p_nubar)^4/(12 D2)
            u2 = dot(k1 - p4, k1 - p4)
            assert ora.msq_w(P, -1, k1, k2, p3, p4) == pytest.approx(g2 * g2 * u2 * u2 / (12 * D2),
                                                                     rel=1e-12, abs=0)
        # total: sigma = G_F^2 m_W^4 s / (18 pi D2) with G_F = sqrt2 g^2 / (8 m_W^2)
        xg, wg = np.polynomial.legendre.leggauss(16)
        avg = sum(w * ora.msq_w(P, +1, *two_to_two(rs, c)) for c, w in zip(xg, wg)) / 2.0
        sigma = avg / (8 * math.pi) / (2 * s)
        GF = math.sqrt(2) * g2 / (8 * mw * mw)
        assert sigma == pytest.approx(GF ** 2 * mw ** 4 * s / (18 * math.pi * D2), rel=1e-9, abs=0)


def _tt_kinematics(rng, rs, m):
    E = rs / 2
    p = math.sqrt(E * E - m * m)
    c = rng.uniform(-1, 1)
    s_ = math.sqrt(1 - c * c)
    ph = rng.uniform(0, 6.28)
    pt = np.array([E, p * s_ * math.cos(ph), p * s_ * math.sin(ph), p * c])
    ptb = np.array([E, -pt[1], -pt[2], -pt[3]])
    return np.array([E, 0, 0, E]), np.array([E, 0, 0, -E]), pt, ptb


def test_ttbar_production_vs_closed_forms(ora, params):
    P = ora.process(2, params)
    m = params["mt"]
    g4 = (4 * math.pi * params["alpha_s"]) ** 2
    rng = np.random.default_rng(3)
    for rs in (350.0, 400.0, 1000.0, 3000.0):
        for _ in range(3):
            k1, k2, pt, ptb = _tt_kinematics(rng, rs, m)
            s = rs * rs
            t1, t2, rho = 2 * dot(k1, pt) / s, 2 * dot(k2, pt) / s, 4 * m * m / s
            gg = g4 * (1 / (6 * t1 * t2) - 3 / 8) * (t1 * t1 + t2 * t2 + rho - rho * rho / (4 * t1 * t2))
            qq = g4 * (4 / 9) * (t1 * t1 + t2 * t2 + rho / 2)
            assert ora.msq_ttbar_production(P, 0, k1, k2, pt, ptb) == pytest.approx(gg, rel=1e-11, abs=0)
            assert ora.msq_ttbar_production(P, 1, k1, k2, pt, ptb) == pytest.approx(qq, rel=1e-11, abs=0)


def test_ttbar_gauge_invariance(ora, params):
    P = ora.process(2, params)
    rng = np.random.default_rng(4)
    for rs in (400.0, 2000.0):
        k1, k2, pt, ptb = _tt_kinematics(rng, rs, params["mt"])
        ref = ora.msq_ttbar_production(P, 0, k1, k2, pt, ptb) / (4 * math.pi * params["alpha_s"]) ** 2
        for which in (0, 1):
            for hel in (0, 1):
                assert ora.ttbar_gauge_probe(P, k1, k2, pt, ptb, which, hel) < 1e-20 * ref * 256


def _random_massless(rng, scale=50.0):
    v = rng.normal(size=3)
    v = v / np.linalg.norm(v) * rng.uniform(0.2, 1.0) * scale
    return np.array([np.linalg.norm(v), *v])


def test_top_decay_spin_analyser(ora, params):
    """sum |ubar_b L/ P_L (p_t/ + m) u_t(s)|^2 = 4 m^2 * 8 (p_b.p_nu) ((p_t - m s).p_l)
    for a top at rest with spin s = +-z: the charged lepton analyses the top spin."""
    P = ora.process(2, params)
    m = params["mt"]
    rng = np.random.default_rng(5)
    for _ in range(5):
        pb, pl, pn = (_random_massless(rng) for _ in range(3))
        out = ora.top_decay_probe(P, pb, pl, pn)
        base = 32 * m ** 3 * dot(pb, pn)
        assert out[0] == pytest.approx(base * (pl[0] + pl[3]), rel=1e-12, abs=0)
        assert out[1] == pytest.approx(base * (pl[0] - pl[3]), rel=1e-12, abs=0)
        # antitop: the down-type quark d is the analyser, (p_bbar . p_ubar) the other factor
        pbb, pd, pu = (_random_massless(rng) for _ in range(3))
        out = ora.top_decay_probe(P, pbb, pd, pu, anti=True)
        base = 32 * m ** 3 * dot(pbb, pu)
        want = sorted([base * (pd[0] + pd[3]), base * (pd[0] - pd[3])])
        assert sorted(out) == pytest.approx(want, rel=1e-12, abs=0)


def _decay3(rng, M, m12):
    """Massless three-body configuration at rest: M -> a + (b c), with (b c) of mass m12."""
    def two(Mp, ma, mb):
        p = math.sqrt((Mp ** 2 - (ma + mb) ** 2) * (Mp ** 2 - (ma - mb) ** 2)) / (2 * Mp)
        c = rng.uniform(-1, 1)
        s = math.sqrt(1 - c * c)
        ph = rng.uniform(0, 6.28)
        d = np.array([s * math.cos(ph), s * math.sin(ph), c])
        return np.array([math.hypot(p, ma), *(p * d)]), np.array([math.hypot(p, mb), *(-p * d)])
    a, w = two(M, 0.0, m12)
    b, c = two(m12, 0.0, 0.0)
    return a, _boost(b, w), _boost(c, w)


def _boost(p, parent):
    E = parent[0]
    b = parent[1:] / E
    b2 = b @ b
    if b2 == 0:
        return p.copy()
    g = 1 / math.sqrt(1 - b2)
    bp = b @ p[1:]
    return np.array([g * (p[0] + bp), *(p[1:] + ((g - 1) * bp / b2 + g * p[0]) * b)])


@pytest.mark.parametrize("channel", [0, 1])
def test_ttbar_full_factorises_after_parity_average(ora, params, channel):
    """With on-shell tops the full 2->6 |M|^2 (propagator denominators removed)
    averaged over parity-reflected decays in each top rest frame equals
    |M|^2(production, top spins summed) * (g_W^2/2)^4 * 6 * c_t * c_tbar,
    c_t = 8 (p_t.p_l)(p_b.p_nu), c_tbar = 8 (p_tbar.p_d)(p_bbar.p_ubar).
    The reflection flips the decay density matrices' spin-dependent parts."""
    P = ora.process(2, params)
    m, mw, ww, wt = params["mt"], params["mw"], params["ww"], params["wt"]
    gw2 = 4 * math.pi * params["alpha"] / params["sw2"]
    rng = np.random.default_rng(6 + channel)
    for rs in (420.0, 900.0):
        k1, k2, pt, ptb = _tt_kinematics(rng, rs, m)
        b0, l0, n0 = _decay3(rng, m, 78.0)
        bb0, d0, u0 = _decay3(rng, m, 83.0)
        acc = 0.0
        for par_t in (1, -1):
            for par_tb in (1, -1):
                pb, pl, pn = (_boost(np.array([v[0], *(par_t * v[1:])]), pt) for v in (b0, l0, n0))
                pbb, pd, pu = (_boost(np.array([v[0], *(par_tb * v[1:])]), ptb) for v in (bb0, d0, u0))
                w1, w2 = pl + pn, pd + pu
                dens = (wt * m) ** 2 * (wt * m) ** 2 * \
                    ((dot(w1, w1) - mw * mw) ** 2 + (mw * ww) ** 2) * \
                    ((dot(w2, w2) - mw * mw) ** 2 + (mw * ww) ** 2)
                acc += ora.msq_ttbar(P, channel, k1, k2, pb, pl, pn, pbb, pd, pu) * dens
                ct = 8 * dot(pt, pl) * dot(pb, pn)
                ctb = 8 * dot(ptb, pd) * dot(pbb, pu)
        prod = ora.msq_ttbar_production(P, channel, k1, k2, pt, ptb)
        assert acc / 4 == pytest.approx(prod * (gw2 / 2) ** 4 * 6 * ct * ctb, rel=1e-9, abs=0)


def test_lorentz_invariance(ora, params, synth):
    rng = np.random.default_rng(7)
    Pd, Pw, Pt = (ora.process(k, params) for k in (0, 1, 2))
    for _ in range(4):
        k1, k2, p3, p4 = two_to_two(rng.uniform(50, 300), rng.uniform(-1, 1), rng.uniform(0, 6))
        L = rot_boost(rng)
        a = ora.msq_dy(Pd, 0, k1, k2, p3, p4)
        b = ora.msq_dy(Pd, 0, L @ k1, L @ k2, L @ p3, L @ p4)
        assert b == pytest.approx(a, rel=1e-11, abs=0)
        a = ora.msq_w(Pw, 1, k1, k2, p3, p4)
        b = ora.msq_w(Pw, 1, L @ k1, L @ k2, L @ p3, L @ p4)
        assert b == pytest.approx(a, rel=1e-11, abs=0)
    # ttbar: gluon polarisations are defined transverse to the beam axis, so use
    # transformations that keep the beams on the z axis (z rotations and z boosts)
    for ch in (0, 1):
        k1, k2, pt, ptb = _tt_kinematics(rng, 800.0, params["mt"])
        b, l, n = _decay3(rng, params["mt"] + 0.7, 80.0)
        bb, d, u = _decay3(rng, params["mt"] - 0.4, 81.0)
        mom = [_boost(v, pt) for v in (b, l, n)] + [_boost(v, ptb) for v in (bb, d, u)]
        a = ora.msq_ttbar(Pt, ch, k1, k2, *mom)
        L = rot_boost(rng, general=False)
        b2 = ora.msq_ttbar(Pt, ch, L @ k1, L @ k2, *[L @ v for v in mom])
        assert b2 == pytest.approx(a, rel=1e-10, abs=0)

"""The synthetic event generators follow the input recipe of the dilepton workloads
(host logic; no oracle arithmetic): generator truth obeys the decay chain, the
records hold what they claim, and the ttbb stand-in differs from ttH only in the extra
pair's mass.
"""
import math

import numpy as np
import pytest


def mass(p):
    return math.sqrt(max(p[0] ** 2 - p[1] ** 2 - p[2] ** 2 - p[3] ** 2, 0.0))


def eta_phi(p):
    pt = math.hypot(p[1], p[2])
    return math.asinh(p[3] / pt), math.atan2(p[2], p[1])


@pytest.mark.parametrize("which", ["tth", "ttbb"])
def test_dilepton_tth_and_ttbb_records(synth, which):
    gen = synth.gen_tth_dilep if which == "tth" else synth.gen_ttbb_dilep
    recs, tr = gen(40, 5, truth=True)
    P = synth.DEFAULT_PROCESS
    for r, t in zip(recs, tr):
        b, bb, lp, lm, nu, nub, h1, h2 = t
        # decay chain: t, tbar and W masses within the generated Breit-Wigner windows
        for q, m0, w in ((b + lp + nu, P["mt"], P["wt"]), (bb + lm + nub, P["mt"], P["wt"]),
                         (lp + nu, P["mw"], P["ww"]), (lm + nub, P["mw"], P["ww"])):
            assert abs(mass(q) - m0) <= 15 * w + 1e-6 * m0
        mp = mass(h1 + h2)
        if which == "tth":
            assert mp == pytest.approx(P["mh"], rel=1e-9, abs=0)
            assert r[27] == 4
        else:
            assert 20.0 - 1e-6 <= mp <= 300.0 + 1e-6
            assert r[27] == 5
        # leptons exact, both within |eta| <= 2.5; four jets sorted by measured energy
        assert r[0] == pytest.approx(lp[0], rel=1e-6, abs=0) and r[3] == 4
        assert r[4] == pytest.approx(lm[0], rel=1e-6, abs=0) and r[7] == 1
        Ej = [r[4 * o] for o in range(2, 6)]
        assert Ej == sorted(Ej, reverse=True) and min(Ej) >= 20.0
        assert all(r[4 * o + 3] == 5 for o in range(2, 6)) and r[26] == 6
        # the truth assignment points at the b and bbar jets' directions
        perm = int(r[28])
        jb, rest = perm // 3, [j for j in range(4) if j != perm // 3]
        jbb = rest[perm % 3]
        for q, j in ((b, jb), (bb, jbb)):
            eta, phi = eta_phi(q)
            assert r[4 * (2 + j) + 1] == pytest.approx(eta, abs=1e-5)
            assert math.cos(r[4 * (2 + j) + 2] - phi) == pytest.approx(1.0, abs=1e-9)
        assert synth.tth_perm_index(jb, jbb) == perm


def test_ttbb_stand_in_shares_the_ttH_stream_layout(synth):
    """Same seed: the ttH records are unchanged by the pair-mass option (the stream of
    draws is identical), and the verified parity cases keep their truth assignments."""
    a = synth.gen_tth_dilep(4, 7300)
    assert [int(v) for v in a[:, 28]] == [9, 4, 2, 9]
    assert np.all(a[:, 27] == 4)


def test_dilepton_ttbar_records(synth):
    recs, tr = synth.gen_ttbar_dilep(40, 9, truth=True)
    for r, t in zip(recs, tr):
        b, bb, lp, lm, nu, nub = t
        assert r[27] == 3 and r[26] == 4
        # MET = nu_T + nubar_T + Gaussian noise of 15 GeV per component (loose 6 sigma)
        assert abs(r[24] - (nu[1] + nub[1])) < 6 * 15.0 and abs(r[25] - (nu[2] + nub[2])) < 6 * 15.0
        jb = 2 if r[28] == 0 else 3
        eta, _ = eta_phi(b)
        assert r[4 * jb + 1] == pytest.approx(eta, abs=1e-5)

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
            assert abs(dot(n1, n1)) < 1e-12 * n1[0] ** 2 and abs(dot(n2, n2)) < 1e-12 * n2[0] ** 2
            got = virtualities(b, bb, lp, lm, n1, n2)
            for g, w in zip(got, q2):
                assert g == pytest.approx(w, rel=1e-11, abs=0)
            assert np.allclose(n1[1:3] + n2[1:3], met, rtol=0, atol=1e-12 * n1[0])
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


# ---------------------------------------------------------------------------
# The dilepton integrand (process kind 3): the change of variables of Sec. 3 with
# the b-jet energies and the four virtualities as integration variables.
# ---------------------------------------------------------------------------

def _dl_setup(ora, synth):
    return (ora.process(synth.PROC_TTBAR_DILEP, synth.DEFAULT_PROCESS),
            ora.tf(synth.DEFAULT_TF[synth.PROC_TTBAR]))


@pytest.fixture(scope="module")
def dl_events(synth):
    return synth.gen_ttbar_dilep(6, 77)


def _phys(lab):
    """(E_b, E_bbar, nu_x, nu_y, nu_z, nubar_z) in the lab frame (lab order b, l+,
    nu, bbar, mu-, nubar)."""
    return np.array([lab[0][0], lab[3][0], lab[2][1], lab[2][2], lab[2][3], lab[5][3]])


def test_dilep_dims(ora, synth):
    assert ora.dims(synth.PROC_TTBAR_DILEP) == 6 and ora.nperm(synth.PROC_TTBAR_DILEP) == 2


def test_dilep_conservation_and_virtualities(ora, synth, dl_events):
    """Every state: q1 + q2 = the sum of the final state, zero total pT (the missing
    pT is the visible imbalance at hadron level, Sec. 4), massless partons, measured
    leptons and jet directions, and the four virtualities the map set are the
    invariant masses of the momenta it produced."""
    P, T = _dl_setup(ora, synth)
    rng = np.random.default_rng(5)
    checked = 0
    for rec in dl_events:
        for _ in range(120):
            x = rng.uniform(0.02, 0.98, size=6)
            perm = int(rng.integers(0, 2))
            n = ora.kinematics(P, T, rec, perm, x, 0)["n"]
            for r in range(n):
                k = ora.kinematics(P, T, rec, perm, x, r)
                fs, lab, k12, aux = k["fs"], k["lab"], k["k12"], k["aux"]
                tot = fs.sum(axis=0)
                assert np.allclose(k12[0] + k12[1], tot, rtol=0, atol=1e-12 * tot[0])
                ltot = lab.sum(axis=0)
                assert abs(ltot[1]) < 1e-10 * ltot[0] and abs(ltot[2]) < 1e-10 * ltot[0]
                for p in lab:
                    assert abs(dot(p, p)) < 1e-10 * p[0] ** 2
                # leptons are the measured ones; jets keep their measured direction
                for slot, o in ((1, 0), (4, 1)):
                    assert lab[slot][0] == pytest.approx(float(rec[4 * o]), rel=1e-7, abs=0)
                for slot, o in ((0, 2 + perm), (3, 3 - perm)):
                    eta = math.atanh(lab[slot][3] / lab[slot][0])
                    assert eta == pytest.approx(float(rec[4 * o + 1]), rel=0, abs=1e-6)
                b, lp, nu, bb, lm, nub = lab
                want = (dot(lp + nu, lp + nu), dot(lm + nub, lm + nub),
                        dot(b + lp + nu, b + lp + nu), dot(bb + lm + nub, bb + lm + nub))
                for g, w in zip(aux[:4], want):
                    assert g == pytest.approx(w, rel=1e-11, abs=0)
                checked += 1
    assert checked > 50


def _roots(ora, P, T, rec, perm, x):
    n = ora.kinematics(P, T, rec, perm, x, 0)["n"]
    return [ora.kinematics(P, T, rec, perm, x, r) for r in range(n)]


def test_dilep_jacobian_is_determinant_of_the_map(ora, synth, dl_events):
    """The Jacobian of each solution equals |det d(E_b, E_bbar, nu_x, nu_y, nu_z,
    nubar_z) / dx| by central differences of the map; the solution at x +- h is the
    one nearest in the neutrino momenta (the solver's root order is not smooth)."""
    P, T = _dl_setup(ora, synth)
    rng = np.random.default_rng(6)
    n_ok = 0
    for rec in dl_events:
        for _ in range(10):
            x = rng.uniform(0.05, 0.95, size=6)
            perm = int(rng.integers(0, 2))
            for k in _roots(ora, P, T, rec, perm, x):
                f0 = _phys(k["lab"])
                M = np.zeros((6, 6))
                ok = True
                for j in range(6):
                    h = 1e-6
                    cols = []
                    for sgn in (1, -1):
                        xs = x.copy()
                        xs[j] += sgn * h
                        cand = [_phys(q["lab"]) for q in _roots(ora, P, T, rec, perm, xs)]
                        if not cand:
                            ok = False
                            break
                        d = [np.max(np.abs(c - f0)) for c in cand]
                        i = int(np.argmin(d))
                        if sorted(d)[1:2] and sorted(d)[1] < 10 * d[i]:
                            ok = False   # ambiguous match near a branch point
                            break
                        cols.append(cand[i])
                    if not ok:
                        break
                    M[:, j] = (cols[0] - cols[1]) / (2 * h)
                if not ok:
                    continue
                assert abs(np.linalg.det(M)) == pytest.approx(k["aux"][6], rel=2e-5, abs=0)
                n_ok += 1
    assert n_ok >= 20


def test_dilep_leptonic_w_branching(ora, synth, dl_events):
    """W- -> mu- nubar is one of the six channels of W- -> q qbar' (three colours,
    two light generations; tree level, no CKM mixing): at the same momenta the
    dilepton flavour-summed |M|^2 is 1/6 of the semileptonic one with mu-, nubar in
    the d, ubar slots."""
    P3, T = _dl_setup(ora, synth)
    P2 = ora.process(synth.PROC_TTBAR, synth.DEFAULT_PROCESS)
    rng = np.random.default_rng(8)
    n = 0
    for rec in dl_events:
        for _ in range(60):
            x = rng.uniform(0.02, 0.98, size=6)
            for k in _roots(ora, P3, T, rec, 0, x):
                x1, x2 = k["aux"][4], k["aux"][5]
                m3 = ora.flavour_msq(P3, k["fs"], k["k12"], x1, x2, rec)
                m2 = ora.flavour_msq(P2, k["fs"], k["k12"], x1, x2, rec)
                assert m3 > 0
                assert 6.0 * m3 == pytest.approx(m2, rel=1e-13, abs=0)
                n += 1
    assert n >= 6


def test_dilep_integrand_is_sum_over_solutions(ora, synth, dl_events):
    """The integrand at x is the sum of the per-solution weights, each positive and
    carrying the solution's own Jacobian; points outside the kinematic region
    (no neutrino solution) weigh zero."""
    P, T = _dl_setup(ora, synth)
    rng = np.random.default_rng(9)
    counts = set()
    for rec in dl_events:
        for _ in range(20):
            x = rng.uniform(0.0, 1.0, size=6)
            perm = int(rng.integers(0, 2))
            w = ora.integrand_roots(P, T, rec, perm, x)
            counts.add(len(w))
            assert all(v >= 0 for v in w)
            assert ora.integrand(P, T, rec, perm, x) == pytest.approx(sum(w), rel=1e-15, abs=0)
    assert 0 in counts and (2 in counts or 4 in counts)

"""Pins of the oracle's density normalisation (Sec. 1, Eq. "mem_def" with the n-body
phase-space element dPhi_n, and the transfer-function convolution for p-hat).

The prefactor the oracle multiplies -- flux 1/(|q1||q2|), (2 pi)^4, the 2/s of the
consumed dx1 dx2, one 1/((2 pi)^3 2E) per final-state particle, the flavour and
beam-orientation sum, and for energy-integrated objects E^2 sin(theta) times the
transfer functions -- is checked against what physics and mathematics fix, by routes
that share none of its formulas:

* Hadronic cross sections. At zero total pT a two-body final state is fixed by
  (m, y, cos theta*, phi*); the oracle's delta-TF density times the Cartesian measure
  d^3p1 d^3p2 delta^2(pT), whose Jacobian is taken by finite differences of the
  momenta built here, integrated over the decay angles, must equal
  dx1 dx2/(dm dy) x sum over flavours and orientations of f f sigma-hat(m^2) with the
  closed-form partonic cross sections: q qbar -> photon* -> l l,
  4 pi alpha^2 Q_q^2/(9 s-hat) (Z decoupled by a huge mass), and
  u dbar -> W+ -> e+ nu, g^4 s-hat/(576 pi [(s-hat - m_W^2)^2 + m_W^2 Gamma_W^2]).
  Eq. "mem_def" writes the flux as 1/(|q1||q2|); for head-on massless partons
  s-hat = 4|q1||q2|, so it is 8 times the textbook 1/(2 s-hat): the density must be
  exactly 8 times the textbook dsigma.
* Change of variables and transfer functions. At any point, each root's integrand
  equals the delta-TF density at that root's lab momenta times |det| of the map from
  the unit cube to the physical variables (finite differences of the oracle's own
  map), times |det d(px, py, pz)/d(E, theta, phi)| of every energy-integrated object
  (finite differences of spherical coordinates: the delta TF in direction is a
  density in theta and phi), times the transfer-function densities from
  scipy.stats.norm.
"""
import math

import numpy as np
import pytest

scipy_stats = pytest.importorskip("scipy.stats")


def _boost_z(p, y):
    ch, sh = math.cosh(y), math.sinh(y)
    return np.array([ch * p[0] + sh * p[3], p[1], p[2], sh * p[0] + ch * p[3]])


def _two_body(m, y, c, phi):
    """Massless pair of invariant mass m and rapidity y, zero pT, first particle at
    polar angle acos(c) and azimuth phi in the pair's rest frame."""
    s = math.sqrt(max(0.0, 1.0 - c * c))
    n = np.array([s * math.cos(phi), s * math.sin(phi), c])
    p1 = _boost_z(np.array([m / 2, *(m / 2 * n)]), y)
    p2 = _boost_z(np.array([m / 2, *(-m / 2 * n)]), y)
    return p1, p2


def _cartesian_jacobian(m, y, c, phi):
    """|det d(p1x, p1y, p1z, p2z)/d(m, y, c, phi)| by central differences (p2's
    transverse momentum is -p1's: the delta^2(pT) of the measure)."""
    v0 = np.array([m, y, c, phi])
    h = np.array([1e-6 * m, 1e-6, 1e-6, 1e-6])
    J = np.zeros((4, 4))
    for j in range(4):
        vp, vm = v0.copy(), v0.copy()
        vp[j] += h[j]
        vm[j] -= h[j]
        a, b = _two_body(*vp), _two_body(*vm)
        fa = np.array([a[0][1], a[0][2], a[0][3], a[1][3]])
        fb = np.array([b[0][1], b[0][2], b[0][3], b[1][3]])
        J[:, j] = (fa - fb) / (2 * h[j])
    return abs(np.linalg.det(J))


def _pdf(params, t, x):
    """The workload's parametric PDF A x^a (1-x)^b (t: quark, antiquark)."""
    return params["pdf_A"][t] * x ** params["pdf_a"][t] * (1 - x) ** params["pdf_b"][t]


def _angular_integral(ora, P, m, y, rec, n_c=12, n_phi=5):
    """int dc dphi |J| density(p1, p2) over the decay angles (Gauss-Legendre in c,
    midpoints in phi)."""
    cg, wg = np.polynomial.legendre.leggauss(n_c)
    total = 0.0
    for c, wc in zip(cg, wg):
        for k in range(n_phi):
            phi = 2 * math.pi * (k + 0.5) / n_phi
            p1, p2 = _two_body(m, y, c, phi)
            w, _ = ora.density(P, np.stack([p1, p2]), rec)
            total += wc * (2 * math.pi / n_phi) * _cartesian_jacobian(m, y, c, phi) * w
    return total


MY_POINTS = [(40.0, 0.0), (91.19, 0.9), (250.0, -1.7), (700.0, 2.4)]


@pytest.mark.parametrize("m,y", MY_POINTS)
def test_drell_yan_photon_cross_section(ora, synth, m, y):
    params = dict(synth.DEFAULT_PROCESS, mz=1.0e7, wz=1.0)   # Z decoupled
    P = ora.process(0, params)
    s = params["sqrt_s"] ** 2
    alpha = params["alpha"]
    tau = m * m / s
    x1, x2 = math.sqrt(tau) * math.exp(y), math.sqrt(tau) * math.exp(-y)
    lum = _pdf(params, 0, x1) * _pdf(params, 1, x2) + _pdf(params, 1, x1) * _pdf(params, 0, x2)
    sig_hat = sum(4 * math.pi * alpha ** 2 * q * q / (9 * m * m) for q in (2 / 3, -1 / 3))
    want = (2 * m / s) * lum * sig_hat          # dx1 dx2 = (2m/s) dm dy
    got = _angular_integral(ora, P, m, y, None)
    assert got / 8.0 == pytest.approx(want, rel=1e-6, abs=0)


@pytest.mark.parametrize("m,y", [(80.4, 0.0), (78.0, 1.3), (120.0, -0.8)])
def test_w_cross_section(ora, synth, m, y):
    params = dict(synth.DEFAULT_PROCESS)
    P = ora.process(1, params)
    s = params["sqrt_s"] ** 2
    g2 = 4 * math.pi * params["alpha"] / params["sw2"]
    mw, ww = params["mw"], params["ww"]
    tau = m * m / s
    x1, x2 = math.sqrt(tau) * math.exp(y), math.sqrt(tau) * math.exp(-y)
    lum = _pdf(params, 0, x1) * _pdf(params, 1, x2) + _pdf(params, 1, x1) * _pdf(params, 0, x2)
    sh = m * m
    sig_hat = g2 * g2 * sh / (576 * math.pi * ((sh - mw * mw) ** 2 + mw * mw * ww * ww))
    want = (2 * m / s) * lum * sig_hat
    rec = np.zeros(32, dtype=np.float32)
    rec[3] = synth.KIND_E_PLUS                   # e+ : the W+ charge
    got = _angular_integral(ora, P, m, y, rec)
    assert got / 8.0 == pytest.approx(want, rel=1e-6, abs=0)


def test_density_is_boost_invariant_in_the_transverse_plane(ora, synth):
    """Reading of Eq. "mem_def" with a flat recoil: the final state is boosted
    transversely to zero pT before |M|^2 and x1, x2 are taken, so the density times
    the product of lab energies (the invariant measure d^3p/E) does not change when
    a zero-pT configuration is boosted transversely."""
    P = ora.process(2, synth.DEFAULT_PROCESS)
    rec = synth.gen_ttbar_parton(4, 91)
    rng = np.random.default_rng(5)
    for r in rec:
        lab = []
        for o in (1, 0, 5, 2, 3, 4):             # b, l+, nu, bbar, d, ubar
            E, eta, phi = (float(v) for v in r[4 * o: 4 * o + 3])
            lab.append([E, E * math.cos(phi) / math.cosh(eta), E * math.sin(phi) / math.cosh(eta),
                        E * math.tanh(eta)])
        lab = np.array(lab)
        tot = lab.sum(axis=0)
        # remove the record's own transverse imbalance exactly (boost to zero pT)
        bx, by = tot[1] / tot[0], tot[2] / tot[0]

        def tboost(p, bx, by):
            b2 = bx * bx + by * by
            g = 1 / math.sqrt(1 - b2)
            bp = bx * p[1] + by * p[2]
            c = (g - 1) * bp / b2 - g * p[0]
            return np.array([g * (p[0] - bp), p[1] + c * bx, p[2] + c * by, p[3]])
        zero = np.array([tboost(p, bx, by) for p in lab])
        w0, _ = ora.density(P, zero)
        for _ in range(3):
            ang = rng.uniform(0, 2 * math.pi)
            beta = rng.uniform(0.05, 0.4)
            moved = np.array([tboost(p, beta * math.cos(ang), beta * math.sin(ang)) for p in zero])
            w1, _ = ora.density(P, moved)
            assert w1 * np.prod(moved[:, 0]) == pytest.approx(w0 * np.prod(zero[:, 0]), rel=1e-9, abs=0)


def _theta_phi(p):
    return math.acos(p[3] / p[0]), math.atan2(p[2], p[1])


def _spherical_jacobian(p):
    """|det d(px, py, pz)/d(E, theta, phi)| at a massless momentum, by central
    differences of spherical coordinates."""
    E = p[0]
    th, ph = _theta_phi(p)

    def cart(E, th, ph):
        return np.array([E * math.sin(th) * math.cos(ph), E * math.sin(th) * math.sin(ph),
                         E * math.cos(th)])
    v0 = [E, th, ph]
    h = [1e-6 * E, 1e-7, 1e-7]
    J = np.zeros((3, 3))
    for j in range(3):
        vp, vm = list(v0), list(v0)
        vp[j] += h[j]
        vm[j] -= h[j]
        J[:, j] = (cart(*vp) - cart(*vm)) / (2 * h[j])
    return abs(np.linalg.det(J))


def _phys(kind, lab):
    """Physical integration variables in map order (lab frame)."""
    if kind == 0:
        return np.array([lab[0][0], lab[1][0]])
    if kind == 1:
        return np.array([lab[0][0], lab[1][1], lab[1][2], lab[1][3]])
    return np.array([lab[4][0], lab[5][0], lab[3][0], lab[2][1], lab[2][2], lab[2][3], lab[0][0]])


def _map_jacobian(ora, P, T, rec, perm, x, root, n_roots, kind):
    d = len(x)
    M = np.zeros((d, d))
    for j in range(d):
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        kp = ora.kinematics(P, T, rec, perm, xp, root)
        km = ora.kinematics(P, T, rec, perm, xm, root)
        if kp["n"] != n_roots or km["n"] != n_roots:
            return None
        M[:, j] = (_phys(kind, kp["lab"]) - _phys(kind, km["lab"])) / (2 * h)
    return abs(np.linalg.det(M))


def _tf_and_measure(kind, tfp, rec, lab):
    """Transfer-function densities (scipy) times the spherical measures of the
    energy-integrated objects: the factors that convert the delta-TF density into
    the integrand's density in the measured variables."""
    norm = scipy_stats.norm.pdf
    out = 1.0
    if kind == 0:
        for i in range(2):
            E = lab[i][0]
            out *= norm(rec[4 * i], loc=E, scale=tfp["lep_rel"] * E) * _spherical_jacobian(lab[i])
        return out
    met = norm(rec[24], loc=lab[-1 if kind == 1 else 2][1], scale=tfp["met_sigma"]) * \
        norm(rec[25], loc=lab[-1 if kind == 1 else 2][2], scale=tfp["met_sigma"])
    if kind == 1:
        E = lab[0][0]
        return met * norm(rec[0], loc=E, scale=tfp["lep_rel"] * E) * _spherical_jacobian(lab[0])
    # ttbar: jets b, bbar, d, ubar (lab slots 0, 3, 4, 5) carry the double Gaussian
    return met


def _jet_objects(perm):
    perms = [p for p in __import__("itertools").permutations(range(4))]
    return [1 + j for j in perms[perm]]          # record objects of b, bbar, d, ubar


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_integrand_is_density_times_measure_and_tfs(ora, synth, kind):
    tfp = synth.DEFAULT_TF[kind]
    P, T = ora.process(kind, synth.DEFAULT_PROCESS), ora.tf(tfp)
    recs = synth.gen_events(kind, 3, 40 + kind)
    d = ora.dims(kind)
    rng = np.random.default_rng(60 + kind)
    norm = scipy_stats.norm.pdf
    checked = 0
    for rec in recs:
        for _ in range(25):
            x = rng.uniform(0.05, 0.95, size=d)
            perm = int(rng.integers(0, ora.nperm(kind)))
            per_root = ora.integrand_roots(P, T, rec, perm, x)
            for r, w in enumerate(per_root):
                k = ora.kinematics(P, T, rec, perm, x, r)
                lab = k["lab"]
                jac = _map_jacobian(ora, P, T, rec, perm, x, r, len(per_root), kind)
                if jac is None or w == 0.0:
                    continue
                dens, _ = ora.density(P, lab, rec)
                fac = _tf_and_measure(kind, tfp, rec, lab)
                if kind == 2:
                    for slot, obj in zip((0, 3, 4, 5), _jet_objects(perm)):
                        E = lab[slot][0]
                        Em = float(rec[4 * (obj)])
                        tf = (1 - tfp["jet_tail_w"]) * norm(Em, loc=E, scale=tfp["jet_core"] * E) + \
                            tfp["jet_tail_w"] * norm(Em, loc=E, scale=tfp["jet_tail"] * E)
                        fac *= tf * _spherical_jacobian(lab[slot])
                assert w == pytest.approx(dens * jac * fac, rel=2e-5, abs=0)
                checked += 1
    assert checked >= 20

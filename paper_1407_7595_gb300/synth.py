"""Seeded synthetic inputs: event records and default parameter sets.

This module is input data only. It holds none of the integrand's arithmetic
(no maps, matrix elements, PDFs, transfer functions or VEGAS); both the CUDA
path and the FP64 oracle consume what it produces, and neither is imported here.

The paper evaluates the matrix element method on MadGraph+Pythia samples of
ttH(bb) and ttbb (Sec. 3, Sec. 4); those samples are not available, so seeded
generators of the same kind of final states stand in for them: resonant
Drell-Yan and W events and semileptonic ttbar events with double-Gaussian
jet-energy smearing (the transfer-function form of Sec. 1 and Fig. "tf_jet").

Event record: 32 float32 values per event.
  [4*o + 0..3] for object o = 0..5 : (E_measured [GeV], eta, phi, kind)
  [24], [25]                        : missing transverse momentum (x, y) [GeV]
  [26]                              : number of objects
  [27]                              : process kind (0 DY, 1 W, 2 ttbar)
  [28]                              : generator truth, ttbar only: index of the
                                      jet permutation that matches the partons
                                      (diagnostic only, never read by the method)
  [29..31]                          : zero
Object kinds: 1 mu-, 2 mu+, 3 e-, 4 e+, 5 jet, 6 neutrino.
Object order: DY (mu-, mu+); W (charged lepton); ttbar (l+, 4 jets by
decreasing measured energy).

Parton-level ttbar record (the parton-level analysis of Sec. 4: every final-state
momentum known exactly): the same layout with exact energies and
  objects 0..5 : l+, the two b quarks (by decreasing energy), d, ubar, neutrino
  [24], [25]   : neutrino (px, py);  [26] = 6;  [27] = 2 (ttbar)
  [28]         : generator truth: 0 if object 1 is the b (object 2 the bbar), else 1
  [29]         : 1 (marks a parton-level record)
"""
from __future__ import annotations

import itertools
import math

import numpy as np

RECORD_FLOATS = 32
KIND_NONE, KIND_MU_MINUS, KIND_MU_PLUS, KIND_E_MINUS, KIND_E_PLUS, KIND_JET, KIND_NU = range(7)
PROC_DY, PROC_W, PROC_TTBAR = 0, 1, 2

SQRT_S = 13000.0

# Physical parameters of the three processes (masses/widths from the workload
# definitions; couplings are a fixed electroweak/QCD parameter set).
DEFAULT_PROCESS = {
    "sqrt_s": SQRT_S,
    "mz": 91.19, "wz": 2.50,
    "mw": 80.4, "ww": 2.09,
    "mt": 173.0, "wt": 1.4,
    "alpha": 1.0 / 128.0, "sw2": 0.2312, "alpha_s": 0.118,
    # parametric PDFs f(x) = A x^a (1-x)^b for (quark, antiquark, gluon)
    "pdf_A": (1.0, 1.0, 1.0),
    "pdf_a": (-0.5, -0.5, -1.0),
    "pdf_b": (3.0, 5.0, 5.0),
    # Higgs (ttH, Sec. 3): mass, width and the b-quark mass of the b Yukawa coupling
    "mh": 125.0, "wh": 0.00407, "mb": 4.7,
}

# Transfer-function parameters per process.
DEFAULT_TF = {
    PROC_DY: {"lep_rel": 0.02, "window_k": 5.0, "jet_core": 0.1, "jet_tail": 0.3,
              "jet_tail_w": 0.2, "jet_lo_div": 1.9, "jet_hi_mul": 10.0,
              "met_sigma": 15.0, "met_box_k": 4.0},
    PROC_W: {"lep_rel": 0.03, "window_k": 5.0, "jet_core": 0.1, "jet_tail": 0.3,
             "jet_tail_w": 0.2, "jet_lo_div": 1.9, "jet_hi_mul": 10.0,
             "met_sigma": 15.0, "met_box_k": 4.0},
    PROC_TTBAR: {"lep_rel": 0.0, "window_k": 5.0, "jet_core": 0.1, "jet_tail": 0.3,
                 "jet_tail_w": 0.2, "jet_lo_div": 1.9, "jet_hi_mul": 10.0,
                 "met_sigma": 15.0, "met_box_k": 4.0},
}

PROC_TTBAR_DILEP = 3
# dilepton ttbar: leptons measured exactly, b jets as in semileptonic ttbar
DEFAULT_TF[PROC_TTBAR_DILEP] = dict(DEFAULT_TF[PROC_TTBAR])
DEFAULT_TF[4] = dict(DEFAULT_TF[PROC_TTBAR])   # dilepton ttH
DEFAULT_TF[5] = dict(DEFAULT_TF[PROC_TTBAR])   # dilepton ttbb (same records as ttH)

DIMS = {PROC_DY: 2, PROC_W: 4, PROC_TTBAR: 7, PROC_TTBAR_DILEP: 6, 4: 8, 5: 8}
NPERM = {PROC_DY: 1, PROC_W: 1, PROC_TTBAR: 24, PROC_TTBAR_DILEP: 2, 4: 12, 5: 12}

# The five workloads: (process, events, points per event, base seed).
SEED_BASE = 0x4D454D00
WORKLOADS = {
    "dy": dict(proc=PROC_DY, n_events=64, n_points=1 << 16, seed=SEED_BASE + 0),
    "w": dict(proc=PROC_W, n_events=1024, n_points=1 << 20, seed=SEED_BASE + 1),
    "ttbar": dict(proc=PROC_TTBAR, n_events=4096, n_points=1 << 22, seed=SEED_BASE + 2),
    "mix": dict(proc=None, n_events=16384, n_points=1 << 24, seed=SEED_BASE + 3),
    "flow": dict(proc=PROC_TTBAR, n_events=4096, n_points=1 << 22, seed=SEED_BASE + 4),
    # parton-level ttbar (Sec. 4): no integration, one weight per b-quark assignment
    "parton": dict(proc=PROC_TTBAR, n_events=1 << 20, n_points=0, seed=SEED_BASE + 5),
    # dilepton ttbar (Sec. 3-4 hadron level without the Higgs): 6 dims x 2 b assignments
    "ttdl": dict(proc=3, n_events=1024, n_points=1 << 18, seed=SEED_BASE + 6),
    # dilepton ttH (Sec. 3-4, the paper's hadron-level signal): 8 dims x 12 jet assignments
    "tth": dict(proc=4, n_events=256, n_points=12 << 16, seed=SEED_BASE + 7),
    "ttbb": dict(proc=5, n_events=64, n_points=12 << 14, seed=SEED_BASE + 8),
}


def jet_permutations():
    """The 24 assignments of 4 measured jets to the partons (b, bbar, d, ubar),
    in lexicographic order: entry p[k] is the jet taking parton slot k."""
    return list(itertools.permutations(range(4)))


# ---------------------------------------------------------------- kinematics
def _bw_mass(rng, m, w, lo, hi, size=None):
    """Breit-Wigner (Cauchy in m^2) mass, truncated to [lo, hi]."""
    a = math.atan((lo * lo - m * m) / (m * w))
    b = math.atan((hi * hi - m * m) / (m * w))
    t = rng.uniform(a, b, size)
    return np.sqrt(m * m + m * w * np.tan(t))


def _two_body(rng, M, m1, m2):
    """Isotropic two-body decay at rest; returns the 4-momenta of both daughters."""
    lam = (M * M - (m1 + m2) ** 2) * (M * M - (m1 - m2) ** 2)
    p = math.sqrt(max(lam, 0.0)) / (2.0 * M)
    c = rng.uniform(-1.0, 1.0)
    s = math.sqrt(max(0.0, 1.0 - c * c))
    ph = rng.uniform(0.0, 2.0 * math.pi)
    d = np.array([s * math.cos(ph), s * math.sin(ph), c])
    p1 = np.concatenate([[math.sqrt(p * p + m1 * m1)], p * d])
    p2 = np.concatenate([[math.sqrt(p * p + m2 * m2)], -p * d])
    return p1, p2


def _boost_to_lab(p, parent):
    """Boost 4-vector p from the rest frame of `parent` into the frame where
    `parent` has the given 4-momentum."""
    E, px, py, pz = parent
    m = math.sqrt(max(E * E - px * px - py * py - pz * pz, 0.0))
    bx, by, bz = px / E, py / E, pz / E
    b2 = bx * bx + by * by + bz * bz
    if b2 == 0.0:
        return np.array(p, dtype=float)
    g = E / m
    bp = bx * p[1] + by * p[2] + bz * p[3]
    g2 = (g - 1.0) / b2
    return np.array([g * (p[0] + bp),
                     p[1] + g2 * bp * bx + g * bx * p[0],
                     p[2] + g2 * bp * by + g * by * p[0],
                     p[3] + g2 * bp * bz + g * bz * p[0]])


def _eta_phi(p):
    pt = math.hypot(p[1], p[2])
    pabs = math.sqrt(pt * pt + p[3] * p[3])
    eta = 0.5 * math.log((pabs + p[3]) / (pabs - p[3])) if pt > 0 else math.copysign(1e9, p[3])
    return eta, math.atan2(p[2], p[1])


def _drell_yan_like(rng, m, rap, lep_kinds):
    """Resonance of mass m at rest in the transverse plane with rapidity rap,
    decaying isotropically into two massless leptons."""
    E = m * math.cosh(rap)
    pz = m * math.sinh(rap)
    p1, p2 = _two_body(rng, m, 0.0, 0.0)
    par = np.array([E, 0.0, 0.0, pz])
    return _boost_to_lab(p1, par), _boost_to_lab(p2, par)


def gen_dy(n, seed, tf=None):
    tf = tf or DEFAULT_TF[PROC_DY]
    P = DEFAULT_PROCESS
    rng = np.random.Generator(np.random.Philox(seed))
    out = np.zeros((n, RECORD_FLOATS), dtype=np.float32)
    i = 0
    while i < n:
        m = _bw_mass(rng, P["mz"], P["wz"], 60.0, 120.0)
        y = rng.uniform(-2.0, 2.0)
        lm, lp = _drell_yan_like(rng, m, y, None)
        eta_m, phi_m = _eta_phi(lm)
        eta_p, phi_p = _eta_phi(lp)
        if abs(eta_m) > 2.5 or abs(eta_p) > 2.5:
            continue
        Em = lm[0] * (1.0 + tf["lep_rel"] * rng.standard_normal())
        Ep = lp[0] * (1.0 + tf["lep_rel"] * rng.standard_normal())
        r = out[i]
        r[0:4] = (Em, eta_m, phi_m, KIND_MU_MINUS)
        r[4:8] = (Ep, eta_p, phi_p, KIND_MU_PLUS)
        r[26] = 2
        r[27] = PROC_DY
        i += 1
    return out


def gen_w(n, seed, tf=None):
    tf = tf or DEFAULT_TF[PROC_W]
    P = DEFAULT_PROCESS
    rng = np.random.Generator(np.random.Philox(seed))
    out = np.zeros((n, RECORD_FLOATS), dtype=np.float32)
    i = 0
    while i < n:
        m = _bw_mass(rng, P["mw"], P["ww"], 50.0, 110.0)
        y = rng.uniform(-2.0, 2.0)
        e, nu = _drell_yan_like(rng, m, y, None)
        eta, phi = _eta_phi(e)
        if abs(eta) > 2.5:
            continue
        Em = e[0] * (1.0 + tf["lep_rel"] * rng.standard_normal())
        r = out[i]
        r[0:4] = (Em, eta, phi, KIND_E_PLUS)
        r[24] = nu[1] + tf["met_sigma"] * rng.standard_normal()
        r[25] = nu[2] + tf["met_sigma"] * rng.standard_normal()
        r[26] = 1
        r[27] = PROC_W
        i += 1
    return out


def gen_ttbar(n, seed, tf=None):
    tf = tf or DEFAULT_TF[PROC_TTBAR]
    P = DEFAULT_PROCESS
    rng = np.random.Generator(np.random.Philox(seed))
    out = np.zeros((n, RECORD_FLOATS), dtype=np.float32)
    perms = jet_permutations()
    i = 0
    while i < n:
        mtt = rng.uniform(350.0, 1000.0)
        mt1 = _bw_mass(rng, P["mt"], P["wt"], P["mt"] - 15 * P["wt"], P["mt"] + 15 * P["wt"])
        mt2 = _bw_mass(rng, P["mt"], P["wt"], P["mt"] - 15 * P["wt"], P["mt"] + 15 * P["wt"])
        if mt1 + mt2 >= mtt:
            continue
        mw1 = _bw_mass(rng, P["mw"], P["ww"], P["mw"] - 15 * P["ww"], P["mw"] + 15 * P["ww"])
        mw2 = _bw_mass(rng, P["mw"], P["ww"], P["mw"] - 15 * P["ww"], P["mw"] + 15 * P["ww"])
        y = rng.uniform(-1.5, 1.5)
        sysp = np.array([mtt * math.cosh(y), 0.0, 0.0, mtt * math.sinh(y)])
        t, tb = _two_body(rng, mtt, mt1, mt2)
        t, tb = _boost_to_lab(t, sysp), _boost_to_lab(tb, sysp)
        b, wp = _two_body(rng, mt1, 0.0, mw1)
        b, wp = _boost_to_lab(b, t), _boost_to_lab(wp, t)
        lep, nu = _two_body(rng, mw1, 0.0, 0.0)
        lep, nu = _boost_to_lab(lep, wp), _boost_to_lab(nu, wp)
        bb, wm = _two_body(rng, mt2, 0.0, mw2)
        bb, wm = _boost_to_lab(bb, tb), _boost_to_lab(wm, tb)
        d, ub = _two_body(rng, mw2, 0.0, 0.0)
        d, ub = _boost_to_lab(d, wm), _boost_to_lab(ub, wm)
        eta_l, phi_l = _eta_phi(lep)
        if abs(eta_l) > 2.5:
            continue
        partons = [b, bb, d, ub]
        jets = []
        ok = True
        for p in partons:
            eta, phi = _eta_phi(p)
            rel = tf["jet_tail"] if rng.uniform() < tf["jet_tail_w"] else tf["jet_core"]
            Em = p[0] * (1.0 + rel * rng.standard_normal())
            if abs(eta) > 2.5 or Em < 20.0:
                ok = False
                break
            jets.append((Em, eta, phi))
        if not ok:
            continue
        order = sorted(range(4), key=lambda k: -jets[k][0])  # jet slot -> parton
        # truth permutation: parton slot k sits in jet position order.index(k)
        truth = tuple(order.index(k) for k in range(4))
        r = out[i]
        r[0:4] = (lep[0], eta_l, phi_l, KIND_E_PLUS)
        for slot, k in enumerate(order):
            r[4 + 4 * slot: 8 + 4 * slot] = (jets[k][0], jets[k][1], jets[k][2], KIND_JET)
        r[24] = nu[1] + tf["met_sigma"] * rng.standard_normal()
        r[25] = nu[2] + tf["met_sigma"] * rng.standard_normal()
        r[26] = 5
        r[27] = PROC_TTBAR
        r[28] = perms.index(truth)
        i += 1
    return out


# ---------------------------------------------------------- tabulated PDFs
def pdf_grid_table(params=None, n_x=512, n_q=64, x_min=1e-6, q_min=10.0, q_max=SQRT_S,
                   q0=91.19, kappa=(0.5, 0.5, 0.5), lam=(0.0, 0.02, 0.04)):
    """Synthetic stand-in for a tabulated PDF set (the LHAPDF/CTEQ grids of Sec. 3
    are not available): f_t(x, Q) = A_t x^(a_t - lam_t L) (1 - x)^(b_t + kappa_t L),
    L = ln(Q / q0), for t = quark, antiquark, gluon, with (A, a, b) of the
    parametric set; at Q = q0 (or with kappa = lam = 0) it is that set. The
    high-x fall-off steepens and the low-x sea and gluon rise with Q, as under
    QCD evolution. Nodes: n_x uniform in ln x over [ln x_min, 0] and n_q uniform
    in ln Q over [ln q_min, ln q_max]. Returns dict(table=(3, n_q, n_x) float32,
    lx=(ln x_min, 0), lq=(ln q_min, ln q_max))."""
    P = params or DEFAULT_PROCESS
    lx = np.linspace(math.log(x_min), 0.0, n_x)
    lq = np.linspace(math.log(q_min), math.log(q_max), n_q)
    x = np.exp(lx)[None, :]
    x[:, -1] = 1.0
    L = (lq - math.log(q0))[:, None]
    tab = np.zeros((3, n_q, n_x))
    for t in range(3):
        a = P["pdf_a"][t] - lam[t] * L
        b = P["pdf_b"][t] + kappa[t] * L
        tab[t] = P["pdf_A"][t] * x ** a * (1.0 - x) ** b
    return {"table": tab.astype(np.float32), "lx": (float(lx[0]), 0.0),
            "lq": (float(lq[0]), float(lq[-1]))}


# ------------------------------------------------ parton-level ttbar (vectorised)
def _bw_mass_v(rng, m, w, k, n):
    """n Breit-Wigner masses (Cauchy in m^2) truncated to m -+ k w."""
    a = np.arctan(((m - k * w) ** 2 - m * m) / (m * w))
    b = np.arctan(((m + k * w) ** 2 - m * m) / (m * w))
    return np.sqrt(m * m + m * w * np.tan(rng.uniform(a, b, n)))


def _two_body_v(rng, M, m1, m2):
    """Isotropic two-body decays at rest of masses M (array) into m1, m2 (arrays
    or scalars); (n, 4) momenta of both daughters."""
    lam = (M * M - (m1 + m2) ** 2) * (M * M - (m1 - m2) ** 2)
    p = np.sqrt(np.maximum(lam, 0.0)) / (2.0 * M)
    c = rng.uniform(-1.0, 1.0, M.shape)
    s = np.sqrt(np.maximum(0.0, 1.0 - c * c))
    ph = rng.uniform(0.0, 2.0 * math.pi, M.shape)
    d = np.stack([s * np.cos(ph), s * np.sin(ph), c], axis=1)
    p1 = np.concatenate([np.sqrt(p * p + m1 * m1 + 0 * M)[:, None], p[:, None] * d], axis=1)
    p2 = np.concatenate([np.sqrt(p * p + m2 * m2 + 0 * M)[:, None], -p[:, None] * d], axis=1)
    return p1, p2


def _boost_v(p, parent):
    """Row-wise version of _boost_to_lab."""
    E = parent[:, 0]
    bvec = parent[:, 1:] / E[:, None]
    b2 = np.sum(bvec * bvec, axis=1)
    m = np.sqrt(np.maximum(E * E - np.sum(parent[:, 1:] ** 2, axis=1), 0.0))
    g = E / m
    bp = np.sum(bvec * p[:, 1:], axis=1)
    g2 = np.where(b2 > 0, (g - 1.0) / np.where(b2 > 0, b2, 1.0), 0.0)
    out = np.empty_like(p)
    out[:, 0] = g * (p[:, 0] + bp)
    out[:, 1:] = p[:, 1:] + (g2 * bp)[:, None] * bvec + (g * p[:, 0])[:, None] * bvec
    return out


def _eta_phi_v(p):
    pt = np.hypot(p[:, 1], p[:, 2])
    return np.arcsinh(p[:, 3] / pt), np.arctan2(p[:, 2], p[:, 1]), pt


def gen_ttbar_parton(n, seed):
    """Parton-level semileptonic ttbar events (Sec. 4, parton level): the same
    production and decay chain as gen_ttbar, no smearing, the neutrino kept as
    object 5; l+ and the quarks within |eta| <= 2.5, quarks with E >= 20 GeV."""
    P = DEFAULT_PROCESS
    rng = np.random.Generator(np.random.Philox(seed))
    out = np.zeros((n, RECORD_FLOATS), dtype=np.float32)
    have = 0
    while have < n:
        m = max(1024, 2 * (n - have))
        mtt = rng.uniform(350.0, 1000.0, m)
        mt1 = _bw_mass_v(rng, P["mt"], P["wt"], 15.0, m)
        mt2 = _bw_mass_v(rng, P["mt"], P["wt"], 15.0, m)
        mw1 = _bw_mass_v(rng, P["mw"], P["ww"], 15.0, m)
        mw2 = _bw_mass_v(rng, P["mw"], P["ww"], 15.0, m)
        y = rng.uniform(-1.5, 1.5, m)
        ok = mt1 + mt2 < mtt
        mtt = np.where(ok, mtt, mt1 + mt2 + 1.0)
        sysp = np.stack([mtt * np.cosh(y), 0 * y, 0 * y, mtt * np.sinh(y)], axis=1)
        t, tb = _two_body_v(rng, mtt, mt1, mt2)
        t, tb = _boost_v(t, sysp), _boost_v(tb, sysp)
        b, wp = _two_body_v(rng, mt1, 0.0, mw1)
        b, wp = _boost_v(b, t), _boost_v(wp, t)
        lep, nu = _two_body_v(rng, mw1, 0.0, 0.0)
        lep, nu = _boost_v(lep, wp), _boost_v(nu, wp)
        bb, wm = _two_body_v(rng, mt2, 0.0, mw2)
        bb, wm = _boost_v(bb, tb), _boost_v(wm, tb)
        d, ub = _two_body_v(rng, mw2, 0.0, 0.0)
        d, ub = _boost_v(d, wm), _boost_v(ub, wm)
        for q in (lep, b, bb, d, ub):
            ok &= np.abs(_eta_phi_v(q)[0]) <= 2.5
        for q in (b, bb, d, ub):
            ok &= q[:, 0] >= 20.0
        swap = (bb[:, 0] > b[:, 0])[:, None]   # object 1 = the more energetic b quark
        objs = [lep, np.where(swap, bb, b), np.where(swap, b, bb), d, ub, nu]
        kinds = [KIND_E_PLUS, KIND_JET, KIND_JET, KIND_JET, KIND_JET, KIND_NU]
        idx = np.nonzero(ok)[0][: n - have]
        r = out[have: have + len(idx)]
        for slot, q in enumerate(objs):
            eta, phi, _ = _eta_phi_v(q[idx])
            r[:, 4 * slot] = q[idx, 0]
            r[:, 4 * slot + 1] = eta
            r[:, 4 * slot + 2] = phi
            r[:, 4 * slot + 3] = kinds[slot]
        r[:, 24] = nu[idx, 1]
        r[:, 25] = nu[idx, 2]
        r[:, 26] = 6
        r[:, 27] = PROC_TTBAR
        r[:, 28] = swap[idx, 0].astype(np.float32)
        r[:, 29] = 1.0
        have += len(idx)
    return out


def gen_ttbar_dilep(n, seed, tf=None, truth=False):
    """Dilepton ttbar events, t -> b l+ nu, tbar -> bbar mu- nubar (the final state of
    the paper's hadron-level analysis without the Higgs, Sec. 3-4): the production
    and decay chain of gen_ttbar; leptons exact within |eta| <= 2.5; the two b
    jets within |eta| <= 2.5 and E >= 20 GeV, smeared by the double Gaussian and
    stored by decreasing measured energy; MET = nu_T + nubar_T + N(0, 15^2).
    Record: objects 0 l+ (e+), 1 mu-, 2 and 3 the b jets; [24], [25] MET;
    [26] = 4; [27] = 3; [28] = 0 if object 2 is the b quark, else 1.
    With truth=True also returns the (n, 6, 4) parton momenta (E, px, py, pz) of
    b, bbar, l+, mu-, nu, nubar."""
    tf = tf or DEFAULT_TF[PROC_TTBAR]
    P = DEFAULT_PROCESS
    rng = np.random.Generator(np.random.Philox(seed))
    out = np.zeros((n, RECORD_FLOATS), dtype=np.float32)
    tr = np.zeros((n, 6, 4))
    have = 0
    while have < n:
        m = max(1024, 2 * (n - have))
        mtt = rng.uniform(350.0, 1000.0, m)
        mt1 = _bw_mass_v(rng, P["mt"], P["wt"], 15.0, m)
        mt2 = _bw_mass_v(rng, P["mt"], P["wt"], 15.0, m)
        mw1 = _bw_mass_v(rng, P["mw"], P["ww"], 15.0, m)
        mw2 = _bw_mass_v(rng, P["mw"], P["ww"], 15.0, m)
        y = rng.uniform(-1.5, 1.5, m)
        ok = mt1 + mt2 < mtt
        mtt = np.where(ok, mtt, mt1 + mt2 + 1.0)
        sysp = np.stack([mtt * np.cosh(y), 0 * y, 0 * y, mtt * np.sinh(y)], axis=1)
        t, tb = _two_body_v(rng, mtt, mt1, mt2)
        t, tb = _boost_v(t, sysp), _boost_v(tb, sysp)
        b, wp = _two_body_v(rng, mt1, 0.0, mw1)
        b, wp = _boost_v(b, t), _boost_v(wp, t)
        lp, nu = _two_body_v(rng, mw1, 0.0, 0.0)
        lp, nu = _boost_v(lp, wp), _boost_v(nu, wp)
        bb, wm = _two_body_v(rng, mt2, 0.0, mw2)
        bb, wm = _boost_v(bb, tb), _boost_v(wm, tb)
        lm, nub = _two_body_v(rng, mw2, 0.0, 0.0)
        lm, nub = _boost_v(lm, wm), _boost_v(nub, wm)
        for q in (lp, lm, b, bb):
            ok &= np.abs(_eta_phi_v(q)[0]) <= 2.5
        def smear(q):
            rel = np.where(rng.uniform(size=m) < tf["jet_tail_w"], tf["jet_tail"], tf["jet_core"])
            return q[:, 0] * (1.0 + rel * rng.standard_normal(m))
        Eb, Ebb = smear(b), smear(bb)
        ok &= (Eb >= 20.0) & (Ebb >= 20.0)
        swap = Ebb > Eb
        idx = np.nonzero(ok)[0][: n - have]
        r = out[have: have + len(idx)]
        for slot, (q, kind) in enumerate(((lp, KIND_E_PLUS), (lm, KIND_MU_MINUS))):
            eta, phi, _ = _eta_phi_v(q[idx])
            r[:, 4 * slot] = q[idx, 0]
            r[:, 4 * slot + 1] = eta
            r[:, 4 * slot + 2] = phi
            r[:, 4 * slot + 3] = kind
        first = np.where(swap[:, None], bb, b)[idx]
        second = np.where(swap[:, None], b, bb)[idx]
        E1 = np.where(swap, Ebb, Eb)[idx]
        E2 = np.where(swap, Eb, Ebb)[idx]
        for slot, q, E in ((2, first, E1), (3, second, E2)):
            eta, phi, _ = _eta_phi_v(q)
            r[:, 4 * slot] = E
            r[:, 4 * slot + 1] = eta
            r[:, 4 * slot + 2] = phi
            r[:, 4 * slot + 3] = KIND_JET
        r[:, 24] = (nu[idx, 1] + nub[idx, 1]) + tf["met_sigma"] * rng.standard_normal(len(idx))
        r[:, 25] = (nu[idx, 2] + nub[idx, 2]) + tf["met_sigma"] * rng.standard_normal(len(idx))
        r[:, 26] = 4
        r[:, 27] = PROC_TTBAR_DILEP
        r[:, 28] = swap[idx].astype(np.float32)
        for k, q in enumerate((b, bb, lp, lm, nu, nub)):
            tr[have: have + len(idx), k] = q[idx]
        have += len(idx)
    return (out, tr) if truth else out


PROC_TTH_DILEP = 4


def tth_perm_index(jb, jbb):
    """Assignment index (0..11) of the dilepton ttH records: jets jb and jbb (0..3,
    objects 2..5) are the b and the bbar, the other two the Higgs pair (unordered)."""
    rest = [j for j in range(4) if j != jb]
    return 3 * jb + rest.index(jbb)


def gen_tth_dilep(n, seed, tf=None, truth=False, pair_mass=None):
    """Dilepton ttH events (Sec. 3-4, the signal of the paper's hadron-level
    analysis): t -> b e+ nu, tbar -> bbar mu- nubar, H -> b bbar. Partonic mass
    uniform in [m_t1 + m_t2 + m_H + 20 GeV, 1500 GeV], rapidity U[-1, 1]; the t tbar
    system mass uniform over its allowed range, two-body splittings isotropic; t, W
    masses from Breit-Wigners truncated at +-15 widths, m_H fixed (its width is
    4 MeV). Leptons exact within |eta| <= 2.5; the four b jets within |eta| <= 2.5 and
    E >= 20 GeV after double-Gaussian smearing, stored by decreasing measured energy.
    Record: objects 0 e+, 1 mu-, 2..5 the b jets; [24], [25] MET = nu_T + nubar_T +
    N(0, 15^2); [26] = 6; [27] = 4; [28] = tth_perm_index of the true b and bbar jets.
    With truth=True also returns the (n, 8, 4) parton momenta of b, bbar, e+, mu-, nu,
    nubar, b(H), bbar(H). pair_mass = (lo, hi): the extra pair's mass uniform over
    [lo, hi] instead of m_H, and [27] = 5 (the ttbb background's stand-in events)."""
    tf = tf or DEFAULT_TF[PROC_TTBAR]
    P = DEFAULT_PROCESS
    mh = P["mh"]
    rng = np.random.Generator(np.random.Philox(seed))
    out = np.zeros((n, RECORD_FLOATS), dtype=np.float32)
    tr = np.zeros((n, 8, 4))
    have = 0
    while have < n:
        m = max(1024, 2 * (n - have))
        mt1 = _bw_mass_v(rng, P["mt"], P["wt"], 15.0, m)
        mt2 = _bw_mass_v(rng, P["mt"], P["wt"], 15.0, m)
        mw1 = _bw_mass_v(rng, P["mw"], P["ww"], 15.0, m)
        mw2 = _bw_mass_v(rng, P["mw"], P["ww"], 15.0, m)
        mp = np.full(m, mh) if pair_mass is None else rng.uniform(pair_mass[0], pair_mass[1], m)
        rs = rng.uniform(0.0, 1.0, m) * (1500.0 - (mt1 + mt2 + mp + 20.0)) + mt1 + mt2 + mp + 20.0
        mtt = rng.uniform(0.0, 1.0, m) * (rs - mp - 1.0 - (mt1 + mt2 + 1.0)) + mt1 + mt2 + 1.0
        y = rng.uniform(-1.0, 1.0, m)
        sysp = np.stack([rs * np.cosh(y), 0 * y, 0 * y, rs * np.sinh(y)], axis=1)
        hq, ttq = _two_body_v(rng, rs, mp, mtt)
        t, tb = _two_body_v(rng, mtt, mt1, mt2)
        t, tb = _boost_v(t, ttq), _boost_v(tb, ttq)
        hq, t, tb = _boost_v(hq, sysp), _boost_v(t, sysp), _boost_v(tb, sysp)
        b, wp = _two_body_v(rng, mt1, 0.0, mw1)
        b, wp = _boost_v(b, t), _boost_v(wp, t)
        lp, nu = _two_body_v(rng, mw1, 0.0, 0.0)
        lp, nu = _boost_v(lp, wp), _boost_v(nu, wp)
        bb, wm = _two_body_v(rng, mt2, 0.0, mw2)
        bb, wm = _boost_v(bb, tb), _boost_v(wm, tb)
        lm, nub = _two_body_v(rng, mw2, 0.0, 0.0)
        lm, nub = _boost_v(lm, wm), _boost_v(nub, wm)
        h1, h2 = _two_body_v(rng, mp, 0.0, 0.0)
        h1, h2 = _boost_v(h1, hq), _boost_v(h2, hq)
        ok = np.ones(m, dtype=bool)
        for q in (lp, lm, b, bb, h1, h2):
            ok &= np.abs(_eta_phi_v(q)[0]) <= 2.5

        def smear(q):
            rel = np.where(rng.uniform(size=m) < tf["jet_tail_w"], tf["jet_tail"], tf["jet_core"])
            return q[:, 0] * (1.0 + rel * rng.standard_normal(m))
        quarks = (b, bb, h1, h2)
        Em = np.stack([smear(q) for q in quarks], axis=1)          # (m, 4) measured energies
        ok &= np.all(Em >= 20.0, axis=1)
        idx = np.nonzero(ok)[0][: n - have]
        r = out[have: have + len(idx)]
        for slot, (q, kind) in enumerate(((lp, KIND_E_PLUS), (lm, KIND_MU_MINUS))):
            eta, phi, _ = _eta_phi_v(q[idx])
            r[:, 4 * slot] = q[idx, 0]
            r[:, 4 * slot + 1] = eta
            r[:, 4 * slot + 2] = phi
            r[:, 4 * slot + 3] = kind
        order = np.argsort(-Em[idx], axis=1)                        # jets by decreasing E
        for k in range(4):
            src = order[:, k]
            Ek = Em[idx, src]
            qk = np.stack([quarks[j][idx] for j in range(4)], axis=1)[np.arange(len(idx)), src]
            eta, phi, _ = _eta_phi_v(qk)
            r[:, 4 * (2 + k)] = Ek
            r[:, 4 * (2 + k) + 1] = eta
            r[:, 4 * (2 + k) + 2] = phi
            r[:, 4 * (2 + k) + 3] = KIND_JET
        r[:, 24] = (nu[idx, 1] + nub[idx, 1]) + tf["met_sigma"] * rng.standard_normal(len(idx))
        r[:, 25] = (nu[idx, 2] + nub[idx, 2]) + tf["met_sigma"] * rng.standard_normal(len(idx))
        r[:, 26] = 6
        r[:, 27] = PROC_TTH_DILEP if pair_mass is None else 5
        slot_of = np.argsort(order, axis=1)                         # quark -> jet slot
        r[:, 28] = [tth_perm_index(int(a), int(c)) for a, c in zip(slot_of[:, 0], slot_of[:, 1])]
        for k, q in enumerate((b, bb, lp, lm, nu, nub, h1, h2)):
            tr[have: have + len(idx), k] = q[idx]
        have += len(idx)
    return (out, tr) if truth else out


PROC_TTBB_DILEP = 5


def gen_ttbb_dilep(n, seed, tf=None, truth=False):
    """Stand-in dilepton ttbb events: the ttH chain with the extra b bbar pair's mass
    uniform in [20, 300] GeV (a continuum instead of the Higgs peak); record layout as
    for gen_tth_dilep with [27] = 5."""
    return gen_tth_dilep(n, seed, tf=tf, truth=truth, pair_mass=(20.0, 300.0))


GENERATORS = {PROC_DY: gen_dy, PROC_W: gen_w, PROC_TTBAR: gen_ttbar,
              PROC_TTBAR_DILEP: gen_ttbar_dilep, PROC_TTH_DILEP: gen_tth_dilep,
              PROC_TTBB_DILEP: gen_ttbb_dilep}


def gen_events(proc, n, seed):
    return GENERATORS[proc](n, seed)


def gen_mix(n, seed, fractions=(0.5, 0.3, 0.2)):
    """Uneven batch: events drawn from the three processes with the given
    fractions, shuffled with a seeded permutation."""
    counts = [int(round(f * n)) for f in fractions]
    counts[0] += n - sum(counts)
    parts = [gen_events(p, c, seed + 1000 * (p + 1)) for p, c in enumerate(counts)]
    recs = np.concatenate(parts, axis=0)
    perm = np.random.Generator(np.random.Philox(seed)).permutation(n)
    return recs[perm]

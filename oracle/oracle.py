"""ctypes binding of the FP64 CPU oracle (oracle/*.c).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and the cpu_baseline
and reference legs of bench.py are the only users. The CUDA product path never
imports this module.

The oracle is compiled with gcc into oracle/liboracle.so by build(); load()
builds it on first use if the shared object is missing or older than a source.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SOURCES = ["ora_philox.c", "ora_dirac.c", "ora_matrix.c", "ora_process.c", "ora_vegas.c",
           "ora_integrate.c", "ora_dilep.c", "ora_ttbb.c"]
NG = 128
REC = 32


class OraProcess(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("sqrt_s", C.c_double),
                ("mz", C.c_double), ("wz", C.c_double), ("mw", C.c_double), ("ww", C.c_double),
                ("mt", C.c_double), ("wt", C.c_double), ("alpha", C.c_double),
                ("sw2", C.c_double), ("alpha_s", C.c_double), ("pdf_A", C.c_double * 3),
                ("pdf_a", C.c_double * 3), ("pdf_b", C.c_double * 3),
                ("pdf_grid", C.POINTER(C.c_double)), ("grid_nx", C.c_int32),
                ("grid_nq", C.c_int32), ("grid_lx", C.c_double * 2), ("grid_lq", C.c_double * 2),
                ("mh", C.c_double), ("wh", C.c_double), ("mb", C.c_double)]


class OraTF(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("lep_rel", "window_k", "jet_core", "jet_tail",
                                          "jet_tail_w", "jet_lo_div", "jet_hi_mul",
                                          "met_sigma", "met_box_k")]


class OraOpts(C.Structure):
    _fields_ = [("n_adapt_iters", C.c_int32), ("n_threads", C.c_int32),
                ("adapt_points", C.c_uint64), ("alpha", C.c_double),
                ("grid_in", C.POINTER(C.c_double)), ("event_id_base", C.c_uint64),
                ("strat_points", C.c_int32), ("pad", C.c_int32)]


def _stale():
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in SOURCES + ["oracle.h",
                                                                               "ora_dirac.h"])


def build(force=False):
    """Compile the oracle with gcc (plain C11, -O2, no target-specific flags)."""
    if not force and not _stale():
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp] + \
          [os.path.join(HERE, s) for s in SOURCES] + ["-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None
_dp = C.POINTER(C.c_double)


def load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(LIB_PATH)
    P, T = C.POINTER(OraProcess), C.POINTER(OraTF)
    fp = C.POINTER(C.c_float)
    u32p = C.POINTER(C.c_uint32)
    lib.ora_philox4x32_10.argtypes = [u32p, u32p, u32p]
    lib.ora_u01.argtypes = [C.c_uint32]
    lib.ora_u01.restype = C.c_double
    lib.ora_point_u.argtypes = [C.c_uint64, C.c_uint64, C.c_int, C.c_uint64, C.c_int, _dp]
    lib.ora_point_u_tag.argtypes = [C.c_uint64, C.c_uint64, C.c_int, C.c_uint64, C.c_int,
                                    C.c_int, _dp]
    lib.ora_integrand.argtypes = [P, T, fp, C.c_int, _dp]
    lib.ora_integrand.restype = C.c_double
    lib.ora_kinematics.argtypes = [P, T, fp, C.c_int, _dp, C.c_int, _dp, _dp, _dp, _dp]
    lib.ora_kinematics.restype = C.c_int
    lib.ora_msq_dy.argtypes = [P, C.c_int, _dp, _dp, _dp, _dp]
    lib.ora_msq_dy.restype = C.c_double
    lib.ora_msq_w.argtypes = [P, C.c_int, _dp, _dp, _dp, _dp]
    lib.ora_msq_w.restype = C.c_double
    lib.ora_integrand_roots.argtypes = [P, T, fp, C.c_int, _dp, _dp]
    lib.ora_flavour_msq.argtypes = [P, _dp, _dp, C.c_double, C.c_double, fp]
    lib.ora_flavour_msq.restype = C.c_double
    lib.ora_discriminant.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, _dp, _dp]
    lib.ora_dilep_nu.argtypes = [_dp, _dp, _dp, _dp] + [C.c_double] * 6 + [_dp, _dp, _dp]
    lib.ora_strat_side.argtypes = [C.c_uint64, C.c_int, C.c_int]
    lib.ora_strat_side.restype = C.c_uint64
    lib.ora_pdf_q.argtypes = [P, C.c_int, C.c_double, C.c_double]
    lib.ora_pdf_q.restype = C.c_double
    lib.ora_density.argtypes = [P, C.c_int, _dp, fp, _dp]
    lib.ora_density.restype = C.c_double
    lib.ora_parton_ttbar.argtypes = [P, fp, C.c_int, _dp]
    lib.ora_parton_ttbar.restype = C.c_double
    lib.ora_parton_batch.argtypes = [P, fp, C.c_int64, C.c_int, _dp, _dp]
    lib.ora_msq_ttbar.argtypes = [P, C.c_int] + [_dp] * 8
    lib.ora_msq_ttbar.restype = C.c_double
    lib.ora_msq_ttbar_production.argtypes = [P, C.c_int, _dp, _dp, _dp, _dp]
    lib.ora_msq_ttbar_production.restype = C.c_double
    lib.ora_ttbar_gauge_probe.argtypes = [P, _dp, _dp, _dp, _dp, C.c_int, C.c_int]
    lib.ora_ttbar_gauge_probe.restype = C.c_double
    lib.ora_msq_tth_production.argtypes = [P, C.c_int, _dp, _dp, _dp, _dp, _dp]
    lib.ora_msq_tth_production.restype = C.c_double
    lib.ora_tth_gauge_probe.argtypes = [P, _dp, _dp, _dp, _dp, _dp, C.c_int, C.c_int]
    lib.ora_msq_tth.argtypes = [P, C.c_int] + [_dp] * 10
    lib.ora_msq_tth.restype = C.c_double
    lib.ora_msq_ttbb_production.argtypes = [P, C.c_int] + [_dp] * 6
    lib.ora_msq_ttbb_production.restype = C.c_double
    lib.ora_ttbb_gauge_probe.argtypes = [P] + [_dp] * 6 + [C.c_int, C.c_int]
    lib.ora_ttbb_gauge_probe.restype = C.c_double
    lib.ora_ttbb_qq_ward_probe.argtypes = [P] + [_dp] * 7
    lib.ora_ttbb_qq_ward_probe.restype = None
    lib.ora_msq_ttbb.argtypes = [P, C.c_int] + [_dp] * 10
    lib.ora_msq_ttbb.restype = C.c_double
    lib.ora_ttbb_colour_matrices.argtypes = [_dp, _dp]
    lib.ora_ttbb_colour_matrices.restype = None
    lib.ora_su3_check.argtypes = [_dp]
    lib.ora_su3_check.restype = None
    lib.ora_tth_gauge_probe.restype = C.c_double
    lib.ora_top_decay_probe.argtypes = [P, _dp, _dp, _dp, _dp]
    lib.ora_antitop_decay_probe.argtypes = [P, _dp, _dp, _dp, _dp]
    lib.ora_pdf.argtypes = [P, C.c_int, C.c_double]
    lib.ora_pdf.restype = C.c_double
    lib.ora_grid_uniform.argtypes = [C.c_int, _dp]
    lib.ora_vegas_map.argtypes = [C.c_int, _dp, _dp, _dp, C.POINTER(C.c_int)]
    lib.ora_vegas_map.restype = C.c_double
    lib.ora_vegas_refine.argtypes = [C.c_int, _dp, _dp, C.c_double, _dp]
    lib.ora_eval_points.argtypes = [P, T, fp, C.c_uint64, C.c_int, C.c_uint64, C.c_uint64,
                                    C.c_int64, _dp, _dp]
    lib.ora_integrate.argtypes = [P, T, fp, C.c_int64, C.c_uint64, C.c_uint64,
                                  C.POINTER(OraOpts), _dp, _dp, C.POINTER(C.c_uint64), _dp,
                                  _dp, _dp]
    lib.ora_integrate.restype = C.c_int
    lib.ora_dims.argtypes = [C.c_int]
    lib.ora_nperm.argtypes = [C.c_int]
    _lib = lib
    return lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def process(kind, params, pdf_grid=None):
    """Process parameters; pdf_grid (optional) = dict(table=(3, nq, nx) array of
    f(x_i, Q_j) for quark, antiquark, gluon, lx=(ln x_min, ln x_max),
    lq=(ln Q_min, ln Q_max)) replaces the parametric PDFs."""
    p = OraProcess()
    p.kind = kind
    for k in ("sqrt_s", "mz", "wz", "mw", "ww", "mt", "wt", "alpha", "sw2", "alpha_s"):
        setattr(p, k, float(params[k]))
    for k in ("pdf_A", "pdf_a", "pdf_b"):
        getattr(p, k)[:] = [float(v) for v in params[k]]
    for k in ("mh", "wh", "mb"):   # Higgs parameters (ttH); absent for the other processes
        setattr(p, k, float(params.get(k, 0.0)))
    if pdf_grid is not None:
        t = np.ascontiguousarray(pdf_grid["table"], dtype=np.float64)
        assert t.ndim == 3 and t.shape[0] == 3 and t.shape[1] >= 2 and t.shape[2] >= 2
        p._table = t  # keeps the array alive with the structure
        p.pdf_grid = t.ctypes.data_as(_dp)
        p.grid_nq, p.grid_nx = t.shape[1], t.shape[2]
        p.grid_lx[:] = [float(v) for v in pdf_grid["lx"]]
        p.grid_lq[:] = [float(v) for v in pdf_grid["lq"]]
    return p


def tf(params):
    t = OraTF()
    for k, _ in OraTF._fields_:
        setattr(t, k, float(params[k]))
    return t


def dims(kind):
    return load().ora_dims(kind)


def nperm(kind):
    return load().ora_nperm(kind)


def philox(ctr, key):
    lib = load()
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib.ora_philox4x32_10(c, k, o)
    return list(o)


def point_u(seed, event_id, perm, idx, d, tag=0):
    u = np.zeros(d)
    load().ora_point_u_tag(seed, event_id, perm, idx, d, tag, u.ctypes.data_as(_dp))
    return u


def _rec_ptr(rec):
    rec = np.ascontiguousarray(rec, dtype=np.float32)
    return rec, rec.ctypes.data_as(C.POINTER(C.c_float))


def integrand(P, T, rec, perm, x):
    rec, rp = _rec_ptr(rec)
    x, xp = _d(x)
    return load().ora_integrand(C.byref(P), C.byref(T), rp, perm, xp)


def kinematics(P, T, rec, perm, x, root):
    rec, rp = _rec_ptr(rec)
    x, xp = _d(x)
    fs = np.zeros(32)
    lab = np.zeros(32)
    k12 = np.zeros(8)
    aux = np.zeros(8)
    n = load().ora_kinematics(C.byref(P), C.byref(T), rp, perm, xp, root,
                              fs.ctypes.data_as(_dp), lab.ctypes.data_as(_dp),
                              k12.ctypes.data_as(_dp), aux.ctypes.data_as(_dp))
    nfs = 2 if P.kind < 2 else (8 if P.kind >= 4 else 6)
    return {"n": n, "fs": fs.reshape(8, 4)[:nfs], "lab": lab.reshape(8, 4)[:nfs], "k12": k12.reshape(2, 4),
            "aux": aux}


def integrand_roots(P, T, rec, perm, x):
    """Per-root contributions of the integrand at x (a list of 0-2 floats)."""
    rec, rp = _rec_ptr(rec)
    x, xp = _d(x)
    w = np.zeros(8)
    n = load().ora_integrand_roots(C.byref(P), C.byref(T), rp, perm, xp, w.ctypes.data_as(_dp))
    return list(w[:n])


def flavour_msq(P, fs, k12, x1, x2, rec):
    """PDF-weighted, flavour-summed |M|^2 at the parton-frame momenta fs (6, 4) and
    k12 (2, 4), with the record supplying the lepton charge where it matters."""
    rec, rp = _rec_ptr(rec)
    f8 = np.zeros((8, 4))
    f8[:len(fs)] = np.asarray(fs)
    fs, fp_ = _d(f8.reshape(-1))
    k12, kp = _d(np.asarray(k12).reshape(-1))
    return load().ora_flavour_msq(C.byref(P), fp_, kp, x1, x2, rp)


def pdf_q(P, t, x, Q):
    return load().ora_pdf_q(C.byref(P), t, x, Q)


def density(P, lab, rec=None):
    """Density at lab-frame final-state momenta lab (nfs, 4) with delta-function
    transfer functions and no change of variables; returns (density, aux = (x1, x2,
    s-hat, PDF-weighted |M|^2)). rec (optional) supplies the W lepton charge."""
    lab = np.ascontiguousarray(lab, dtype=np.float64).reshape(-1, 4)
    if rec is None:
        rec = np.zeros(REC, dtype=np.float32)
    rec, rp = _rec_ptr(rec)
    aux = np.zeros(4)
    w = load().ora_density(C.byref(P), lab.shape[0], lab.ctypes.data_as(_dp), rp,
                           aux.ctypes.data_as(_dp))
    return w, aux


def parton_ttbar(P, rec, bperm):
    """Parton-level ttbar weight of one record and b-quark assignment (Sec. 4);
    returns (weight, aux = (x1, x2, s-hat, PDF-weighted |M|^2))."""
    rec, rp = _rec_ptr(rec)
    aux = np.zeros(4)
    w = load().ora_parton_ttbar(C.byref(P), rp, bperm, aux.ctypes.data_as(_dp))
    return w, aux


def parton_batch(P, recs, n_threads=None):
    """Parton-level weights of many records: (prob (n,), w (n, 2))."""
    recs = np.ascontiguousarray(recs, dtype=np.float32).reshape(-1, REC)
    n = recs.shape[0]
    prob = np.zeros(n)
    w = np.zeros((n, 2))
    load().ora_parton_batch(C.byref(P), recs.ctypes.data_as(C.POINTER(C.c_float)), n,
                            n_threads or os.cpu_count() or 1, prob.ctypes.data_as(_dp),
                            w.ctypes.data_as(_dp))
    return prob, w


def msq_dy(P, flavour, kq, kqb, plm, plp):
    args = [_d(v) for v in (kq, kqb, plm, plp)]
    return load().ora_msq_dy(C.byref(P), flavour, *[a[1] for a in args])


def msq_w(P, charge, kq, kqb, pl, pn):
    args = [_d(v) for v in (kq, kqb, pl, pn)]
    return load().ora_msq_w(C.byref(P), charge, *[a[1] for a in args])


def msq_ttbar(P, channel, k1, k2, pb, pl, pn, pbb, pd, pu):
    args = [_d(v) for v in (k1, k2, pb, pl, pn, pbb, pd, pu)]
    return load().ora_msq_ttbar(C.byref(P), channel, *[a[1] for a in args])


def msq_tth_production(P, channel, k1, k2, pt, ptb, pH):
    args = [_d(v) for v in (k1, k2, pt, ptb, pH)]
    return load().ora_msq_tth_production(C.byref(P), channel, *[a[1] for a in args])


def msq_tth(P, channel, k1, k2, pb, pl, pn, pbb, pm, pnb, ph1, ph2):
    args = [_d(v) for v in (k1, k2, pb, pl, pn, pbb, pm, pnb, ph1, ph2)]
    return load().ora_msq_tth(C.byref(P), channel, *[a[1] for a in args])


def msq_ttbb_production(P, channel, k1, k2, p1, p2, p3, p4):
    args = [_d(v) for v in (k1, k2, p1, p2, p3, p4)]
    return load().ora_msq_ttbb_production(C.byref(P), channel, *[a[1] for a in args])


def ttbb_gauge_probe(P, k1, k2, p1, p2, p3, p4, which, hel):
    args = [_d(v) for v in (k1, k2, p1, p2, p3, p4)]
    return load().ora_ttbb_gauge_probe(C.byref(P), *[a[1] for a in args], which, hel)


def ttbb_qq_ward_probe(P, k1, k2, p1, p2, p3, p4):
    args = [_d(v) for v in (k1, k2, p1, p2, p3, p4)]
    out = np.zeros(2)
    load().ora_ttbb_qq_ward_probe(C.byref(P), *[a[1] for a in args], out.ctypes.data_as(_dp))
    return out


def msq_ttbb(P, channel, k1, k2, pb, pl, pn, pbb, pm, pnb, p3, p4):
    args = [_d(v) for v in (k1, k2, pb, pl, pn, pbb, pm, pnb, p3, p4)]
    return load().ora_msq_ttbb(C.byref(P), channel, *[a[1] for a in args])


def ttbb_colour_matrices():
    kgg = np.zeros(38 * 38 * 2)
    kqq = np.zeros(7 * 7 * 2)
    load().ora_ttbb_colour_matrices(kgg.ctypes.data_as(_dp), kqq.ctypes.data_as(_dp))
    return kgg.view(np.complex128).reshape(38, 38), kqq.view(np.complex128).reshape(7, 7)


def su3_check():
    out = np.zeros(5)
    load().ora_su3_check(out.ctypes.data_as(_dp))
    return out


def tth_gauge_probe(P, k1, k2, pt, ptb, pH, which, hel):
    args = [_d(v) for v in (k1, k2, pt, ptb, pH)]
    return load().ora_tth_gauge_probe(C.byref(P), *[a[1] for a in args], which, hel)


def msq_ttbar_production(P, channel, k1, k2, pt, ptb):
    args = [_d(v) for v in (k1, k2, pt, ptb)]
    return load().ora_msq_ttbar_production(C.byref(P), channel, *[a[1] for a in args])


def ttbar_gauge_probe(P, k1, k2, pt, ptb, which, hel):
    args = [_d(v) for v in (k1, k2, pt, ptb)]
    return load().ora_ttbar_gauge_probe(C.byref(P), *[a[1] for a in args], which, hel)


def top_decay_probe(P, pb, pl, pn, anti=False):
    args = [_d(v) for v in (pb, pl, pn)]
    out = np.zeros(2)
    f = load().ora_antitop_decay_probe if anti else load().ora_top_decay_probe
    f(C.byref(P), *[a[1] for a in args], out.ctypes.data_as(_dp))
    return out


def pdf(P, typ, x):
    return load().ora_pdf(C.byref(P), typ, x)


def grid_uniform(d):
    g = np.zeros(d * (NG + 1))
    load().ora_grid_uniform(d, g.ctypes.data_as(_dp))
    return g.reshape(d, NG + 1)


def vegas_map(grid, u):
    grid, gp = _d(grid)
    u, up = _d(u)
    d = grid.shape[0]
    x = np.zeros(d)
    bins = (C.c_int * d)()
    J = load().ora_vegas_map(d, gp, up, x.ctypes.data_as(_dp), bins)
    return x, J, list(bins)


def vegas_refine(hist, grid, alpha=1.5):
    hist, hp = _d(hist)
    grid, gp = _d(grid)
    d = grid.shape[0]
    out = np.zeros_like(grid)
    load().ora_vegas_refine(d, hp, gp, alpha, out.ctypes.data_as(_dp))
    return out


def eval_points(P, T, rec, event_id, perm, seed, point0, n, grid=None):
    rec, rp = _rec_ptr(rec)
    w = np.zeros(n)
    gp = None
    if grid is not None:
        grid, gp = _d(grid)
    load().ora_eval_points(C.byref(P), C.byref(T), rp, event_id, perm, seed, point0, n, gp,
                           w.ctypes.data_as(_dp))
    return w


def dilep_nu(pb, pbb, plp, plm, met, q2wp, q2wm, q2t, q2tb):
    """Neutrino solutions of the dilepton ttbar constraints: list of (nu, nubar, jac)
    with nu, nubar = (E, px, py, pz)."""
    args = [_d(v) for v in (pb, pbb, plp, plm)]
    nu = np.zeros(16)
    nb = np.zeros(16)
    jac = np.zeros(4)
    n = load().ora_dilep_nu(*[a[1] for a in args], float(met[0]), float(met[1]), q2wp, q2wm,
                            q2t, q2tb, nu.ctypes.data_as(_dp), nb.ctypes.data_as(_dp),
                            jac.ctypes.data_as(_dp))
    return [(nu[4 * i:4 * i + 4].copy(), nb[4 * i:4 * i + 4].copy(), jac[i]) for i in range(n)]


def discriminant(p_s, e_s, p_b, e_b):
    """(D, sigma_D, status) of one event."""
    D, e = C.c_double(), C.c_double()
    rc = load().ora_discriminant(p_s, e_s, p_b, e_b, C.byref(D), C.byref(e))
    return D.value, e.value, rc


def strat_side(n, d, k):
    return load().ora_strat_side(n, d, k)


def integrate(P, T, recs, seed, n_points, n_adapt_iters=5, adapt_points=0, alpha=1.5,
              grid_in=None, event_id_base=0, n_threads=None, want_items=False,
              want_grids=False, strat_points=0):
    recs = np.ascontiguousarray(recs, dtype=np.float32).reshape(-1, REC)
    n = recs.shape[0]
    npm = nperm(P.kind)
    d = dims(P.kind)
    o = OraOpts()
    o.n_adapt_iters = n_adapt_iters
    o.n_threads = n_threads or os.cpu_count() or 1
    o.adapt_points = adapt_points
    o.alpha = alpha
    o.event_id_base = event_id_base
    o.strat_points = strat_points
    keep = None
    if grid_in is not None:
        keep, gp = _d(grid_in)
        o.grid_in = gp
    prob = np.zeros(n)
    err = np.zeros(n)
    used = np.zeros(n, dtype=np.uint64)
    im = np.zeros(n * npm)
    ie = np.zeros(n * npm)
    go = np.zeros(n * npm * d * (NG + 1)) if want_grids else None
    rc = load().ora_integrate(C.byref(P), C.byref(T),
                              recs.ctypes.data_as(C.POINTER(C.c_float)), n, seed, n_points,
                              C.byref(o), prob.ctypes.data_as(_dp), err.ctypes.data_as(_dp),
                              used.ctypes.data_as(C.POINTER(C.c_uint64)), im.ctypes.data_as(_dp),
                              ie.ctypes.data_as(_dp),
                              go.ctypes.data_as(_dp) if go is not None else None)
    del keep
    if rc != 0:
        raise ValueError("oracle: n_points too small for the adaptation plan")
    out = {"prob": prob, "err": err, "n_used": used}
    if want_items:
        out["item_mean"] = im
        out["item_err"] = ie
    if want_grids:
        out["grids"] = go.reshape(n * npm, d, NG + 1)
    return out

"""Thin ctypes binding of libmem.so (declarations in include/mem.h).

Argument marshalling only: every step of the integration runs in the CUDA
library. Functions keep the C names (mem_create_process, mem_upload_events,
mem_integrate, mem_destroy, ...). Device arrays are passed as torch CUDA
tensors (data_ptr), host arrays as numpy arrays. If the library has not been
built, lib() raises; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmem.so")

MEM_OK, MEM_ERR_INVALID_ARG, MEM_ERR_CUDA, MEM_ERR_OOM, MEM_ERR_NONFINITE, \
    MEM_NOT_CONVERGED, MEM_ERR_TIMEOUT = range(7)
MEM_PROC_DY, MEM_PROC_W, MEM_PROC_TTBAR = 0, 1, 2
NG = 128
REC = 32


class MemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mem status {status}: {msg}")
        self.status = status


class mem_process_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("sqrt_s", C.c_double),
                ("mz", C.c_double), ("wz", C.c_double), ("mw", C.c_double), ("ww", C.c_double),
                ("mt", C.c_double), ("wt", C.c_double), ("alpha", C.c_double),
                ("sw2", C.c_double), ("alpha_s", C.c_double), ("pdf_A", C.c_double * 3),
                ("pdf_a", C.c_double * 3), ("pdf_b", C.c_double * 3),
                ("mh", C.c_double), ("wh", C.c_double), ("mb", C.c_double)]


class mem_tf_desc(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("lep_rel", "window_k", "jet_core", "jet_tail",
                                          "jet_tail_w", "jet_lo_div", "jet_hi_mul",
                                          "met_sigma", "met_box_k")]


class mem_plan(C.Structure):
    _fields_ = [("n_adapt_iters", C.c_int32), ("tiles_per_cta", C.c_int32),
                ("adapt_points", C.c_uint64), ("min_points", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class mem_opts(C.Structure):
    _fields_ = [("target_rel_err", C.c_double), ("max_points", C.c_uint64),
                ("min_points", C.c_uint64), ("n_adapt_iters", C.c_int32),
                ("flow_guided", C.c_int32), ("adapt_points", C.c_uint64), ("alpha", C.c_double),
                ("grid_in", C.POINTER(C.c_double)), ("event_id_base", C.c_uint64),
                ("phase_events", C.c_void_p), ("flow_screen", C.c_double),
                ("flow_cost", C.c_double), ("plans", C.POINTER(mem_plan)),
                ("strat_points", C.c_int32), ("reserved1", C.c_int32)]


_lib = None
_vp = C.c_void_p

# (name, restype, argtypes) of every exported symbol declared in include/mem.h
SIGNATURES = [
    ("mem_process_dims", C.c_int32, [C.c_int32]),
    ("mem_process_nperm", C.c_int32, [C.c_int32]),
    ("mem_create_process", C.c_int, [C.POINTER(mem_process_desc), C.POINTER(_vp)]),
    ("mem_upload_events", C.c_int, [_vp, _vp, C.c_int64, C.c_int32, _vp, C.POINTER(_vp)]),
    ("mem_integrate", C.c_int, [_vp, _vp, C.POINTER(mem_tf_desc), C.c_uint64, C.c_uint64,
                                C.POINTER(mem_opts), _vp, _vp, _vp, _vp, _vp]),
    ("mem_integrate_batch", C.c_int, [C.c_int32, _vp, _vp, _vp, C.c_uint64, C.POINTER(mem_opts),
                                      _vp, _vp, _vp, _vp, _vp]),
    ("mem_set_tc_wait_limit", C.c_int, [C.c_uint32]),
    ("mem_dilep_solve", C.c_int, [_vp, C.c_int64, _vp, _vp, _vp]),
    ("mem_integrate_noalloc", C.c_int, [C.POINTER(mem_process_desc), C.POINTER(mem_tf_desc),
                                        _vp, C.c_int64, C.c_uint64, C.c_uint64, C.c_uint64,
                                        _vp, _vp, _vp, _vp]),
    ("mem_flow_param_count", C.c_int64, []),
    ("mem_flow_create", C.c_int, [C.c_uint64, C.POINTER(_vp)]),
    ("mem_flow_set_params", C.c_int, [_vp, _vp, C.c_int64]),
    ("mem_flow_get_params", C.c_int, [_vp, _vp, C.c_int64]),
    ("mem_flow_map", C.c_int, [_vp, _vp, _vp, C.c_int64, _vp, _vp, _vp]),
    ("mem_flow_grad", C.c_int, [_vp, _vp, _vp, _vp, C.c_int64, _vp, C.POINTER(C.c_double),
                                _vp]),
    ("mem_flow_train", C.c_int, [_vp, _vp, _vp, _vp, C.c_int64, C.c_int32, C.c_int32,
                                 C.c_float, C.c_uint64, _vp, _vp]),
    ("mem_flow_samples", C.c_int, [_vp, _vp, C.POINTER(mem_tf_desc), C.c_uint64,
                                   C.POINTER(mem_opts), C.c_int32, _vp, _vp, _vp, _vp, _vp]),
    ("mem_integrate_flow", C.c_int, [_vp, _vp, C.POINTER(mem_tf_desc), _vp, C.c_uint64,
                                     C.POINTER(mem_opts), _vp, _vp, _vp, _vp, _vp, _vp]),
    ("mem_flow_eval_points", C.c_int, [_vp, C.POINTER(mem_tf_desc), _vp, _vp, C.c_int32,
                                       C.c_uint64, C.c_uint32, C.c_uint32, C.c_int64, _vp, _vp,
                                       _vp, _vp]),
    ("mem_autotune", C.c_int, [_vp, _vp, C.POINTER(mem_tf_desc), C.c_uint64, C.POINTER(mem_opts),
                               C.POINTER(mem_plan), C.POINTER(C.c_double), C.POINTER(C.c_int32), _vp]),
    ("mem_parton_weights", C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    ("mem_process_set_pdf_grid", C.c_int, [_vp, _vp, C.c_int32, C.c_int32, C.c_double,
                                           C.c_double, C.c_double, C.c_double]),
    ("mem_discriminant", C.c_int, [C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("mem_ttbb_colour_matrices", C.c_int, [_vp, _vp]),
    ("mem_ttbb_colour_factors", C.c_int, [_vp, _vp, _vp]),
    ("mem_destroy", None, [_vp]),
    ("mem_last_error", C.c_char_p, []),
    ("mem_eval_points", C.c_int, [_vp, _vp, C.POINTER(mem_tf_desc), C.c_int64, C.c_int32,
                                  C.c_uint64, C.c_uint64, C.c_int64, _vp, _vp, _vp]),
    ("mem_philox_uniforms", C.c_int, [C.c_uint64, C.c_uint64, C.c_int32, C.c_uint64, C.c_int64,
                                      C.c_int32, _vp, _vp]),
    ("mem_vegas_refine", C.c_int, [C.c_int32, C.c_int32, _vp, _vp, C.c_double, _vp]),
]


def lib():
    """Load libmem.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != MEM_OK:
        raise MemError(status, lib().mem_last_error().decode())


def _ptr(a):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def process_desc(kind, params):
    d = mem_process_desc()
    d.kind = kind
    d.reserved = 0
    for k in ("sqrt_s", "mz", "wz", "mw", "ww", "mt", "wt", "alpha", "sw2", "alpha_s"):
        setattr(d, k, float(params[k]))
    for k in ("pdf_A", "pdf_a", "pdf_b"):
        getattr(d, k)[:] = [float(v) for v in params[k]]
    for k in ("mh", "wh", "mb"):   # Higgs parameters (ttH only)
        setattr(d, k, float(params.get(k, 0.0)))
    return d


def tf_desc(params):
    t = mem_tf_desc()
    for k, _ in mem_tf_desc._fields_:
        setattr(t, k, float(params[k]))
    return t


def make_opts(n_adapt_iters=5, adapt_points=0, alpha=1.5, grid_in=None, event_id_base=0,
              target_rel_err=0.0, max_points=0, min_points=0, phase_events=None,
              flow_screen=0.0, flow_cost=0.0, flow_guided=0, plans=None, strat_points=0):
    """phase_events: optional list of 4 torch.cuda.Event (created with
    enable_timing=True) recorded at the phase boundaries on the call's stream."""
    o = mem_opts()
    o.target_rel_err = target_rel_err
    o.max_points = max_points
    o.min_points = min_points
    o.n_adapt_iters = n_adapt_iters
    o.flow_guided = flow_guided
    o.adapt_points = adapt_points
    o.alpha = alpha
    keep = None
    if grid_in is not None:
        keep = np.ascontiguousarray(grid_in, dtype=np.float64)
        o.grid_in = keep.ctypes.data_as(C.POINTER(C.c_double))
    o.event_id_base = event_id_base
    o.flow_screen = flow_screen
    o.flow_cost = flow_cost
    o.strat_points = strat_points
    plan_arr = None
    if plans is not None:
        plan_arr = (mem_plan * len(plans))(*plans)
        o.plans = C.cast(plan_arr, C.POINTER(mem_plan))
    ev_arr = None
    if phase_events is not None:
        assert len(phase_events) == 4
        ev_arr = (C.c_void_p * 4)(*[e.cuda_event for e in phase_events])
        o.phase_events = C.cast(ev_arr, C.c_void_p)
    o._keep = (keep, ev_arr, plan_arr)
    return o


def mem_process_dims(kind):
    return lib().mem_process_dims(kind)


def mem_process_nperm(kind):
    return lib().mem_process_nperm(kind)


def mem_create_process(desc):
    h = _vp()
    _check(lib().mem_create_process(C.byref(desc), C.byref(h)))
    return h


def mem_upload_events(proc, records, stream=None):
    """records: host numpy (n, 32) float32 or device torch tensor."""
    on_dev = int(hasattr(records, "is_cuda") and records.is_cuda)
    n = records.shape[0]
    h = _vp()
    _check(lib().mem_upload_events(proc, _ptr(records), n, on_dev, stream, C.byref(h)))
    return h


def mem_integrate(events, proc, tf, n_points, seed, opts, prob, err, n_used=None,
                  ev_status=None, stream=None):
    _check(lib().mem_integrate(events, proc, C.byref(tf), n_points, seed,
                               C.byref(opts) if opts is not None else None, _ptr(prob),
                               _ptr(err), _ptr(n_used), _ptr(ev_status), stream))


def mem_integrate_batch(groups, seed, opts, prob, err, n_used=None, ev_status=None,
                        stream=None):
    """groups: list of (events handle, process handle, mem_tf_desc); outputs concatenated."""
    n = len(groups)
    evs = (C.c_void_p * n)(*[g[0] for g in groups])
    prs = (C.c_void_p * n)(*[g[1] for g in groups])
    tfs = (C.c_void_p * n)(*[C.addressof(g[2]) for g in groups])
    _check(lib().mem_integrate_batch(n, C.cast(evs, C.c_void_p), C.cast(prs, C.c_void_p),
                                     C.cast(tfs, C.c_void_p), seed, C.byref(opts), _ptr(prob),
                                     _ptr(err), _ptr(n_used), _ptr(ev_status), stream))


def mem_autotune(events, proc, tf, seed, opts, stream=None):
    """Best batched schedule for one process on calibration events:
    (mem_plan, converged events/s, plans timed)."""
    best = mem_plan()
    rate = C.c_double()
    tried = C.c_int32()
    _check(lib().mem_autotune(events, proc, C.byref(tf), seed, C.byref(opts), C.byref(best),
                              C.byref(rate), C.byref(tried), stream))
    return best, rate.value, tried.value


def mem_ttbb_colour_matrices():
    """The dilepton ttbb kernels' colour matrices: (38, 38) and (7, 7) complex64."""
    kgg = np.zeros(38 * 38 * 2, dtype=np.float32)
    kqq = np.zeros(7 * 7 * 2, dtype=np.float32)
    _check(lib().mem_ttbb_colour_matrices(kgg.ctypes.data, kqq.ctypes.data))
    return (kgg.view(np.complex64).reshape(38, 38), kqq.view(np.complex64).reshape(7, 7))


def mem_ttbb_colour_factors():
    """The factor rows conj(u_k) of the ttbb colour matrices, K = sum_k u_k u_k^dagger:
    ((38, 38) complex64, (7, 7) complex64, (rank_gg, rank_qq)); rows beyond the rank
    are zero."""
    ugg = np.zeros(38 * 38 * 2, dtype=np.float32)
    uqq = np.zeros(7 * 7 * 2, dtype=np.float32)
    ranks = np.zeros(2, dtype=np.int32)
    _check(lib().mem_ttbb_colour_factors(ugg.ctypes.data, uqq.ctypes.data, ranks.ctypes.data))
    return (ugg.view(np.complex64).reshape(38, 38), uqq.view(np.complex64).reshape(7, 7),
            (int(ranks[0]), int(ranks[1])))


def mem_process_set_pdf_grid(proc, grid):
    """Attach tabulated PDFs: grid = dict(table=(3, n_q, n_x) float32,
    lx=(ln x_min, ln x_max), lq=(ln Q_min, ln Q_max)); None restores the
    parametric set."""
    if grid is None:
        _check(lib().mem_process_set_pdf_grid(proc, None, 0, 0, 0.0, 0.0, 0.0, 0.0))
        return
    t = np.ascontiguousarray(grid["table"], dtype=np.float32)
    _check(lib().mem_process_set_pdf_grid(proc, t.ctypes.data, t.shape[2], t.shape[1],
                                          grid["lx"][0], grid["lx"][1], grid["lq"][0],
                                          grid["lq"][1]))


def mem_parton_weights(events, proc, prob, w_assign=None, ev_status=None, stream=None):
    """Parton-level ttbar weights (delta transfer functions): prob (n_events float64)
    and optionally the weight per b-quark assignment (n_events x 2 float64) and the
    per-event status (int32); all host or all device tensors."""
    _check(lib().mem_parton_weights(events, proc, _ptr(prob), _ptr(w_assign), _ptr(ev_status),
                                    stream))


def mem_discriminant(prob_s, err_s, prob_b, err_b, D, err_D=None, status=None, stream=None):
    """D = log10(p_S / p_B) and its error per event; arrays all host or all device."""
    _check(lib().mem_discriminant(len(D), _ptr(prob_s), _ptr(err_s), _ptr(prob_b), _ptr(err_b),
                                  _ptr(D), _ptr(err_D), _ptr(status), stream))


def mem_integrate_noalloc(desc, tf, records, n_points, seed, event_id_base, prob, err,
                          ev_status=None, stream=None):
    """Allocation-free integration: records (n, 32) float32, prob and err (>= n)
    float64, ev_status (>= n, optional) int32, all contiguous CUDA tensors on the
    current device. Anything else raises MemError(MEM_ERR_INVALID_ARG) here,
    before the library is called, so that no kernel reads or writes past a
    buffer."""
    import torch
    dev = torch.cuda.current_device()

    def check(t, name, dtype, n=None, width=None):
        ok = (isinstance(t, torch.Tensor) and t.is_cuda and t.device.index == dev and
              t.dtype == dtype and t.is_contiguous())
        if ok and width is not None:
            ok = t.dim() == 2 and t.shape[1] == width
        if ok and n is not None:
            ok = t.numel() >= n
        if not ok:
            msg = (f"{name} must be a contiguous {dtype} CUDA tensor on device {dev}"
                   + (f" of shape (n, {width})" if width else f" with at least {n} elements"))
            raise MemError(MEM_ERR_INVALID_ARG, msg)
    check(records, "records", torch.float32, width=REC)
    n = records.shape[0]
    check(prob, "prob", torch.float64, n)
    check(err, "err", torch.float64, n)
    if ev_status is not None:
        check(ev_status, "ev_status", torch.int32, n)
    _check(lib().mem_integrate_noalloc(C.byref(desc), C.byref(tf), _ptr(records), n, n_points,
                                       seed, event_id_base, _ptr(prob), _ptr(err),
                                       _ptr(ev_status), stream))


def mem_dilep_solve(systems):
    """The integrand's dilepton neutrino solver on host systems (n, 22) float64:
    (nsol (n,), solutions (n, 4, 2, 4) nu / nubar in GeV, jacobians (n, 4))."""
    a = np.ascontiguousarray(systems, dtype=np.float64).reshape(-1, 22)
    n = a.shape[0]
    ns = np.zeros(n, dtype=np.int32)
    nu = np.zeros((n, 4, 2, 4))
    jac = np.zeros((n, 4))
    _check(lib().mem_dilep_solve(a.ctypes.data, n, ns.ctypes.data, nu.ctypes.data, jac.ctypes.data))
    return ns, nu, jac


MEM_TC_WAIT_DEFAULT = 1 << 20


def mem_set_tc_wait_limit(polls):
    """Poll limit of the flow kernels' tensor-core waits on the current device."""
    _check(lib().mem_set_tc_wait_limit(polls))


def mem_destroy(handle):
    lib().mem_destroy(handle)


def mem_flow_param_count():
    return lib().mem_flow_param_count()


def mem_flow_create(seed=0):
    h = _vp()
    _check(lib().mem_flow_create(seed, C.byref(h)))
    return h


def mem_flow_set_params(flow, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(lib().mem_flow_set_params(flow, _ptr(p), p.size))


def mem_flow_get_params(flow):
    p = np.zeros(mem_flow_param_count(), dtype=np.float32)
    _check(lib().mem_flow_get_params(flow, _ptr(p), p.size))
    return p


def mem_flow_grad(flow, ys, ws, cs, stream=None):
    """ys (n, 128, 7), ws (n, 128), cs (n, 16): device tensors -> (flat grad, loss)."""
    g = np.zeros(mem_flow_param_count(), dtype=np.float32)
    loss = C.c_double(0.0)
    _check(lib().mem_flow_grad(flow, _ptr(ys), _ptr(ws), _ptr(cs), ys.shape[0], _ptr(g),
                               C.byref(loss), stream))
    return g, loss.value


def mem_flow_train(flow, ys, ws, cs, n_steps, batch_items, lr=1e-3, seed=0, stream=None):
    trace = np.zeros(n_steps, dtype=np.float32)
    _check(lib().mem_flow_train(flow, _ptr(ys), _ptr(ws), _ptr(cs), ys.shape[0], n_steps,
                                batch_items, lr, seed, _ptr(trace), stream))
    return trace


FLOW_SAMPLES_PER_ITEM = 128


def mem_flow_samples(events, proc, tf, n_events, seed, opts=None, per_event=False,
                     want_logj=False, stream=None):
    """Training set of the ttbar flow: (ys, ws, cs[, log_jv]) device tensors of
    shapes (n_items, 128, 7), (n_items, 128), (n_items, 16), (n_items, 128),
    n_items = 24 n_events."""
    import torch
    n_items = n_events * 24
    ys = torch.empty(n_items, FLOW_SAMPLES_PER_ITEM, 7, dtype=torch.float32, device="cuda")
    ws = torch.empty(n_items, FLOW_SAMPLES_PER_ITEM, dtype=torch.float32, device="cuda")
    cs = torch.empty(n_items, 16, dtype=torch.float32, device="cuda")
    lj = torch.empty(n_items, FLOW_SAMPLES_PER_ITEM, dtype=torch.float32,
                     device="cuda") if want_logj else None
    _check(lib().mem_flow_samples(events, proc, C.byref(tf), seed,
                                  None if opts is None else C.byref(opts), int(per_event),
                                  _ptr(ys), _ptr(ws), _ptr(cs), _ptr(lj), stream))
    return (ys, ws, cs, lj) if want_logj else (ys, ws, cs)


def mem_integrate_flow(events, proc, tf, flow, seed, opts, prob, err, n_used=None,
                       ev_status=None, item_sampler=None, stream=None):
    _check(lib().mem_integrate_flow(events, proc, C.byref(tf), flow, seed, C.byref(opts),
                                    _ptr(prob), _ptr(err), _ptr(n_used), _ptr(ev_status),
                                    _ptr(item_sampler), stream))


def mem_flow_eval_points(proc, tf, flow, record, perm, seed, event_id, point0, n, z, logj, w,
                         stream=None):
    """record: device tensor of one event record; z (n, 7) final logits, logj (n,),
    w (n,) float64: device tensors."""
    _check(lib().mem_flow_eval_points(proc, C.byref(tf), flow, _ptr(record), perm, seed,
                                      event_id, point0, n, _ptr(z), _ptr(logj), _ptr(w), stream))


def mem_flow_map(flow, cond, u, y, logj, stream=None):
    """cond (16,), u (n, 7), y (n, 7), logj (n,): device tensors."""
    _check(lib().mem_flow_map(flow, _ptr(cond), _ptr(u), u.shape[0], _ptr(y), _ptr(logj), stream))


def mem_eval_points(events, proc, tf, event_index, perm, seed, point0, n, grid, w_out,
                    stream=None):
    g = None if grid is None else np.ascontiguousarray(grid, dtype=np.float64)
    _check(lib().mem_eval_points(events, proc, C.byref(tf), event_index, perm, seed, point0, n,
                                 _ptr(g), _ptr(w_out), stream))


def mem_philox_uniforms(seed, event_id, perm, point0, n, d, out, stream=None):
    _check(lib().mem_philox_uniforms(seed, event_id, perm, point0, n, d, _ptr(out), stream))


def mem_vegas_refine(hist, grid_in, alpha=1.5):
    hist = np.ascontiguousarray(hist, dtype=np.float64)
    grid_in = np.ascontiguousarray(grid_in, dtype=np.float64)
    n, d = grid_in.shape[0], grid_in.shape[1]
    out = np.zeros_like(grid_in)
    _check(lib().mem_vegas_refine(n, d, _ptr(hist), _ptr(grid_in), alpha, _ptr(out)))
    return out


# ------------------------------------------------------------------ helpers
class Integrator:
    """Owns a process handle and uploaded events; integrate() returns numpy results."""

    def __init__(self, kind, records, process_params, tf_params, stream=None, pdf_grid=None):
        self.kind = kind
        self.tf = tf_desc(tf_params)
        self.proc = mem_create_process(process_desc(kind, process_params))
        if pdf_grid is not None:
            mem_process_set_pdf_grid(self.proc, pdf_grid)
        self.events = mem_upload_events(self.proc, records, stream)
        self.n = records.shape[0]

    def integrate(self, n_points, seed, opts=None, stream=None):
        prob = np.zeros(self.n)
        err = np.zeros(self.n)
        used = np.zeros(self.n, dtype=np.uint64)
        st = np.zeros(self.n, dtype=np.int32)
        mem_integrate(self.events, self.proc, self.tf, n_points, seed, opts, prob, err, used, st,
                      stream)
        return {"prob": prob, "err": err, "n_used": used, "status": st}

    def parton_weights(self, stream=None):
        """Parton-level ttbar weights of the uploaded parton-level records:
        (prob (n,), per-assignment weights (n, 2), status (n,))."""
        prob = np.zeros(self.n)
        w = np.zeros((self.n, 2))
        st = np.zeros(self.n, dtype=np.int32)
        mem_parton_weights(self.events, self.proc, prob, w, st, stream)
        return prob, w, st

    def eval_points(self, event_index, perm, seed, point0, n, grid=None):
        w = np.zeros(n)
        mem_eval_points(self.events, self.proc, self.tf, event_index, perm, seed, point0, n, grid,
                        w)
        return w

    def close(self):
        if self.events:
            mem_destroy(self.events)
            self.events = None
        if self.proc:
            mem_destroy(self.proc)
            self.proc = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

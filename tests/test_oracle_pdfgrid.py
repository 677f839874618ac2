"""Pins of the oracle's tabulated parton densities (Sec. 3: per-flavour grids in
(x, Q), evaluated by bilinear interpolation; factorisation scale Q = sqrt(x1 x2 s)).

* At the nodes the interpolation returns the table.
* A table of a function bilinear in (ln x, ln Q) is reproduced everywhere,
  outside the table too (the edge cells continue linearly).
* A table of the parametric set converges to it as O(h^2) and is within 1 % of
  it over the x range the workloads use (the paper's stated interpolation
  precision).
* The integrand takes both beams' densities at Q = sqrt(x1 x2 s): a table
  flat in x and linear in ln Q multiplies a flat-density integrand by
  (c ln sqrt(x1 x2 s))^2 at every point.
"""
import math

import numpy as np
import pytest


def _flat(params):
    return dict(params, pdf_A=(1.0, 1.0, 1.0), pdf_a=(0.0, 0.0, 0.0), pdf_b=(0.0, 0.0, 0.0))


def test_nodes(ora, synth):
    g = synth.pdf_grid_table(n_x=64, n_q=16)
    P = ora.process(1, synth.DEFAULT_PROCESS, pdf_grid=g)
    lx = np.linspace(g["lx"][0], g["lx"][1], 64)
    lq = np.linspace(g["lq"][0], g["lq"][1], 16)
    for t in range(3):
        for i in (0, 5, 40, 62):
            for j in (0, 7, 15):
                want = float(g["table"][t, j, i])
                got = ora.pdf_q(P, t, math.exp(lx[i]), math.exp(lq[j]))
                assert got == pytest.approx(want, rel=1e-12, abs=0)


def test_bilinear_function_reproduced(ora, synth):
    nx, nq = 20, 9
    lx0, lx1, lq0, lq1 = -9.0, 0.0, 2.0, 9.0
    lx = np.linspace(lx0, lx1, nx)[None, :]
    lq = np.linspace(lq0, lq1, nq)[:, None]
    c = [(50.0, 1.5, 2.0, 0.25), (80.0, 2.0, -1.0, 0.1), (30.0, -1.0, 0.5, 0.05)]
    tab = np.stack([c0 + c1 * lx + c2 * lq + c3 * lx * lq for c0, c1, c2, c3 in c])
    P = ora.process(0, synth.DEFAULT_PROCESS,
                    pdf_grid={"table": tab, "lx": (lx0, lx1), "lq": (lq0, lq1)})
    rng = np.random.default_rng(1)
    for _ in range(200):
        x = math.exp(rng.uniform(-10.5, -1e-3))     # below the table too
        q = math.exp(rng.uniform(1.0, 10.0))        # both sides of the Q range
        for t, (c0, c1, c2, c3) in enumerate(c):
            a, b = math.log(x), math.log(q)
            want = max(c0 + c1 * a + c2 * b + c3 * a * b, 0.0)
            assert ora.pdf_q(P, t, x, q) == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_converges_to_parametric(ora, synth):
    p = synth.DEFAULT_PROCESS
    Ppar = ora.process(2, p)
    xs = np.exp(np.linspace(math.log(1e-5), math.log(0.5), 400))
    errs = []
    for nx in (256, 512):
        g = synth.pdf_grid_table(n_x=nx, n_q=8, kappa=(0, 0, 0), lam=(0, 0, 0))
        g["table"] = g["table"].astype(np.float64)
        # float64 table from the same formula for the convergence check
        lx = np.linspace(g["lx"][0], 0.0, nx)
        x = np.exp(lx)
        x[-1] = 1.0
        for t in range(3):
            g["table"][t] = (p["pdf_A"][t] * x ** p["pdf_a"][t] * (1 - x) ** p["pdf_b"][t])[None, :]
        P = ora.process(2, p, pdf_grid=g)
        e = max(abs(ora.pdf_q(P, t, x, 500.0) / ora.pdf(Ppar, t, x) - 1) for t in range(3) for x in xs)
        errs.append(e)
    assert errs[1] < 0.01
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_scale_is_partonic_mass(ora, synth):
    flat = _flat(synth.DEFAULT_PROCESS)
    c = 0.2
    lq0, lq1 = math.log(5.0), math.log(20000.0)
    lq = np.linspace(lq0, lq1, 6)[:, None]
    tab = np.repeat((c * lq * np.ones((1, 4)))[None], 3, axis=0)
    for kind in (0, 1, 2):
        P0 = ora.process(kind, flat)
        Pg = ora.process(kind, flat, pdf_grid={"table": tab, "lx": (-12.0, 0.0), "lq": (lq0, lq1)})
        T = ora.tf(synth.DEFAULT_TF[kind])
        rec = synth.gen_events(kind, 1, 300 + kind)[0]
        perm = int(rec[28]) if kind == 2 else 0
        rng = np.random.default_rng(kind)
        d = ora.dims(kind)
        n_ok = 0
        for _ in range(20):
            x = rng.uniform(0.05, 0.95, d)
            w0 = ora.integrand_roots(P0, T, rec, perm, x)
            wg = ora.integrand_roots(Pg, T, rec, perm, x)
            assert len(w0) == len(wg)
            for r, (a, b) in enumerate(zip(w0, wg)):
                if a == 0:
                    continue
                k = ora.kinematics(P0, T, rec, perm, x, r)
                Q = math.sqrt(k["aux"][4] * k["aux"][5]) * synth.SQRT_S
                assert b == pytest.approx(a * (c * math.log(Q)) ** 2, rel=1e-10, abs=0)
                n_ok += 1
            assert sum(wg) == pytest.approx(ora.integrand(Pg, T, rec, perm, x), rel=1e-14, abs=0)
        assert n_ok >= 5, kind

"""GPU <-> oracle parity of stratified sampling in the frozen-grid phase
(Sec. 4: the VEGAS integrator's stratified sampling; mem_opts.strat_points),
through the C ABI.

At a frozen grid both sides evaluate the integrand at the same Philox points
placed in the same hypercubes. Unlike plain sampling, whose map inputs are the
exact 24-bit Philox fractions on both sides, a stratified input
(cell + u) / n_s is rounded to FP32 on the device (~3e-8), which moves a point
by a few millionths of a VEGAS bin; near Breit-Wigner peaks that changes a
weight by up to ~1e-5. The estimate is a mean of weights, so it inherits the
per-point rule: 1e-5 (measured: 1.6e-6 to 3.5e-6 for W). The variance is
a sum of per-cube sample variances of 2-4 points whose differences are formed
in FP32; cubes where the integrand is nearly flat lose relative accuracy there,
but they contribute little to the sum: the error agrees to 1e-3.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_1407_7595_gb300 import abi, synth
    abi.lib()
    return abi, synth, O


@pytest.mark.parametrize("kind,k,n", [(0, 2, 20000), (1, 2, 3 * 8192 + 777), (1, 4, 50000),
                                      (2, 2, 3000)])
def test_frozen_grid(env, kind, k, n):
    abi, synth, O = env
    recs = synth.gen_events(kind, 2 if kind < 2 else 1, 5100 + kind)
    P = O.process(kind, synth.DEFAULT_PROCESS)
    T = O.tf(synth.DEFAULT_TF[kind])
    na = 4096 if kind < 2 else 512
    r = O.integrate(P, T, recs, seed=8, n_points=3 * na + 2, n_adapt_iters=3, adapt_points=na,
                    want_grids=True)
    d = synth.DIMS[kind]
    for e in range(len(recs)):
        grid = r["grids"][e * synth.NPERM[kind] + (int(recs[e, 28]) if kind == 2 else 0)]
        one = abi.Integrator(kind, recs[e:e + 1], synth.DEFAULT_PROCESS, synth.DEFAULT_TF[kind])
        opts = abi.make_opts(n_adapt_iters=0, grid_in=grid, event_id_base=e, strat_points=k)
        g = one.integrate(n, seed=21, opts=opts)
        o = O.integrate(P, T, recs[e:e + 1], seed=21, n_points=n, n_adapt_iters=0, grid_in=grid,
                        event_id_base=e, strat_points=k)
        one.close()
        s = O.strat_side(n, d, k)
        assert g["n_used"][0] == o["n_used"][0] == k * s ** d * synth.NPERM[kind]
        assert g["status"][0] == 0
        assert g["prob"][0] == pytest.approx(o["prob"][0], rel=1e-5, abs=0)
        assert g["err"][0] == pytest.approx(o["err"][0], rel=1e-3, abs=0)


def test_adaptive_run_agrees(env):
    abi, synth, O = env
    recs = synth.gen_w(3, 5200)
    integ = abi.Integrator(1, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[1])
    g = integ.integrate(1 << 18, seed=3, opts=abi.make_opts(strat_points=2))
    integ.close()
    P = O.process(1, synth.DEFAULT_PROCESS)
    T = O.tf(synth.DEFAULT_TF[1])
    o = O.integrate(P, T, recs, seed=3, n_points=1 << 18, strat_points=2)
    pull = (g["prob"] - o["prob"]) / np.hypot(g["err"], o["err"])
    assert np.all(np.abs(pull) < 3.5), pull
    assert np.all(g["status"] == 0)


def test_invalid_options(env):
    abi, synth, O = env
    recs = synth.gen_w(1, 5300)
    integ = abi.Integrator(1, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[1])
    with pytest.raises(abi.MemError):
        integ.integrate(4096, seed=1, opts=abi.make_opts(strat_points=1))
    with pytest.raises(abi.MemError):
        integ.integrate(4096, seed=1, opts=abi.make_opts(strat_points=2, target_rel_err=0.01))
    with pytest.raises(abi.MemError):   # the phase has fewer points than one hypercube needs
        integ.integrate(50, seed=1, opts=abi.make_opts(n_adapt_iters=0, strat_points=64))
    integ.close()

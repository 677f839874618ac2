"""Fault paths of the C ABI, made on the host or by a deliberately exhausted wait
limit; nothing here faults, traps or hangs the GPU.

* Non-finite integrand: an event whose record passes upload validation but makes
  every integrand value NaN (a NaN pseudorapidity) ends with MEM_ERR_NONFINITE
  in ev_status, and every other event of the same call equals a call without
  it to rounding (events are independent integrals with their own Philox
  streams).
* Exhausted tensor-core wait: with the flow kernels' poll limit at 0 every
  MMA-completion wait gives up at once; each CTA drains its committed products
  (a second bounded wait), releases its tensor memory and stops, and the call
  returns MEM_ERR_TIMEOUT -- for the sampling kernel (mem_flow_eval_points) and
  the training kernel (mem_flow_grad). With the default limit restored the same
  calls give the same results as before: the context stayed usable.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_7595_gb300 import abi, synth
    abi.lib()
    return torch, abi, synth


def test_nonfinite_event_is_flagged_and_isolated(env):
    torch, abi, synth = env
    kind, n_ev, n_pts = synth.PROC_W, 12, 1 << 15
    recs = synth.gen_events(kind, n_ev, 8100)
    ref = abi.Integrator(kind, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[kind])
    want = ref.integrate(n_pts, seed=5)
    ref.close()
    bad = recs.copy()
    bad[4, 1] = math.nan           # pseudorapidity of the electron of event 4
    integ = abi.Integrator(kind, bad, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[kind])
    got = integ.integrate(n_pts, seed=5)
    integ.close()
    assert got["status"][4] == abi.MEM_ERR_NONFINITE
    keep = np.arange(n_ev) != 4
    assert np.all(got["status"][keep] == abi.MEM_OK)
    # the same points; the adaptation histograms use FP32 shared-memory atomics, so
    # two calls agree to rounding, not bit for bit
    np.testing.assert_allclose(got["prob"][keep], want["prob"][keep], rtol=1e-6)
    np.testing.assert_allclose(got["err"][keep], want["err"][keep], rtol=1e-4)
    assert np.array_equal(got["n_used"], want["n_used"])


def test_exhausted_tensor_core_wait_returns_timeout(env):
    torch, abi, synth = env
    kind = synth.PROC_TTBAR
    recs = synth.gen_events(kind, 2, 8200)
    integ = abi.Integrator(kind, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[kind])
    f = abi.mem_flow_create(3)
    rec = torch.tensor(recs[0], device="cuda")
    n = 2048

    def run():
        z = torch.zeros(n, 7, dtype=torch.float32, device="cuda")
        lj = torch.zeros(n, dtype=torch.float32, device="cuda")
        w = torch.zeros(n, dtype=torch.float64, device="cuda")
        abi.mem_flow_eval_points(integ.proc, integ.tf, f, rec, int(recs[0, 28]), 9, 0, 0, n, z, lj, w)
        return z.cpu().numpy(), w.cpu().numpy()

    # training data: 4 items of 128 samples (the gradient kernel's tensor-core waits)
    rng = np.random.default_rng(5)
    ys = torch.tensor(rng.uniform(0.05, 0.95, (4, 128, 7)), dtype=torch.float32, device="cuda")
    ws = torch.full((4, 128), 1.0 / 128, dtype=torch.float32, device="cuda")
    cs = torch.tensor(rng.normal(size=(4, 16)), dtype=torch.float32, device="cuda")
    try:
        z0, w0 = run()
        g0, l0 = abi.mem_flow_grad(f, ys, ws, cs)
        abi.mem_set_tc_wait_limit(0)
        with pytest.raises(abi.MemError) as e:
            run()
        assert e.value.status == abi.MEM_ERR_TIMEOUT
        with pytest.raises(abi.MemError) as e:
            abi.mem_flow_grad(f, ys, ws, cs)
        assert e.value.status == abi.MEM_ERR_TIMEOUT
    finally:
        abi.mem_set_tc_wait_limit(abi.MEM_TC_WAIT_DEFAULT)
    z1, w1 = run()
    assert np.array_equal(z0, z1) and np.array_equal(w0, w1)
    g1, l1 = abi.mem_flow_grad(f, ys, ws, cs)
    # the gradient sums FP32 atomics across CTAs: equal to rounding
    np.testing.assert_allclose(g1, g0, rtol=1e-4, atol=1e-6 * np.abs(g0).max())
    assert l1 == pytest.approx(l0, rel=1e-5)
    # the fixed-budget path still works in the same context
    res = integ.integrate(1 << 12, seed=3, opts=abi.make_opts(n_adapt_iters=1, adapt_points=512))
    assert np.all(res["status"] == abi.MEM_OK)
    abi.mem_destroy(f)
    integ.close()

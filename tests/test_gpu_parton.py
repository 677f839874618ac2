"""GPU <-> oracle parity of the parton-level ttbar weights (Sec. 4, parton level:
delta transfer functions, average over the two b-quark assignments), through
the C ABI.

Tolerance: the kernel evaluates the FP32 record in FP32. The resonance
virtualities come from sums of positive pairwise terms, so they carry a few
ulp (~3e-7 relative, ~1e-2 GeV^2 on the top's 3e4 GeV^2); a normalised
propagator (m G)^2 / |D|^2 then changes by at most dq^2 / (m G), ~4e-5 for each
top (m G = 242 GeV^2), and the two tops' errors add. The helicity amplitudes add
~1e-6. Hence: every weight of the generator-truth assignment within 1e-4 and
99 % of them within 5e-5;
the wrong assignment (both tops far off-shell, weights 1e-6 to 1e-10 of the
right one) within 1e-3; the per-event mean within 1e-4.
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
    P = O.process(2, synth.DEFAULT_PROCESS)
    return abi, synth, O, P, torch


def _check(recs, prob, w, st, prob_o, w_o):
    assert np.all(st == 0)
    truth = recs[:, 28].astype(int)
    idx = np.arange(len(recs))
    rel_t = np.abs(w[idx, truth] / w_o[idx, truth] - 1)
    rel_f = np.abs(w[idx, 1 - truth] / w_o[idx, 1 - truth] - 1)
    assert rel_t.max() < 1e-4, rel_t.max()
    assert np.quantile(rel_t, 0.99) < 5e-5
    assert rel_f.max() < 1e-3, rel_f.max()
    assert np.max(np.abs(prob / prob_o - 1)) < 1e-4
    np.testing.assert_allclose(prob, 0.5 * (w[:, 0] + w[:, 1]), rtol=1e-15, atol=0)


@pytest.mark.parametrize("n", [1, 255, 4097])
def test_parity_small_and_ragged(env, n):
    abi, synth, O, P, torch = env
    recs = synth.gen_ttbar_parton(n, 1000 + n)
    integ = abi.Integrator(2, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[2])
    prob, w, st = integ.parton_weights()
    integ.close()
    prob_o, w_o = O.parton_batch(P, recs)
    _check(recs, prob, w, st, prob_o, w_o)


def test_full_size_sampled(env):
    """2^20 events (the throughput batch of the benchmark), device outputs, the
    oracle on a seeded sample of 2048 of them."""
    abi, synth, O, P, torch = env
    n = 1 << 20
    recs = synth.gen_ttbar_parton(n, 5150)
    integ = abi.Integrator(2, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[2])
    prob = torch.zeros(n, dtype=torch.float64, device="cuda")
    w = torch.zeros(n, 2, dtype=torch.float64, device="cuda")
    st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    abi.mem_parton_weights(integ.events, integ.proc, prob, w, st)
    torch.cuda.synchronize()
    integ.close()
    prob, w, st = prob.cpu().numpy(), w.cpu().numpy(), st.cpu().numpy()
    assert np.all(st == 0) and np.all(prob > 0)
    sample = np.random.default_rng(3).choice(n, 2048, replace=False)
    prob_o, w_o = O.parton_batch(P, recs[sample])
    _check(recs[sample], prob[sample], w[sample], st[sample], prob_o, w_o)


def test_host_and_device_outputs_agree(env):
    abi, synth, O, P, torch = env
    recs = synth.gen_ttbar_parton(300, 17)
    integ = abi.Integrator(2, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[2])
    prob_h, w_h, st_h = integ.parton_weights()
    prob = torch.zeros(300, dtype=torch.float64, device="cuda")
    abi.mem_parton_weights(integ.events, integ.proc, prob)
    torch.cuda.synchronize()
    integ.close()
    assert np.array_equal(prob.cpu().numpy(), prob_h)


def test_invalid_records_and_kinematic_edge(env):
    """A record with a wrong object kind gets status MEM_ERR_INVALID_ARG and zero
    weights without disturbing its neighbours; an event whose momentum fraction
    reaches 1 has weight 0 on both sides."""
    abi, synth, O, P, torch = env
    recs = synth.gen_ttbar_parton(6, 23)
    recs[2, 4 * 5 + 3] = 5.0         # neutrino marked as a jet
    recs[4, 0:24:4] *= 40.0          # x1 or x2 beyond 1 after the 40x energy scale
    integ = abi.Integrator(2, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[2])
    prob, w, st = integ.parton_weights()
    integ.close()
    assert st[2] == abi.MEM_ERR_INVALID_ARG and prob[2] == 0 and np.all(w[2] == 0)
    assert O.parton_ttbar(P, recs[4], 0)[0] == 0.0 and O.parton_ttbar(P, recs[4], 1)[0] == 0.0
    assert prob[4] == 0 and np.all(w[4] == 0)
    keep = [0, 1, 3, 5]
    prob_o, w_o = O.parton_batch(P, recs[keep])
    _check(recs[keep], prob[keep], w[keep], st[keep], prob_o, w_o)


def test_wrong_process_rejected(env):
    abi, synth, O, P, torch = env
    recs = synth.gen_w(4, 3)
    integ = abi.Integrator(1, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[1])
    with pytest.raises(abi.MemError):
        integ.parton_weights()
    integ.close()

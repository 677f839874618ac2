"""mem_integrate_noalloc, the entry point for callers that may not allocate
device memory while running (e.g. an online event selection that reserves all
GPU memory at start-up): its results must match mem_integrate's, call after
call, while its working memory comes from the library's fixed device array.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_7595_gb300 import abi, synth
    abi.lib()
    return torch, abi, synth


@pytest.mark.parametrize("kind", [0, 1])
def test_noalloc_matches_mem_integrate_on_two_calls(setup, kind):
    torch, abi, synth = setup
    n_ev, n_pts = 40, 50000
    recs = synth.gen_events(kind, n_ev, 6100 + kind)
    ref = abi.Integrator(kind, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[kind])
    want = ref.integrate(n_pts, seed=77, opts=abi.make_opts(event_id_base=5))
    ref.close()
    desc = abi.process_desc(kind, synth.DEFAULT_PROCESS)
    tf = abi.tf_desc(synth.DEFAULT_TF[kind])
    d_recs = torch.from_numpy(recs).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        prob = torch.full((n_ev,), -1.0, dtype=torch.float64, device="cuda")
        err = torch.full_like(prob, -1.0)
        st = torch.full((n_ev,), 99, dtype=torch.int32, device="cuda")
        abi.mem_integrate_noalloc(desc, tf, d_recs, n_pts, 77, 5, prob, err, st, stream)
        torch.cuda.synchronize()
        # same kernels and points; the adaptation histograms use FP32 shared-memory
        # atomics, so the two paths agree to rounding, not bit for bit
        np.testing.assert_allclose(prob.cpu().numpy(), want["prob"], rtol=1e-6)
        np.testing.assert_allclose(err.cpu().numpy(), want["err"], rtol=1e-4)
        assert np.all(st.cpu().numpy() == want["status"])


def test_noalloc_rejects_oversize_and_host_buffers(setup):
    torch, abi, synth = setup
    kind = 1
    desc = abi.process_desc(kind, synth.DEFAULT_PROCESS)
    tf = abi.tf_desc(synth.DEFAULT_TF[kind])
    recs = synth.gen_events(kind, 8, 6200)
    d_recs = torch.from_numpy(recs).cuda()
    prob = torch.zeros(8, dtype=torch.float64, device="cuda")
    err = torch.zeros_like(prob)
    with pytest.raises(abi.MemError) as e:
        abi.mem_integrate_noalloc(desc, tf, d_recs, 1 << 32, 1, 0, prob, err)
    assert e.value.status == abi.MEM_ERR_INVALID_ARG
    big = torch.from_numpy(synth.gen_events(kind, 1, 6201)).cuda().repeat(20000, 1)
    pb = torch.zeros(20000, dtype=torch.float64, device="cuda")
    with pytest.raises(abi.MemError) as e:
        abi.mem_integrate_noalloc(desc, tf, big, 1 << 20, 1, 0, pb, torch.zeros_like(pb))
    assert "working memory" in str(e.value)
    with pytest.raises(abi.MemError):
        abi.mem_integrate_noalloc(desc, tf, d_recs, 50000, 1, 0, np.zeros(8), np.zeros(8))

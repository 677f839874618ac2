"""GPU event discriminant (Sec. 3: D = log10(p_S / p_B)) through the C ABI,
against the oracle's definition: FP64 on both sides, so D agrees to a few ulp
(1e-14 absolute + relative); non-positive densities give NaN and
MEM_ERR_INVALID_ARG; host and device arrays give the same numbers; and D from
two GPU integrals (Drell-Yan under the generating Z mass and one 10 GeV
heavier) agrees with D from the oracle's integrals within their errors.
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
    from oracle import oracle as O
    from paper_1407_7595_gb300 import abi, synth
    abi.lib()
    return abi, synth, O, torch


def test_elementwise(env):
    abi, synth, O, torch = env
    rng = np.random.default_rng(9)
    n = 1001
    ps = 10.0 ** rng.uniform(-40, -10, n)
    pb = 10.0 ** rng.uniform(-40, -10, n)
    es, eb = ps * rng.uniform(0, 0.1, n), pb * rng.uniform(0, 0.1, n)
    ps[5], pb[7], ps[9] = 0.0, -1e-30, -2.0
    D, eD, st = np.zeros(n), np.zeros(n), np.zeros(n, dtype=np.int32)
    abi.mem_discriminant(ps, es, pb, eb, D, eD, st)
    for i in range(n):
        d, e, rc = O.discriminant(ps[i], es[i], pb[i], eb[i])
        if rc:
            assert st[i] == abi.MEM_ERR_INVALID_ARG and math.isnan(D[i]) and math.isnan(eD[i])
        else:
            assert st[i] == 0
            assert abs(D[i] - d) <= 1e-14 * (1 + abs(d))
            assert eD[i] == pytest.approx(e, rel=1e-14, abs=0)
    dev = [torch.tensor(a, device="cuda") for a in (ps, es, pb, eb)]
    Dd = torch.zeros(n, dtype=torch.float64, device="cuda")
    abi.mem_discriminant(*dev, Dd)
    torch.cuda.synchronize()
    Dh = Dd.cpu().numpy()
    ok = st == 0
    assert np.array_equal(Dh[ok], D[ok]) and np.all(np.isnan(Dh[~ok]))


def test_from_integrals(env):
    abi, synth, O, torch = env
    recs = synth.gen_dy(12, 77)
    heavy = dict(synth.DEFAULT_PROCESS, mz=101.19)
    gs = abi.Integrator(0, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[0]).integrate(1 << 15, seed=1)
    gb = abi.Integrator(0, recs, heavy, synth.DEFAULT_TF[0]).integrate(1 << 15, seed=2)
    D, eD = np.zeros(12), np.zeros(12)
    abi.mem_discriminant(gs["prob"], gs["err"], gb["prob"], gb["err"], D, eD)
    T = O.tf(synth.DEFAULT_TF[0])
    os_ = O.integrate(O.process(0, synth.DEFAULT_PROCESS), T, recs, seed=3, n_points=1 << 15)
    ob = O.integrate(O.process(0, heavy), T, recs, seed=4, n_points=1 << 15)
    for i in range(12):
        d, e, rc = O.discriminant(os_["prob"][i], os_["err"][i], ob["prob"][i], ob["err"][i])
        assert rc == 0 and abs(D[i] - d) < 4 * math.hypot(e, eD[i])
    assert np.mean(D > 0) >= 0.75

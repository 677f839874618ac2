"""The learned sampler inside the ttbar integral, through the C ABI.

* Training set (mem_flow_samples): on the uniform grid its points are the
  Philox points of the integration stream, its weights the oracle integrand
  normalised per item, its features the oracle's conditioning features.
* Flow-sampled points (mem_flow_eval_points): the base draws follow the
  oracle's Philox stream 2 through the FP64 reference flow (BF16 weights), the
  weight at the GPU's own point equals the oracle integrand times the GPU's
  |dy/du| (TT_RULE, the ttbar per-point tolerance), and E_u |dy/du| = 1 for the
  fused kernel's Jacobian.
* Integrals (mem_integrate_flow): unbiased against plain VEGAS within the
  combined errors for the identity flow, a random flow and a distorted flow
  with the VEGAS judge; the judge's choices and point accounting are checked.
"""
import numpy as np
import pytest

from test_gpu_parity import check_points
from test_gpu_parity_ttbar import TT_RULE

pytestmark = pytest.mark.gpu
KIND, NEV = 2, 6


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import flow_ref as F
    from oracle import oracle as O
    from paper_1407_7595_gb300 import abi, synth
    abi.lib()
    recs = synth.gen_events(KIND, NEV, 7100)
    integ = abi.Integrator(KIND, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[KIND])
    P = O.process(KIND, synth.DEFAULT_PROCESS)
    T = O.tf(synth.DEFAULT_TF[KIND])
    yield torch, abi, synth, O, F, recs, integ, P, T
    integ.close()


def bf16(torch, a):
    return torch.tensor(a).to(torch.bfloat16).to(torch.float64).numpy()


def random_flow(torch, abi, F, seed, out_scale=1.0):
    layers = F.init_params(7, 6, 128, 16, seed=seed, zero_last=False)
    for L in layers:
        L["W3"] = L["W3"] * out_scale
        L["W2"] = bf16(torch, L["W2"])
        L["W3"] = bf16(torch, L["W3"])
    f = abi.mem_flow_create(0)
    abi.mem_flow_set_params(f, F.to_flat(layers))
    return f, layers


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def test_training_set_uniform_grid(env):
    torch, abi, synth, O, F, recs, integ, P, T = env
    seed = 5
    ys, ws, cs = abi.mem_flow_samples(integ.events, integ.proc, integ.tf, NEV, seed,
                                      abi.make_opts(n_adapt_iters=0))
    ys, ws, cs = ys.cpu().numpy(), ws.cpu().numpy(), cs.cpu().numpy()
    assert np.all((ys > 0) & (ys < 1))
    s = ws.sum(axis=1)
    assert np.all((np.abs(s - 1) < 1e-5) | (s == 0))
    for e in range(NEV):
        for perm in range(24):
            assert np.allclose(cs[e * 24 + perm], F.features(recs[e], perm), rtol=1e-6, atol=1e-6)
    for e, perm in ((0, int(recs[0, 28])), (1, 13), (2, int(recs[2, 28]))):
        item = e * 24 + perm
        u = np.array([O.point_u(seed, e, perm, k, 7) for k in range(128)])
        assert np.array_equal(ys[item], u.astype(np.float32))
        f = np.array([O.integrand(P, T, recs[e], perm, uk) for uk in u])
        assert f.sum() > 0
        check_points(ws[item].astype(np.float64), f / f.sum(), **TT_RULE)


def test_flow_points_vs_reference_and_oracle(env):
    torch, abi, synth, O, F, recs, integ, P, T = env
    f, layers = random_flow(torch, abi, F, seed=31)
    seed, point0 = 77, 1000
    n = 2 * 2048 + 300     # two full passes and a ragged tail
    for e, perm in ((0, int(recs[0, 28])), (3, 7)):
        rec = torch.tensor(recs[e], device="cuda")
        z = torch.zeros(n, 7, dtype=torch.float32, device="cuda")
        lj = torch.zeros(n, dtype=torch.float32, device="cuda")
        w = torch.zeros(n, dtype=torch.float64, device="cuda")
        abi.mem_flow_eval_points(integ.proc, integ.tf, f, rec, perm, seed, e, point0, n, z, lj, w)
        z, lj, w = z.cpu().numpy().astype(np.float64), lj.cpu().numpy(), w.cpu().numpy()
        y = sigmoid(z)
        u = np.array([O.point_u(seed, e, perm, point0 + i, 7, tag=2) for i in range(n)])
        c = np.tile(F.features(recs[e], perm), (n, 1))
        yr, ljr = F.forward(layers, u, c)
        dy, dl = np.abs(y - yr), np.abs(lj - ljr)
        assert np.median(dy) < 2e-3 and dy.max() < 5e-2, (np.median(dy), dy.max())
        assert np.median(dl) < 2e-2 and dl.max() < 2e-1, (np.median(dl), dl.max())
        idx = np.r_[0:200, 2040:2060, n - 100:n]    # pass boundaries and the tail
        w_ora = np.array([O.integrand(P, T, recs[e], perm, y[i]) for i in idx]) * np.exp(lj[idx])
        assert np.count_nonzero(w_ora) > 20
        check_points(w[idx], w_ora, **TT_RULE)
    abi.mem_destroy(f)


def test_fused_jacobian_normalised(env):
    torch, abi, synth, O, F, recs, integ, P, T = env
    f, _ = random_flow(torch, abi, F, seed=32)
    n = 1 << 20
    rec = torch.tensor(recs[1], device="cuda")
    z = torch.zeros(n, 7, dtype=torch.float32, device="cuda")
    lj = torch.zeros(n, dtype=torch.float32, device="cuda")
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    abi.mem_flow_eval_points(integ.proc, integ.tf, f, rec, 0, 9, 1, 0, n, z, lj, w)
    J = torch.exp(lj.double())
    mean, sd = J.mean().item(), J.std().item()
    assert sd > 0.05
    assert abs(mean - 1.0) < 5 * sd / np.sqrt(n), (mean, sd)
    abi.mem_destroy(f)


def _flow_run(abi, integ, f, seed, **kw):
    n = integ.n
    prob, err = np.zeros(n), np.zeros(n)
    used, st = np.zeros(n, dtype=np.uint64), np.zeros(n, dtype=np.int32)
    samp = np.zeros(n * 24, dtype=np.uint8)
    abi.mem_integrate_flow(integ.events, integ.proc, integ.tf, f, seed, abi.make_opts(**kw), prob,
                           err, used, st, samp)
    return prob, err, used, st, samp


def _vegas_run(abi, integ, seed, **kw):
    n = integ.n
    prob, err = np.zeros(n), np.zeros(n)
    used, st = np.zeros(n, dtype=np.uint64), np.zeros(n, dtype=np.int32)
    abi.mem_integrate_batch([(integ.events, integ.proc, integ.tf)], seed, abi.make_opts(**kw),
                            prob, err, used, st)
    return prob, err, used, st


def _pulls(a, b):
    return (a[0] - b[0]) / np.sqrt(a[1] ** 2 + b[1] ** 2)


def test_integral_unbiased_against_vegas(env):
    torch, abi, synth, O, F, recs, integ, P, T = env
    ref = _vegas_run(abi, integ, 11, target_rel_err=0.01, n_adapt_iters=5, adapt_points=4096,
                     max_points=1 << 24)
    assert np.all(ref[3] == 0)
    ident = abi.mem_flow_create(0)
    rnd, _ = random_flow(torch, abi, F, seed=33, out_scale=0.3)
    for f in (ident, rnd):
        r = _flow_run(abi, integ, f, 12, target_rel_err=0.02, max_points=1 << 24,
                      min_points=1 << 15, flow_screen=1e30)
        assert np.all(r[4] == 0)                 # nothing judged
        assert np.all(r[0] > 0)
        assert np.all(np.abs(_pulls(r, ref)) < 4.0), _pulls(r, ref)
        assert np.all(r[2] % 128 == 0)           # whole flow passes, no adaptation counted
    abi.mem_destroy(ident)
    abi.mem_destroy(rnd)


def test_vegas_judge_and_fallback(env):
    torch, abi, synth, O, F, recs, integ, P, T = env
    ref = _vegas_run(abi, integ, 21, target_rel_err=0.01, n_adapt_iters=5, adapt_points=4096,
                     max_points=1 << 24)
    bad, _ = random_flow(torch, abi, F, seed=34, out_scale=3.0)
    pilot = ((1 << 15) // 24 + 127) // 128 * 128
    r = _flow_run(abi, integ, bad, 22, target_rel_err=0.02, max_points=1 << 24,
                  min_points=1 << 15, n_adapt_iters=3, adapt_points=2048, flow_screen=-1.0)
    samp = r[4]
    assert np.all((samp == 1) | (samp == 2))     # every item judged
    assert np.count_nonzero(samp == 2) > 0        # VEGAS wins somewhere against a distorted flow
    assert np.all(np.abs(_pulls(r, ref)) < 4.0), _pulls(r, ref)
    assert np.all(r[2] >= 24 * (pilot + 3 * 2048))
    # a screen that flags nothing keeps the flow everywhere
    r2 = _flow_run(abi, integ, bad, 23, target_rel_err=0.05, max_points=1 << 22,
                   min_points=1 << 15, flow_screen=1e30)
    assert np.all(r2[4] == 0)
    abi.mem_destroy(bad)


def test_guided_grid_unbiased(env):
    """Judge grids seeded by the pilot's per-bin w^2: estimates stay unbiased and
    every judged item's adaptation is counted."""
    torch, abi, synth, O, F, recs, integ, P, T = env
    ref = _vegas_run(abi, integ, 31, target_rel_err=0.01, n_adapt_iters=5, adapt_points=4096,
                     max_points=1 << 24)
    rnd, _ = random_flow(torch, abi, F, seed=35, out_scale=0.3)
    pilot = ((1 << 14) // 24 + 127) // 128 * 128
    r = _flow_run(abi, integ, rnd, 32, target_rel_err=0.02, max_points=1 << 24,
                  min_points=1 << 14, n_adapt_iters=1, adapt_points=2048, flow_screen=-1.0,
                  flow_guided=1, flow_cost=6.0)
    assert np.all((r[4] == 1) | (r[4] == 2))
    assert np.all(np.abs(_pulls(r, ref)) < 4.0), _pulls(r, ref)
    assert np.all(r[2] >= 24 * (pilot + 2048))
    abi.mem_destroy(rnd)


def test_trained_flow_gains(env):
    """What the trained network adds: trained on VEGAS samples of 1024 training
    events, then on 128 fresh events the flow-guided path (pilot -> seeded VEGAS
    grid -> judge) reaches 1 % in fewer points than the same schedule with an
    untrained (identity) flow and than plain VEGAS with the same adaptation
    (median and total over events, cap 2^22 points per event)."""
    torch, abi, synth, O, F, recs, integ, P, T = env
    train = synth.gen_events(KIND, 1024, 7200)
    It = abi.Integrator(KIND, train, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[KIND])
    ys, ws, cs = abi.mem_flow_samples(It.events, It.proc, It.tf, 1024, 1,
                                      abi.make_opts(n_adapt_iters=5, adapt_points=8192))
    f = abi.mem_flow_create(1)
    tr = abi.mem_flow_train(f, ys, ws, cs, n_steps=6000, batch_items=304, lr=1e-3)
    tr2 = abi.mem_flow_train(f, ys, ws, cs, n_steps=2000, batch_items=304, lr=3e-4, seed=1)
    assert tr2[-100:].mean() < tr[:100].mean()
    fresh = synth.gen_events(KIND, 128, 7300)
    Ie = abi.Integrator(KIND, fresh, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[KIND])
    opts = dict(target_rel_err=0.01, max_points=1 << 22, n_adapt_iters=2, adapt_points=4096,
                flow_screen=-1.0, flow_guided=1, flow_cost=6.0)
    trained = _flow_run(abi, Ie, f, 41, **opts)
    ident = abi.mem_flow_create(1)
    untrained = _flow_run(abi, Ie, ident, 41, **opts)
    plain = _vegas_run(abi, Ie, 42, target_rel_err=0.01, max_points=1 << 22, n_adapt_iters=2,
                       adapt_points=4096)
    med = [float(np.median(r[2])) for r in (trained, untrained, plain)]
    tot = [int(r[2].sum()) for r in (trained, untrained, plain)]
    assert med[0] < 0.9 * med[1] and tot[0] < tot[1], (med, tot)
    assert med[0] < 0.9 * med[2] and tot[0] < tot[2], (med, tot)
    ok = (trained[3] == 0) & (plain[3] == 0)
    assert np.all(np.abs(_pulls(trained, plain)[ok]) < 4.5)
    for h in (f, ident):
        abi.mem_destroy(h)
    It.close()
    Ie.close()

"""Batched adaptive-budget integration (uneven mix of processes, per-event stop
rule at a target relative error, one CUDA graph) through the C ABI.

* Every event either reaches err/prob <= target (MEM_OK) or hits the cap
  (MEM_NOT_CONVERGED), and the reported points respect the schedule.
* Converged estimates agree with the FP64 oracle (Drell-Yan, W) and with a
  large fixed-budget GPU run (ttbar) within 3.5 sigma of the combined error.
* mem_integrate with target_rel_err gives the same schedule for one group.
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


def make_group(abi, synth, kind, n, seed):
    recs = synth.gen_events(kind, n, seed)
    integ = abi.Integrator(kind, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[kind])
    return recs, integ


def test_mixed_batch_to_one_percent(env):
    abi, synth, O = env
    groups = [make_group(abi, synth, k, n, 8100 + k) for k, n in ((0, 24), (1, 16), (2, 3))]
    n_tot = sum(len(r) for r, _ in groups)
    prob, err = np.zeros(n_tot), np.zeros(n_tot)
    used, st = np.zeros(n_tot, dtype=np.uint64), np.zeros(n_tot, dtype=np.int32)
    target, cap = 0.01, 1 << 22
    opts = abi.make_opts(target_rel_err=target, max_points=cap, adapt_points=4096)
    abi.mem_integrate_batch([(g.events, g.proc, g.tf) for _, g in groups], 77, opts, prob, err,
                            used, st)
    assert np.all((st == abi.MEM_OK) | (st == abi.MEM_NOT_CONVERGED)), st
    ok = st == abi.MEM_OK
    assert ok.mean() > 0.8
    assert np.all(err[ok] <= target * prob[ok] * (1 + 1e-12))
    assert np.all(used <= cap)
    # Drell-Yan and W against the oracle (fixed budget, independent seed)
    off = 0
    for (recs, g), kind in zip(groups, (0, 1, 2)):
        n = len(recs)
        sl = slice(off, off + n)
        if kind < 2:
            P = O.process(kind, synth.DEFAULT_PROCESS)
            T = O.tf(synth.DEFAULT_TF[kind])
            o = O.integrate(P, T, recs[:6], seed=5, n_points=1 << 16)
            pull = (prob[sl][:6] - o["prob"]) / np.sqrt(err[sl][:6] ** 2 + o["err"] ** 2)
            assert np.all(np.abs(pull) < 3.5), (kind, pull)
        else:
            ref = g.integrate((1 << 22) // 24, seed=9)
            pull = (prob[sl] - ref["prob"]) / np.sqrt(err[sl] ** 2 + ref["err"] ** 2)
            assert np.all(np.abs(pull) < 3.5), pull
        off += n
    for _, g in groups:
        g.close()


def test_single_group_through_mem_integrate(env):
    abi, synth, O = env
    recs, g = make_group(abi, synth, 1, 10, 8200)
    opts = abi.make_opts(target_rel_err=0.005, max_points=1 << 22, adapt_points=4096)
    r = g.integrate(0, seed=3, opts=opts)
    prob, err = np.zeros(10), np.zeros(10)
    used, st = np.zeros(10, dtype=np.uint64), np.zeros(10, dtype=np.int32)
    abi.mem_integrate_batch([(g.events, g.proc, g.tf)], 3, opts, prob, err, used, st)
    # same schedule and points; adaptation histograms use FP32 atomics (rounding-level)
    np.testing.assert_allclose(prob, r["prob"], rtol=1e-5)
    assert np.array_equal(st, r["status"])
    assert np.all(r["status"] == 0) and np.all(r["err"] <= 0.005 * r["prob"] * (1 + 1e-12))
    # tighter targets take more points
    opts2 = abi.make_opts(target_rel_err=0.002, max_points=1 << 22, adapt_points=4096)
    r2 = g.integrate(0, seed=3, opts=opts2)
    assert np.all(r2["n_used"] >= r["n_used"])
    with pytest.raises(abi.MemError):
        abi.mem_integrate_batch([(g.events, g.proc, g.tf)], 3,
                                abi.make_opts(target_rel_err=0.0), prob, err)
    g.close()


def test_per_group_plans_and_autotune(env):
    """Each group follows its own schedule (mem_plan), and the autotuner returns
    a plan from its candidate list that integrates its calibration events."""
    abi, synth, O = env
    groups = [make_group(abi, synth, k, n, 8300 + k) for k, n in ((0, 16), (2, 2))]
    n_tot = sum(len(r) for r, _ in groups)
    prob, err = np.zeros(n_tot), np.zeros(n_tot)
    used, st = np.zeros(n_tot, dtype=np.uint64), np.zeros(n_tot, dtype=np.int32)
    plans = [abi.mem_plan(n_adapt_iters=2, tiles_per_cta=2, adapt_points=1024, min_points=1 << 13),
             abi.mem_plan(n_adapt_iters=3, tiles_per_cta=8, adapt_points=2048, min_points=1 << 14)]
    opts = abi.make_opts(target_rel_err=0.02, max_points=1 << 22, plans=plans)
    abi.mem_integrate_batch([(g.events, g.proc, g.tf) for _, g in groups], 5, opts, prob, err, used, st)
    assert np.all((st == 0) | (st == 3))
    # adaptation points are part of n_used: 2 x 1024 per DY event, >= one ttbar item's 3 x 2048
    assert np.all(used[:16] >= 2 * 1024 + ((1 << 13) // 256) * 256)
    assert np.all(used[16:] >= 3 * 2048)
    ok = st == 0
    assert np.all(err[ok] <= 0.02 * prob[ok] * (1 + 1e-12))
    recs, integ = groups[0]
    plan, rate, tried = abi.mem_autotune(integ.events, integ.proc, integ.tf, 9,
                                         abi.make_opts(target_rel_err=0.02, max_points=1 << 22))
    assert tried >= 9 and rate > 0
    assert plan.n_adapt_iters in (2, 3, 4, 5) and plan.adapt_points in (2048, 4096, 8192)
    assert plan.tiles_per_cta in (2, 4, 8) and plan.min_points in (1 << 13, 1 << 14, 1 << 15)
    p2, e2 = np.zeros(16), np.zeros(16)
    u2, s2 = np.zeros(16, dtype=np.uint64), np.zeros(16, dtype=np.int32)
    abi.mem_integrate_batch([(integ.events, integ.proc, integ.tf)], 11,
                            abi.make_opts(target_rel_err=0.02, max_points=1 << 22, plans=[plan]),
                            p2, e2, u2, s2)
    assert np.mean(s2 == 0) >= 0.9
    for _, g in groups:
        g.close()

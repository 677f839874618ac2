"""GPU <-> oracle parity for the dilepton ttbb integrand (the background of Sec. 3-4:
the variables and 12 jet assignments of dilepton ttH, the extra b bbar pair's mass
mapped log-uniformly over its jet window, its jets as (b, bbar) and (bbar, b)),
through the C ABI.

The kernel writes the 36 g g and 7 q qbar production diagrams in light-cone Weyl form
(FP32) around the Fierz-collapsed top decays, with colour matrices computed on the
host from its own SU(3) sums; the oracle uses explicit Dirac matrices and colour
sums in FP64 (about 0.7 s per point in the region, so batches are short). The
records are dilepton ttH events (the same layout: two leptons, four b jets)
relabelled as ttbb, and events of the ttbb generator itself (continuum pair
masses). Rule as for dilepton ttH (the same FP32 inputs to the FP64 neutrino
solution): over the points where either side is nonzero, the zero pattern
identical (one edge point allowed), >= 95 % within 1e-4, every point within
max(1e-4, 100 s_i) (s_i the oracle's own sensitivity to 2^-24 moves of the
point's coordinates), capped at 5e-2, or 1e-6 of the mean weight, the sum over the
well-conditioned points within 1e-4; the frozen-grid integral equals the ratio of
its point sums to 1e-7 and agrees within 1e-4 plus its ill-conditioned points'
bounds.
"""
import numpy as np
import pytest

from parity_rules import check_conditioned, check_frozen_integral
from test_gpu_parity_tth import TH_RULE, check_nonzero_points

pytestmark = pytest.mark.gpu
KIND = 5


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_1407_7595_gb300 import abi, synth
    abi.lib()
    recs = synth.gen_events(4, 4, 7300).copy()
    recs[:, 27] = KIND
    integ = abi.Integrator(KIND, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[KIND])
    P = O.process(KIND, synth.DEFAULT_PROCESS)
    T = O.tf(synth.DEFAULT_TF[KIND])
    yield abi, synth, O, recs, integ, P, T
    integ.close()


def test_dims_and_perms(env):
    abi = env[0]
    assert abi.mem_process_dims(KIND) == 8 and abi.mem_process_nperm(KIND) == 12


# (event, assignment) pairs and batch lengths: 20-30 points of each reach the region
CASES = [(2, 2, 256), (1, 4, 192)]


def test_points_uniform_grid(env):
    abi, synth, O, recs, integ, P, T = env
    for e, perm, n in CASES:
        w_gpu = integ.eval_points(e, perm, 42, 0, n)
        w_ora = O.eval_points(P, T, recs[e], e, perm, 42, 0, n)
        check_nonzero_points(w_gpu, w_ora, (O, P, T, recs[e], e, perm, 42, 0, 8, None))


# events of the ttbb generator itself (continuum pair masses, not relabelled ttH)
GEN_CASES = [(0, 0, 256), (2, 10, 192)]


def test_points_uniform_grid_generator_events(env):
    abi, synth, O, recs, integ, P, T = env
    gen = synth.gen_events(KIND, 4, 7600)
    it = abi.Integrator(KIND, gen, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[KIND])
    for e, perm, n in GEN_CASES:
        w_gpu = it.eval_points(e, perm, 42, 0, n)
        w_ora = O.eval_points(P, T, gen[e], e, perm, 42, 0, n)
        check_nonzero_points(w_gpu, w_ora, (O, P, T, gen[e], e, perm, 42, 0, 8, None))
    it.close()


def test_integral_frozen_grid(env):
    abi, synth, O, recs, integ, P, T = env
    n = 4096 + 333
    g = integ.integrate(n, seed=21, opts=abi.make_opts(n_adapt_iters=0))
    # event 0: few points of each assignment reach the region, so the oracle run is short
    o = O.integrate(P, T, recs[0:1], seed=21, n_points=n, n_adapt_iters=0, event_id_base=0)
    assert o["prob"][0] > 0
    parts = [check_conditioned(integ.eval_points(0, perm, 21, 0, n),
                               O.eval_points(P, T, recs[0], 0, perm, 21, 0, n),
                               (O, P, T, recs[0], 0, perm, 21, 0, 8, None), **TH_RULE)
             for perm in range(12)]
    check_frozen_integral(g["prob"][0], o["prob"][0], parts, 1e-4)
    assert np.all(g["n_used"] == 12 * n) and np.all(g["status"] == 0)


def test_adaptive_budget_agrees_with_fixed_budget(env):
    """Per-event stopping (mem_integrate with target_rel_err, the batched schedule)
    against a fixed-budget run of the same events with independent points: the two
    estimates agree within 4 combined standard errors (the per-event stop rule and
    the optimistic errors near the neutrino branch points, see the dilepton ttbar
    tests, widen the pulls)."""
    abi, synth, O, recs, integ, P, T = env
    ev = synth.gen_events(KIND, 3, 7500)
    it = abi.Integrator(KIND, ev, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[KIND])
    fixed = it.integrate(1 << 16, seed=31)
    ad = it.integrate(0, seed=32, opts=abi.make_opts(target_rel_err=0.05, max_points=12 << 16,
                                                    min_points=12 << 12, n_adapt_iters=3,
                                                    adapt_points=4096))
    it.close()
    assert np.all(fixed["status"] == 0)
    assert np.all((ad["status"] == 0) | (ad["status"] == abi.MEM_NOT_CONVERGED))
    assert np.all(ad["n_used"] <= 12 << 16) and np.all(ad["n_used"] > 0)
    ok = (fixed["prob"] > 0) & (ad["prob"] > 0)
    assert np.count_nonzero(ok) >= 2
    pull = (ad["prob"] - fixed["prob"])[ok] / np.sqrt(ad["err"] ** 2 + fixed["err"] ** 2)[ok]
    assert np.all(np.abs(pull) < 4.0), pull
    conv = ad["status"] == 0
    assert np.all(ad["err"][conv] <= 0.05 * ad["prob"][conv] * (1 + 1e-12))

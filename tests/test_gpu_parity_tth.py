"""GPU <-> oracle parity for the dilepton ttH integrand (Sec. 3-4, Eq. "integrand"
with Eq. "mhsolve": 8 dimensions, 12 jet assignments, up to 2 x 4 kinematic
solutions per point), through the C ABI.

The kernel evaluates the ttH production amplitude with light-cone Weyl spinors
(Fierz-collapsed decays) in FP32 and the neutrinos in FP64 with its own solver;
the oracle uses explicit Dirac matrices and FP64 throughout. Between 4 % and 22 % of
the uniform-grid points of the assignments below reach the kinematic region (both
neutrinos real; the Higgs-pair map lands inside both jet windows by construction).

Tolerance: as for dilepton ttbar (FP32 virtualities and jet energies feeding the
FP64 neutrino solution, double-Gaussian TFs; parity_rules.check_conditioned),
with two more jets and the Higgs pair's energies from (m_H^2, f) in FP32 and the
longer FP32 spinor chains: >= 95 % of the points within 1e-4 (98-99.5 % on the GPU),
every point within max(1e-4, 100 s_i) capped at 5e-2 (s_i the oracle's own
sensitivity to 2^-24 moves of the point's coordinates; on the GPU such points
differ by 0.1-20 s_i, the worst seen, s_i = 4e-4 and 49 % of its batch, by 5e-4),
the zero pattern identical (one edge point allowed), and the sum over the points
within 1e-4 or well conditioned within 1e-4 (on the GPU: <= 1.1e-5). The
frozen-grid integral equals the ratio of its point sums to 1e-7 and agrees within
1e-5 plus its ill-conditioned points' bounds (on the GPU: 2.5e-6).
"""
import numpy as np
import pytest

from parity_rules import check_conditioned, check_frozen_integral

pytestmark = pytest.mark.gpu
KIND = 4


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_1407_7595_gb300 import abi, synth
    abi.lib()
    recs = synth.gen_events(KIND, 4, 7300)
    integ = abi.Integrator(KIND, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[KIND])
    P = O.process(KIND, synth.DEFAULT_PROCESS)
    T = O.tf(synth.DEFAULT_TF[KIND])
    yield abi, synth, O, recs, integ, P, T
    integ.close()


TH_RULE = dict(rel=1e-4, frac=0.95, sum_rel=1e-4)


def check_nonzero_points(w_gpu, w_ora, ctx):
    """The dilepton ttH/ttbb rule on one batch (ctx as for check_conditioned)."""
    assert np.count_nonzero((w_gpu != 0) | (w_ora != 0)) >= 10
    return check_conditioned(w_gpu, w_ora, ctx, **TH_RULE)


def test_dims_and_perms(env):
    abi = env[0]
    assert abi.mem_process_dims(KIND) == 8 and abi.mem_process_nperm(KIND) == 12


# (event, assignment) pairs whose uniform-grid points reach the kinematic region
# often enough to compare (the true assignment and others; some assignments of some
# events have no real neutrino solution anywhere near)
CASES = [(1, 4), (1, 1), (2, 2), (3, 9), (3, 5), (0, 9)]


def test_points_uniform_grid(env):
    abi, synth, O, recs, integ, P, T = env
    assert [int(recs[e, 28]) for e in (1, 2, 3, 0)] == [4, 2, 9, 9]
    for e, perm in CASES:
        w_gpu = integ.eval_points(e, perm, 42, 0, 4096)
        w_ora = O.eval_points(P, T, recs[e], e, perm, 42, 0, 4096)
        check_nonzero_points(w_gpu, w_ora, (O, P, T, recs[e], e, perm, 42, 0, 8, None))


def test_integral_frozen_grid(env):
    abi, synth, O, recs, integ, P, T = env
    n = 4096 + 333   # one full sampling chunk and a ragged tail per item
    g = integ.integrate(n, seed=21, opts=abi.make_opts(n_adapt_iters=0))
    # event 3: every assignment reaches the region; event ids follow the upload order
    o = O.integrate(P, T, recs[3:4], seed=21, n_points=n, n_adapt_iters=0, event_id_base=3)
    parts = [check_conditioned(integ.eval_points(3, perm, 21, 0, n),
                               O.eval_points(P, T, recs[3], 3, perm, 21, 0, n),
                               (O, P, T, recs[3], 3, perm, 21, 0, 8, None), **TH_RULE)
             for perm in range(12)]
    check_frozen_integral(g["prob"][3], o["prob"][0], parts, 1e-5)
    assert np.all(g["n_used"] == 12 * n) and np.all(g["status"] == 0)


def test_adaptive_budget_agrees_with_fixed_budget(env):
    """Per-event stopping (mem_integrate with target_rel_err, the batched schedule)
    against a fixed-budget run of the same events with independent points: the two
    estimates agree within 4 combined standard errors (the per-event stop rule and
    the optimistic errors near the neutrino branch points, see the dilepton ttbar
    tests, widen the pulls)."""
    abi, synth, O, recs, integ, P, T = env
    ev = synth.gen_events(KIND, 3, 7400)
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

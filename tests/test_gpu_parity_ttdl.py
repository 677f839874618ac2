"""GPU <-> oracle parity for the dilepton ttbar integrand (6 dimensions, 2 b-jet
assignments, up to 4 neutrino solutions per point; Sec. 3-4, Eq. "dilepsolv"),
through the C ABI.

The kernel solves for the neutrinos in FP64 with its own method (real roots of
the resultant quartic through the derivative chain, safeguarded Newton) and does
everything else in FP32; the oracle uses the Durand-Kerner iteration and FP64
throughout. The batched, per-event-stopping entry point is covered too.

Per-point tolerance: the kernel's FP64 solver receives FP32 inputs -- the four
virtualities from the Breit-Wigner maps and the b-jet energies from the log map,
each with a few 1e-7 of relative rounding. The neutrino momenta move by the
inverse of d(q^2)/d(nu) times that rounding, so the Jacobian 1/|det| and the
decay invariants inherit the conditioning of the solution; the double-Gaussian
jet TF amplifies an energy error by z/sigma ~ 10-50 as in semileptonic ttbar.
Most points agree within 1e-5 (92-98 % per batch on the GPU) and 97 % within 3e-5.
Next to a branch point, where two solutions merge and the Jacobian peaks, the
weight is ill-conditioned and one point can carry a fifth of a batch; there the
oracle measures the conditioning itself (s_i, the summed relative change of its
weight under 2^-24 moves of the point's unit-cube coordinates, see
parity_rules.check_conditioned) and a point may differ by up to 100 s_i (the
FP32 rounding of a Breit-Wigner output is worth a move of u up to m / (pi Gamma)
~ 40 times larger), capped at 5e-2 (a missed or spurious solution is an O(1) change); on the GPU
such points differ by 0.1-1.5 s_i.
Rule: >= 97 % of the points within 3e-5, every point within its conditioning
bound, the sum over the points within 3e-5 or well conditioned within 1e-5 (on
the GPU: <= 1.3e-6); the frozen-grid integral equals the ratio of its point sums
to 1e-7 and agrees within 1e-5 plus the bounds of its ill-conditioned points
(on the GPU: 7.5e-7).
"""
import numpy as np
import pytest

from parity_rules import check_conditioned, check_frozen_integral

pytestmark = pytest.mark.gpu
KIND = 3
DL_RULE = dict(rel=3e-5, frac=0.97, sum_rel=1e-5)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_1407_7595_gb300 import abi, synth
    abi.lib()
    recs = synth.gen_events(KIND, 3, 7100)
    integ = abi.Integrator(KIND, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[KIND])
    P = O.process(KIND, synth.DEFAULT_PROCESS)
    T = O.tf(synth.DEFAULT_TF[KIND])
    yield abi, synth, O, recs, integ, P, T
    integ.close()


def test_dims_and_perms(env):
    abi = env[0]
    assert abi.mem_process_dims(KIND) == 6 and abi.mem_process_nperm(KIND) == 2


def test_points_uniform_grid(env):
    abi, synth, O, recs, integ, P, T = env
    for e in range(len(recs)):
        for perm in (0, 1):
            w_gpu = integ.eval_points(e, perm, 42, 0, 512)
            w_ora = O.eval_points(P, T, recs[e], e, perm, 42, 0, 512)
            assert np.count_nonzero(w_ora) > 20     # the kinematic region is reached
            check_conditioned(w_gpu, w_ora, (O, P, T, recs[e], e, perm, 42, 0, 6, None), **DL_RULE)


def test_points_adapted_grid(env):
    abi, synth, O, recs, integ, P, T = env
    e = 0
    perm = int(recs[e, 28])
    r = O.integrate(P, T, recs[e:e + 1], seed=7, n_points=6000, n_adapt_iters=3,
                    adapt_points=1500, want_grids=True)
    grid = r["grids"][perm]
    w_gpu = integ.eval_points(e, perm, 43, 10, 768, grid=grid)
    w_ora = O.eval_points(P, T, recs[e], e, perm, 43, 10, 768, grid=grid)
    check_conditioned(w_gpu, w_ora, (O, P, T, recs[e], e, perm, 43, 10, 6, grid), **DL_RULE)


def test_integral_frozen_grid(env):
    abi, synth, O, recs, integ, P, T = env
    n = 2 * 4096 + 333   # two full sampling chunks and a ragged tail per item
    g = integ.integrate(n, seed=21, opts=abi.make_opts(n_adapt_iters=0))
    o = O.integrate(P, T, recs[:1], seed=21, n_points=n, n_adapt_iters=0)
    parts = [check_conditioned(integ.eval_points(0, perm, 21, 0, n),
                               O.eval_points(P, T, recs[0], 0, perm, 21, 0, n),
                               (O, P, T, recs[0], 0, perm, 21, 0, 6, None), **DL_RULE)
             for perm in (0, 1)]
    check_frozen_integral(g["prob"][0], o["prob"][0], parts, DL_RULE["sum_rel"])
    assert g["err"][0] == pytest.approx(o["err"][0], rel=1e-3, abs=0)
    assert g["n_used"][0] == 2 * n and g["status"][0] == 0


def test_adaptive_agrees_within_errors(env):
    abi, synth, O, recs, integ, P, T = env
    n = 4096
    g = integ.integrate(n, seed=3, opts=abi.make_opts(n_adapt_iters=2, adapt_points=1024))
    o = O.integrate(P, T, recs[:2], seed=3, n_points=n, n_adapt_iters=2, adapt_points=1024)
    pull = (g["prob"][:2] - o["prob"]) / np.sqrt(g["err"][:2] ** 2 + o["err"] ** 2)
    assert np.all(np.abs(pull) < 3.5), pull
    assert np.all(g["status"] == 0)


def test_batched_and_adaptive_budget(env):
    """Per-event stopping at a target relative error: the batched entry point and
    mem_integrate's adaptive schedule (the same schedule) agree within their MC
    errors, every event either converges (status 0, error within the target) or
    reaches the point cap (MEM_NOT_CONVERGED: a few dilepton events have heavy
    tails near the solution branch points). GPU-oracle agreement of full runs is
    checked at a fixed budget above; here an independent oracle run is not used as
    a check: where two neutrino solutions merge the Jacobian has an integrable
    1/sqrt singularity whose weight variance diverges logarithmically, so the MC
    error of a few thousand points understates the spread (one 8,192-point oracle
    run sat 4.1 of its nominal sigma from the converged GPU estimate)."""
    abi, synth, O, recs, integ, P, T = env
    recs6 = synth.gen_events(KIND, 6, 7200)
    g = abi.Integrator(KIND, recs6, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[KIND])
    opts = abi.make_opts(target_rel_err=0.02, max_points=1 << 21, adapt_points=4096)
    r = g.integrate(0, seed=5, opts=opts)
    prob, err = np.zeros(6), np.zeros(6)
    used, st = np.zeros(6, dtype=np.uint64), np.zeros(6, dtype=np.int32)
    abi.mem_integrate_batch([(g.events, g.proc, g.tf)], 5, opts, prob, err, used, st)
    g.close()
    for s_, p_, e_ in ((st, prob, err), (r["status"], r["prob"], r["err"])):
        assert np.all((s_ == 0) | (s_ == abi.MEM_NOT_CONVERGED)), s_
        assert np.count_nonzero(s_ == 0) >= 3
        ok = s_ == 0
        assert np.all(e_[ok] <= 0.02 * p_[ok] * (1 + 1e-12))
        assert np.all(p_ > 0)
    assert np.all(np.abs(prob - r["prob"]) <= 3.5 * np.hypot(err, r["err"]))

"""GPU <-> oracle parity with tabulated parton densities (Sec. 3: per-flavour
(x, Q) grids, bilinear interpolation in (ln x, ln Q), factorisation scale
Q = sqrt(x1 x2 s)), through the C ABI (mem_process_set_pdf_grid).

Both sides interpolate the same float32 table (the oracle in FP64). The kernel
forms ln x in FP32 (a few ulp, ~1e-6 absolute) and the node offsets from
float32 bounds; on a 512 x 64 table a cell spans 0.027 in ln x, so the
interpolation weight moves by < 1e-4 and a density by < 1e-5 of a cell's
change (~3 %): ~1e-6 relative. The per-point rules of the parametric tests
therefore stand unchanged (DY, W: 1e-5 on 99.9 %; ttbar: 1e-5 on 97 %, all
within 3e-4), and so does the frozen-grid integral (1e-6).
"""
import numpy as np
import pytest

from test_gpu_parity import check_points

pytestmark = pytest.mark.gpu

TT_RULE = dict(rel=1e-5, frac=0.97, cap=3e-4, sum_rel=1e-5)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_1407_7595_gb300 import abi, synth
    abi.lib()
    grid = synth.pdf_grid_table()
    return abi, synth, O, grid


def _setup(env, kind, n, seed):
    abi, synth, O, grid = env
    recs = synth.gen_events(kind, n, seed)
    integ = abi.Integrator(kind, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[kind],
                           pdf_grid=grid)
    P = O.process(kind, synth.DEFAULT_PROCESS, pdf_grid=grid)
    T = O.tf(synth.DEFAULT_TF[kind])
    return recs, integ, P, T


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_points_with_table(env, kind):
    abi, synth, O, grid = env
    recs, integ, P, T = _setup(env, kind, 2, 4100 + kind)
    n = 2048 if kind < 2 else 384
    for e in range(len(recs)):
        perm = int(recs[e, 28]) if kind == 2 else 0
        w_gpu = integ.eval_points(e, perm, 51, 0, n)
        w_ora = O.eval_points(P, T, recs[e], e, perm, 51, 0, n)
        check_points(w_gpu, w_ora, **(TT_RULE if kind == 2 else {}))
    integ.close()


def test_table_changes_the_result_and_detaches(env):
    """The table is in effect (results differ from the parametric set by the
    Q dependence) and detaching it restores the parametric results bitwise."""
    abi, synth, O, grid = env
    recs, integ, P, T = _setup(env, 1, 1, 4200)
    w_tab = integ.eval_points(0, 0, 5, 0, 1024)
    ref = abi.Integrator(1, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[1])
    w_par = ref.eval_points(0, 0, 5, 0, 1024)
    assert abs(w_tab.sum() / w_par.sum() - 1) > 1e-3
    abi.mem_process_set_pdf_grid(integ.proc, None)
    assert np.array_equal(integ.eval_points(0, 0, 5, 0, 1024), w_par)
    integ.close()
    ref.close()


def test_integral_frozen_grid_with_table(env):
    abi, synth, O, grid = env
    recs, integ, P, T = _setup(env, 1, 1, 4300)
    r = O.integrate(P, T, recs, seed=8, n_points=40000, n_adapt_iters=4, adapt_points=8192,
                    want_grids=True)
    n = 3 * 8192 + 777
    g = integ.integrate(n, seed=21, opts=abi.make_opts(n_adapt_iters=0, grid_in=r["grids"][0]))
    o = O.integrate(P, T, recs, seed=21, n_points=n, n_adapt_iters=0, grid_in=r["grids"][0])
    assert g["prob"][0] == pytest.approx(o["prob"][0], rel=1e-6, abs=0)
    assert g["status"][0] == 0
    integ.close()


def test_parton_level_with_table(env):
    abi, synth, O, grid = env
    recs = synth.gen_ttbar_parton(513, 77)
    integ = abi.Integrator(2, recs, synth.DEFAULT_PROCESS, synth.DEFAULT_TF[2], pdf_grid=grid)
    prob, w, st = integ.parton_weights()
    integ.close()
    P = O.process(2, synth.DEFAULT_PROCESS, pdf_grid=grid)
    prob_o, w_o = O.parton_batch(P, recs)
    assert np.all(st == 0)
    assert np.max(np.abs(prob / prob_o - 1)) < 1e-4


def test_invalid_tables_rejected(env):
    abi, synth, O, grid = env
    proc = abi.mem_create_process(abi.process_desc(0, synth.DEFAULT_PROCESS))
    bad = dict(grid, table=grid["table"][:, :1, :])            # n_q = 1
    with pytest.raises(abi.MemError):
        abi.mem_process_set_pdf_grid(proc, bad)
    neg = dict(grid, table=grid["table"].copy())
    neg["table"][1, 3, 7] = -1.0
    with pytest.raises(abi.MemError):
        abi.mem_process_set_pdf_grid(proc, neg)
    with pytest.raises(abi.MemError):
        abi.mem_process_set_pdf_grid(proc, dict(grid, lx=(-5.0, 0.5)))  # x beyond 1
    abi.mem_destroy(proc)

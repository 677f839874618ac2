"""The multi-GPU path on CPU ranks (gloo, world size 2): events are independent
integrals, so the job shards events over ranks with disjoint Philox event ids
(no collective on the data path) and reduces only the timing (max over ranks).

* Two ranks integrating halves of an event list with event_id_base offsets give
  bit-identical results to one process integrating the whole list (the oracle
  stands in for the device integrator: it follows the same counter layout).
* The max-over-ranks reduction that bench.py applies to step times returns the
  slowest rank's time on every rank.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

WORLD = 2
N_PER_RANK = 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        import bench
        from oracle import oracle as O
        from paper_1407_7595_gb300 import synth
        kind = synth.PROC_W
        recs = synth.gen_events(kind, WORLD * N_PER_RANK, 4242)
        sh = bench.shard(rank, N_PER_RANK)
        mine = recs[rank * N_PER_RANK:(rank + 1) * N_PER_RANK]
        P = O.process(kind, synth.DEFAULT_PROCESS)
        T = O.tf(synth.DEFAULT_TF[kind])
        r = O.integrate(P, T, mine, seed=11, n_points=2048, n_adapt_iters=1, adapt_points=512,
                        event_id_base=sh["event_id_base"], n_threads=1)
        parts = [None] * WORLD
        dist.all_gather_object(parts, (rank, r["prob"].tolist(), r["err"].tolist()))
        t_max = bench.max_over_ranks(10.0 + rank, WORLD, "cpu")
        np.save(os.path.join(out_dir, f"rank{rank}.npy"),
                np.array([[p for _, pr, _ in sorted(parts) for p in pr],
                          [e for _, _, er in sorted(parts) for e in er]]))
        np.save(os.path.join(out_dir, f"tmax{rank}.npy"), np.array([t_max]))
    finally:
        dist.destroy_process_group()


def test_event_shards_match_single_process(tmp_path):
    from oracle import oracle as O
    from paper_1407_7595_gb300 import synth
    port = _free_port()
    mp.start_processes(_rank_main, args=(port, str(tmp_path)), nprocs=WORLD, join=True,
                       start_method="spawn")
    kind = synth.PROC_W
    recs = synth.gen_events(kind, WORLD * N_PER_RANK, 4242)
    P = O.process(kind, synth.DEFAULT_PROCESS)
    T = O.tf(synth.DEFAULT_TF[kind])
    whole = O.integrate(P, T, recs, seed=11, n_points=2048, n_adapt_iters=1, adapt_points=512,
                        event_id_base=0, n_threads=1)
    for rank in range(WORLD):
        got = np.load(tmp_path / f"rank{rank}.npy")
        assert np.array_equal(got[0], whole["prob"])
        assert np.array_equal(got[1], whole["err"])
        assert float(np.load(tmp_path / f"tmax{rank}.npy")[0]) == 10.0 + (WORLD - 1)


# ---- cost-balanced split of one event list (paper_1407_7595_gb300.shard) ----

def _brute_best(costs, world):
    """Smallest possible largest range cost over all contiguous splits (DP)."""
    n = len(costs)
    pre = np.concatenate([[0], np.cumsum(costs)])
    INF = float("inf")
    best = [[INF] * (n + 1) for _ in range(world + 1)]
    best[0][0] = 0
    for r in range(1, world + 1):
        for j in range(n + 1):
            for i in range(j + 1):
                if best[r - 1][i] < INF:
                    best[r][j] = min(best[r][j], max(best[r - 1][i], pre[j] - pre[i]))
    return best[world][n]


def test_balanced_ranges_are_optimal_contiguous_and_complete():
    from paper_1407_7595_gb300 import shard
    rng = np.random.default_rng(3)
    for trial in range(60):
        n = int(rng.integers(0, 12))
        world = int(rng.integers(1, 5))
        costs = rng.integers(0, 50, size=n)
        ranges = shard.balanced_ranges(costs, world)
        assert len(ranges) == world
        assert ranges[0][0] == 0 and ranges[-1][1] == n
        for (a, b), (c, _) in zip(ranges, ranges[1:]):
            assert a <= b == c
        loads = [int(costs[a:b].sum()) for a, b in ranges]
        if n:
            assert max(loads) == _brute_best(costs, world)


def test_event_cost_is_dims_perms_points():
    from paper_1407_7595_gb300 import shard, synth
    c = shard.event_cost([synth.PROC_DY, synth.PROC_W, synth.PROC_TTBAR], [100, 10, 1])
    assert list(c) == [2 * 1 * 100, 4 * 1 * 10, 7 * 24 * 1]


MIX = [(0, 4), (1, 3), (2, 1)]    # (kind, events): the list is grouped by kind
PTS = 128


def _mix_list(synth):
    kinds, recs = [], []
    for k, n in MIX:
        recs.append(synth.gen_events(k, n, 5100 + k))
        kinds += [k] * n
    return np.array(kinds), np.concatenate(recs)


def _integrate_range(O, synth, kinds, recs, start, stop):
    """Oracle integration of events [start, stop), kind segment by kind segment,
    event ids = global indices."""
    out = {"prob": np.zeros(stop - start), "err": np.zeros(stop - start)}
    i = start
    while i < stop:
        j = i
        while j < stop and kinds[j] == kinds[i]:
            j += 1
        k = int(kinds[i])
        r = O.integrate(O.process(k, synth.DEFAULT_PROCESS), O.tf(synth.DEFAULT_TF[k]), recs[i:j],
                        seed=13, n_points=PTS, n_adapt_iters=1, adapt_points=64,
                        event_id_base=i, n_threads=1)
        out["prob"][i - start:j - start] = r["prob"]
        out["err"][i - start:j - start] = r["err"]
        i = j
    return out


def _split_main(rank, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        from oracle import oracle as O
        from paper_1407_7595_gb300 import shard, synth
        kinds, recs = _mix_list(synth)
        costs = shard.event_cost(kinds, PTS)
        start, stop = shard.my_range(costs, rank, WORLD)
        mine = _integrate_range(O, synth, kinds, recs, start, stop)
        full = shard.gather_results(mine, start, stop, len(kinds), WORLD)
        if rank == 0:
            np.save(os.path.join(out_dir, "gathered.npy"), np.array([full["prob"], full["err"]]))
        np.save(os.path.join(out_dir, f"range{rank}.npy"), np.array([start, stop]))
    finally:
        dist.destroy_process_group()


def test_cost_balanced_split_and_gather_match_single_process(tmp_path):
    from oracle import oracle as O
    from paper_1407_7595_gb300 import shard, synth
    port = _free_port()
    mp.start_processes(_split_main, args=(port, str(tmp_path)), nprocs=WORLD, join=True,
                       start_method="spawn")
    kinds, recs = _mix_list(synth)
    whole = _integrate_range(O, synth, kinds, recs, 0, len(kinds))
    got = np.load(tmp_path / "gathered.npy")
    assert np.array_equal(got[0], whole["prob"]) and np.array_equal(got[1], whole["err"])
    # the split follows the cost: the tt-bar event (7 x 24 x 128) weighs more than the
    # seven Drell-Yan and W events together, so it fills one rank
    r0, r1 = (tuple(np.load(tmp_path / f"range{r}.npy")) for r in range(WORLD))
    assert r0[1] == r1[0] and r0[0] == 0 and r1[1] == len(kinds)
    costs = shard.event_cost(kinds, PTS)
    assert max(costs[r0[0]:r0[1]].sum(), costs[r1[0]:r1[1]].sum()) == _brute_best(costs, WORLD)

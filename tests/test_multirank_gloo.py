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

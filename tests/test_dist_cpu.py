"""The multi-rank path of bench.py on the CPU: two `gloo` ranks (spawned
processes, rendezvous on 127.0.0.1) go through bench.py's own process-group
set-up, barrier and the max / sum reductions that turn per-rank step times and
evaluation counts into the whole-job value (weak scaling: every rank solves
its own replica, so value = evaluations of all ranks / slowest rank's time).
No GPU and no data-path collective is involved."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    os.environ.update({"WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    w, r, local, pg = bench.dist_setup()
    try:
        assert (w, r, local) == (world, rank, rank) and pg is not None
        bench.barrier(pg)
        step_ms = 10.0 * (rank + 1)          # rank 1 is the slowest
        evals = 1000.0 * (rank + 1)
        total = bench.max_over_ranks(pg, step_ms, "cpu")
        evals_all = bench.sum_over_ranks(pg, evals, "cpu")
        results[rank] = (total, evals_all, evals_all / (total / 1e3))
        bench.barrier(pg)
    finally:
        pg.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_work():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    results = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, results), nprocs=world, join=True,
                       start_method="spawn")
    assert set(results.keys()) == {0, 1}
    for r in range(world):
        total, evals_all, value = results[r]
        assert total == 20.0 and evals_all == 3000.0
        assert abs(value - 3000.0 / 0.020) < 1e-6


def test_single_process_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    import bench
    world, rank, local, pg = bench.dist_setup()
    assert (world, rank, local, pg) == (1, 0, 0, None)
    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5
    assert bench.sum_over_ranks(None, 2.0, "cpu") == 2.0

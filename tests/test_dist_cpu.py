"""The multi-rank path of bench.py on the CPU: two `gloo` ranks (spawned
processes, rendezvous on 127.0.0.1) go through bench.py's own process-group
set-up, barrier and the max / sum reductions that turn per-rank step times and
evaluation counts into the whole-job value (value = evaluations of all ranks /
slowest rank's time), and through the sharding of work units
(paper_2101_12348_gb300/shard.py): each rank takes its part of a survey's
curves (balanced by cost) or of a bank's templates (strided), produces
per-unit results, and rank 0 merges the parts into the single-rank layout.
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


def _fake_results(idx):
    """Per-unit results of a fake computation: two values a unit, from its index."""
    import numpy as np
    idx = np.asarray(idx, dtype=np.int64)
    return np.stack([np.sin(0.37 * idx), idx * 0.5 + 3.0], axis=1)


def _shard_rank_main(rank, world, port, results):
    os.environ.update({"WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import numpy as np

    import bench
    from paper_2101_12348_gb300 import shard
    w, r, local, pg = bench.dist_setup()
    try:
        rng = np.random.default_rng(5)
        cost = rng.lognormal(0.0, 1.0, 301)        # a survey's uneven curves
        curves = shard.partition_by_cost(cost, world)[rank]
        got = shard.gather_to_root(pg, (curves, _fake_results(curves)), rank, world)
        tpls = shard.partition_strided(32, world)[rank]
        got_t = shard.gather_to_root(pg, (tpls, _fake_results(tpls)), rank, world)
        if rank == 0:
            results["curves"] = shard.merge_parts(cost.size, got)
            results["templates"] = shard.merge_parts(32, got_t)
            results["parts"] = [g[0] for g in got]
        bench.barrier(pg)
    finally:
        pg.destroy_process_group()


def test_two_gloo_ranks_shard_and_merge():
    import numpy as np

    from paper_2101_12348_gb300 import shard
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    results = mgr.dict()
    mp.start_processes(_shard_rank_main, args=(world, port, results), nprocs=world, join=True,
                       start_method="spawn")
    # the merged parts equal what one rank computes over every unit
    np.testing.assert_array_equal(results["curves"], _fake_results(np.arange(301)))
    np.testing.assert_array_equal(results["templates"], _fake_results(np.arange(32)))
    parts = results["parts"]
    assert sum(p.size for p in parts) == 301
    assert np.intersect1d(parts[0], parts[1]).size == 0
    cost = np.random.default_rng(5).lognormal(0.0, 1.0, 301)
    loads = shard.part_loads(cost, parts)
    assert loads.max() - loads.min() <= cost.max()  # greedy LPT bound


def test_partitions_are_disjoint_covering_and_balanced():
    import numpy as np

    from paper_2101_12348_gb300 import shard
    rng = np.random.default_rng(9)
    for world in (1, 2, 3, 8):
        cost = rng.lognormal(0.0, 1.5, 1000)
        parts = shard.partition_by_cost(cost, world)
        cat = np.concatenate(parts)
        assert np.array_equal(np.sort(cat), np.arange(cost.size))
        loads = shard.part_loads(cost, parts)
        assert loads.max() - loads.min() <= cost.max()
        assert loads.max() <= cost.sum() / world + cost.max()
        st = shard.partition_strided(32, world)
        assert np.array_equal(np.sort(np.concatenate(st)), np.arange(32))
        assert max(p.size for p in st) - min(p.size for p in st) <= 1
    with pytest.raises(ValueError):  # overlapping parts
        shard.merge_parts(4, [(np.array([0, 1]), np.zeros(2)), (np.array([1, 2, 3]), np.zeros(3))])
    with pytest.raises(ValueError):  # a unit missing
        shard.merge_parts(4, [(np.array([0, 1]), np.zeros(2)), (np.array([3]), np.zeros(1))])


def test_single_process_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    import bench
    world, rank, local, pg = bench.dist_setup()
    assert (world, rank, local, pg) == (1, 0, 0, None)
    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5
    assert bench.sum_over_ranks(None, 2.0, "cpu") == 2.0

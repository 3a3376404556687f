"""The multi-rank bench path on CPU: two gloo ranks, each with its own
(different) duration; the job's duration is the maximum and its throughput
counts every rank's work (weak scaling, no data-path collective)."""
import os
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 1000.0 + 500.0 * rank
    total = bench.max_over_ranks(local_ms, dist)
    value = bench.job_throughput(1e9, world, 3, total)
    out[rank] = (total, value)
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    port = 29500 + os.getpid() % 1000
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for rank in range(2):
        total, value = out[rank]
        assert total == pytest.approx(1500.0)
        assert value == pytest.approx(1e9 * 2 * 3 / 1.5)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(100.0, 1, 2, 1000.0) == pytest.approx(200.0)


def _shard_worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    import oracle as O

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    systems = [(4, 1.5, 0.0, 61), (4, 0.9, 0.2, 40)]  # (L, T, h, paths of the whole ensemble)
    # this rank's share of every system (the system index is part of the
    # random-number counter, so each rank runs the whole batch)
    shares = [bench.rank_path_range(P, rank, world, weak=False) for (_, _, _, P) in systems]
    mine = O.run([O.System(L, T, h=h, n_paths=P, path_begin=b, path_count=c)
                  for (L, T, h, P), (b, c) in zip(systems, shares)], 20, 30, seed=4)
    gathered = [bench.gather_records(r, dist) for r in mine]
    out[rank] = gathered
    dist.destroy_process_group()


def test_two_gloo_ranks_split_one_ensemble():
    """Two ranks run disjoint path-id ranges of the same systems and seed; the
    gathered records equal those of one process running every path, bit for
    bit, and so do the estimates."""
    sys.path.insert(0, ROOT)
    import oracle as O

    port = 29500 + (os.getpid() + 7) % 1000
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_shard_worker, args=(2, port, out), nprocs=2, join=True)
    whole = O.run([O.System(4, 1.5, n_paths=61), O.System(4, 0.9, h=0.2, n_paths=40)], 20, 30, seed=4)
    for rank in range(2):
        for k, (T, P) in enumerate(((1.5, 61), (0.9, 40))):
            got = out[rank][k]
            assert got.shape == (P, O.NREC)
            np.testing.assert_array_equal(got, whole[k])
            a, b = O.estimates(got, 64, T), O.estimates(whole[k], 64, T)
            assert all(a[key] == b[key] or (np.isnan(a[key]) and np.isnan(b[key])) for key in a)


def test_rank_path_ranges():
    sys.path.insert(0, ROOT)
    import bench

    assert [bench.rank_path_range(10, r, 3, weak=False) for r in range(3)] == [(0, 4), (4, 3), (7, 3)]
    assert [bench.rank_path_range(4096, r, 4) for r in range(4)] == [(0, 4096), (4096, 4096), (8192, 4096),
                                                                     (12288, 4096)]

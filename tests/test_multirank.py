"""The multi-rank bench path on CPU: two gloo ranks, each with its own
(different) duration; the job's duration is the maximum and its throughput
counts every rank's work (weak scaling, no data-path collective)."""
import os
import sys

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

"""The multi-GPU leg of bench.py runs independent replicas (the path has no exchange step): check
its rank logic, the max-over-ranks step time and the whole-job value, on two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 2.0 + rank  # rank 1 is slower
    ms = bench.max_over_ranks(local_ms, dist, torch.device("cpu"))
    value = bench.job_value(62.4, world, ms)
    results[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of this multi-threaded process
        results = m.dict()
        mp.spawn(_rank_main, args=(world, port, results), nprocs=world, join=True)
        res = dict(results)
    assert res[0][0] == res[1][0] == 3.0
    assert abs(res[0][1] - 2 * 62.4 / 3.0e-3) < 1e-6


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(1.5, None, None) == 1.5
    assert bench.job_value(10.0, 1, 2.0) == 5000.0

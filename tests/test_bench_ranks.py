"""Host-side multi-process timing helpers of bench.py on CPU (gloo, world size 2).

With N GPUs every rank times its own steps and the slowest rank's time sets the job's time
(the max over ranks); replicated workloads (the batched configuration) count every rank's work
in the whole-job throughput.  These two host steps are exercised here with two gloo ranks; the
pole-sharded exchange is in test_pole_shard_ranks.py.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench._max_over_ranks(10.0 + 5.0 * rank, dist, world, torch.device("cpu"))
        out[rank] = (t, bench._job_value(1000, world, t))
    finally:
        dist.destroy_process_group()


def test_replica_timing_two_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    # both ranks see the slowest replica's time; throughput counts both replicas' work
    assert out[0] == out[1]
    t, v = out[0]
    assert t == 15.0
    assert abs(v - 2 * 1000 / 15e-3) < 1e-6


def test_single_rank_helpers():
    import bench
    assert bench._max_over_ranks(3.5, None, 1, None) == 3.5
    assert abs(bench._job_value(81 * 4096, 1, 45.5) - 81 * 4096 / 45.5e-3) < 1e-6

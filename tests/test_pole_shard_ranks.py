"""Pole-sharded density on several processes, host side on CPU (gloo, world size 2 and 3).

The poles of Eq. 8 are independent (Sec. III.D): each rank sums its share of the points
(ndsi_pole_shard picks the share, ndsi_density_poles computes it on the GPU) and one sum
all-reduce of rho and Tr(rho S) gives the whole result.  Here every rank takes the share the
library assigns, sums the oracle's per-pole terms of that share, and the ranks exchange their
partial sums through bench.py's all-reduce helper; the total must equal the single-process
oracle result.
"""
import os
import socket

import numpy as np
import pytest

from tests.libtools import lib


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _system():
    from synth import lattice_system
    return lattice_system((4, 3, 1), 2, "2d", 4242)


MU, KT, M = -0.05, 0.02, 9


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    from oracle.dense import density_inv_terms, on_pattern
    nd = lib()
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = _system()
        Hd, Sd = s.dense()
        terms = density_inv_terms(Hd, Sd, MU, KT, M)   # [M0, pole 1, ..., pole M]
        b, e, m0 = nd.ndsi_pole_shard(M, rank, world)
        part = np.zeros_like(Hd)
        if m0:
            part += terms[0]
        for p in range(b, e):
            part += terms[1 + p]
        rho = on_pattern(part, s)
        buf = torch.tensor(np.concatenate([rho, [float(np.dot(rho, s.S))]]), dtype=torch.float64)
        bench._sum_over_ranks(buf, dist, world)
        out[rank] = (b, e, m0, buf.numpy().tolist())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_pole_shards_sum_to_single_rank_density(world):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from oracle.dense import density_inv, on_pattern
    lib()                                   # build once before the ranks start
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    s = _system()
    Hd, Sd = s.dense()
    ref = on_pattern(density_inv(Hd, Sd, MU, KT, M), s)
    # the shares partition the poles and exactly one rank holds M0
    ranges = sorted((out[r][0], out[r][1]) for r in range(world))
    assert ranges[0][0] == 0 and ranges[-1][1] == M
    assert all(ranges[i][1] == ranges[i + 1][0] for i in range(world - 1))
    assert sum(out[r][2] for r in range(world)) == 1
    for r in range(world):
        tot = np.asarray(out[r][3])
        assert np.max(np.abs(tot[:-1] - ref)) < 1e-14
        assert abs(tot[-1] - float(np.dot(ref, s.S))) < 1e-12


@pytest.mark.parametrize("M", [1, 2, 7, 40, 80, 160])
@pytest.mark.parametrize("world", [1, 2, 3, 8, 12])
def test_pole_shard_partition(M, world):
    nd = lib()
    shares = [nd.ndsi_pole_shard(M, r, world) for r in range(world)]
    assert shares[0][0] == 0 and shares[-1][1] == M
    counts = []
    for r in range(world):
        b, e, _ = shares[r]
        assert b <= e
        if r:
            assert b == shares[r - 1][1]
        counts.append(e - b)
    assert max(counts) - min(counts) <= 1
    m0 = [r for r in range(world) if shares[r][2]]
    assert len(m0) == 1
    # M0 sits on a rank with the fewest poles, so the points per rank differ by at most one
    points = [c + (1 if r == m0[0] else 0) for r, c in enumerate(counts)]
    assert max(points) - min(points) <= 1


def test_pole_shard_rejects_bad_arguments():
    nd = lib()
    for args in [(0, 0, 1), (10, 2, 2), (10, -1, 2), (10, 0, 0)]:
        with pytest.raises(nd.NdsiError):
            nd.ndsi_pole_shard(*args)

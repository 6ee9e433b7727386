"""Multi-rank host logic on CPU (gloo, world size 2): work split and timing reductions."""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp

from paper_2401_14564_gb300 import dist as ppd


def test_shard_covers_every_unit_once():
    for n in (0, 1, 7, 1024, 1025):
        for world in (1, 2, 3, 8):
            parts = [ppd.shard(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        ppd.shard(10, 2, 2)


def test_reductions_without_a_group_are_identity():
    assert ppd.max_over_ranks(3.5) == 3.5 and ppd.sum_over_ranks(2.0) == 2.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [1.5, 2.25][rank]  # per-rank step time
        units = 1000
        start, stop = ppd.shard(units, rank, world)
        got = ppd.sum_over_ranks(stop - start)
        slowest = ppd.max_over_ranks(ms)
        # whole-job throughput as the benchmark reports it: all ranks' units over the slowest rank
        q.put((rank, got, slowest, world * units / (slowest * 1e-3)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, slowest, value in res:
        assert total == 1000
        assert slowest == 2.25
        assert value == pytest.approx(2 * 1000 / 2.25e-3)

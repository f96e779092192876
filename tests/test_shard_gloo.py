"""Host logic of the multi-GPU path, on CPU: two gloo ranks shard a frequency grid (disjoint,
covering, contiguous, balanced), reduce their step times to the maximum, and agree on the
whole-job throughput."""
import os
import socket

import numpy as np
import pytest

from paper_1511_04355_gb300 import shard as SH


def test_shard_bounds_cover_and_balance():
    for n in (0, 1, 7, 128, 256, 1000):
        for world in (1, 2, 3, 8):
            parts = [SH.shard_bounds(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        SH.shard_bounds(10, 2, 2)
    assert SH.aggregate_rate(128, 4, 2.0) == 256.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        grid = W.fsm_frequencies(0.02, 250.0, 128 * world)
        mine = SH.shard(grid, rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine.tolist())
        t = SH.max_over_ranks(1.0 + rank)            # rank r "took" 1 + r seconds
        out.put((rank, gathered, t, SH.aggregate_rate(len(mine), world, t)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp

    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import workloads as W
    grid = W.fsm_frequencies(0.02, 250.0, 128 * world)
    for rank, gathered, t, rate in res:
        allf = np.concatenate([np.array(g) for g in gathered])
        assert np.array_equal(allf, grid)            # disjoint, covering, in order
        assert all(len(g) == 128 for g in gathered)
        assert t == 2.0                              # the slowest rank's time on every rank
        assert rate == 128 * world / 2.0

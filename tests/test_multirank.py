"""Several ranks on the CPU (gloo, world size 2): the host logic bench.py uses
with one process per GPU. The explicit step runs one replica per rank and the
ranks meet only to take the slowest rank's time; the request mix is sharded
round robin with no collective until the totals are combined."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench
    from paper_1806_06917_gb300 import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [1.5, 4.0][rank]
        ms = bench.rank_reduce(torch, local_ms, "max", "cpu")
        work = bench.rank_reduce(torch, 100.0 * (rank + 1), "sum", "cpu")
        mix = W.serving_mix(count=11, side_median=10.0, side_lo=6, side_hi=12, steps_lo=1, steps_hi=3)
        mine = bench.shard(mix, rank, world)
        seeds = [r.seed for r in mine]
        parts = [None] * world
        dist.all_gather_object(parts, seeds)
        out[rank] = (ms, work, parts)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_shard_the_mix():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert set(res) == {0, 1}
    for rank in range(world):
        ms, work, parts = res[rank]
        assert ms == 4.0 and work == 300.0
        # every request in exactly one shard, in round-robin order
        allseeds = parts[0] + parts[1]
        assert len(allseeds) == 11 and len(set(allseeds)) == 11
        assert len(parts[0]) == 6 and len(parts[1]) == 5


def test_one_process_needs_no_process_group():
    import bench
    assert bench.rank_reduce(torch, 2.5, "max", "cpu") == 2.5
    assert bench.shard(list(range(7)), 0, 1) == list(range(7))
    assert bench.shard(list(range(7)), 1, 3) == [1, 4]

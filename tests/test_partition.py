"""Host logic of the multi-rank path: sharding covers every unit once, and a two-rank gloo
group reduces the per-rank timings with a max, as bench.py does."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1812_03717_gb300.partition import block_range, units_for_step


@pytest.mark.parametrize("n,world", [(0, 1), (7, 1), (7, 2), (2048, 3), (5, 8)])
def test_block_range_covers_once(n, world):
    seen = []
    for r in range(world):
        lo, hi = block_range(n, world, r)
        seen.extend(range(lo, hi))
        assert hi - lo in (n // world, n // world + 1)
    assert seen == list(range(n))


def test_units_for_step_weak_scaling():
    # 4 k-points, 2 ranks: each step covers two distinct units, two steps cover all four
    got = [[units_for_step(s, 2, r, 4) for r in range(2)] for s in range(2)]
    assert got == [[0, 1], [2, 3]]
    with pytest.raises(ValueError):
        units_for_step(0, 2, 2, 4)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units = [units_for_step(s, world, rank, 4) for s in range(2)]
    t = torch.tensor([10.0 * (rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    all_units = [None] * world
    dist.all_gather_object(all_units, units)
    if rank == 0:
        q.put((float(t.item()), all_units))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_sharding_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    tmax, units = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert tmax == 20.0
    flat = sorted(u for us in units for u in us)
    assert flat == [0, 1, 2, 3]

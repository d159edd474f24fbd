"""Host logic of the multi-rank path: sharding covers every unit once, a two-rank gloo group
reduces the per-rank timings with a max, as bench.py does, and the k-point sum of the
density response (Eq. 5) over ranks equals the single-process sum."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1812_03717_gb300.partition import allreduce_density, block_range, units_for_step


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


def _density_contribution(k):
    """A seeded stand-in for one k-point's contribution dn_k[G][G'][omega]."""
    g = torch.Generator().manual_seed(100 + k)
    re = torch.randn(5, 5, 3, generator=g, dtype=torch.float64)
    im = torch.randn(5, 5, 3, generator=g, dtype=torch.float64)
    return torch.complex(re, im)


def _density_worker(rank, world, port, nk, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dn = torch.zeros(5, 5, 3, dtype=torch.complex128)
    lo, hi = block_range(nk, world, rank)
    for k in range(lo, hi):
        dn += _density_contribution(k)
    allreduce_density(dn)
    # a non-contiguous slice is refused before any communication
    wide = torch.zeros(5, 10, 3, dtype=torch.complex128)
    try:
        allreduce_density(wide[:, ::2])
        refused = False
    except ValueError:
        refused = True
    q.put((rank, dn.numpy(), refused))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_density_allreduce_equals_serial_sum():
    nk, world = 5, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_density_worker, args=(r, world, port, nk, q)) for r in range(world)]
    for p in procs:
        p.start()
    items = [q.get(timeout=120) for _ in range(world)]
    got = {r: d for r, d, _ in items}
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(refused for _, _, refused in items)
    serial = sum(_density_contribution(k) for k in range(nk)).numpy()
    for r in range(world):
        assert abs(got[r] - serial).max() <= 1e-12 * abs(serial).max()


def test_density_allreduce_single_process_is_identity():
    dn = _density_contribution(0)
    before = dn.clone()
    assert allreduce_density(dn) is dn
    assert torch.equal(dn, before)

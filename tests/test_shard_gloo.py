"""Multi-GPU sharding logic, run as two gloo ranks on the CPU: every tile
lands in exactly one shard and shard loads differ by at most one tile."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from paper_1405_7958_gb300.shard import lpt_shards


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, sizes, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = lpt_shards(sizes, world)[rank]
    got = [None] * world
    dist.all_gather_object(got, mine)
    load = torch.tensor([sum(sizes[i][0] * sizes[i][1] for i in mine)], dtype=torch.int64)
    loads = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(loads, load)
    if rank == 0:
        q.put((got, [int(x.item()) for x in loads]))
    dist.destroy_process_group()


def test_shards_cover_tiles_once_and_balance():
    sizes = [(H, W) for H, W, _, _ in synth.batch_sizes(64, 3)]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, sizes, q)) for r in range(world)]
    for p in procs:
        p.start()
    got, loads = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(i for s in got for i in s)
    assert flat == list(range(len(sizes)))
    assert max(loads) - min(loads) <= max(H * W for H, W in sizes)


def test_lpt_single_rank_is_identity():
    sizes = [(10, 10), (5, 5), (7, 3)]
    assert lpt_shards(sizes, 1) == [[0, 1, 2]]
    with pytest.raises(ValueError):
        lpt_shards(sizes, 0)

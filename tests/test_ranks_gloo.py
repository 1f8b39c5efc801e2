"""Multi-rank host logic on CPU: two gloo ranks (one process per GPU in a real run).

The product exchanges no data between ranks; the ranks share only the bench's bookkeeping: the
timed region counts as long as its slowest rank, and independent units are split into blocks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1303_1651_gb300 import ranks


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # the slowest rank decides the time
        t = ranks.max_over_ranks(1.5 + rank, dist, "cpu")
        # every unit lands on exactly one rank, in rank order
        mine = list(ranks.shard_range(1001, rank, world))
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        out.put((rank, t, gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, gathered in results:
        assert t == 1.5 + (world - 1)
        flat = [u for block in gathered for u in block]
        assert flat == list(range(1001))


def test_shard_range_properties():
    for n in (0, 1, 5, 31, 1000):
        for world in (1, 2, 3, 8):
            blocks = [ranks.shard_range(n, r, world) for r in range(world)]
            assert [u for b in blocks for u in b] == list(range(n))
            sizes = [len(b) for b in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        ranks.shard_range(10, 2, 2)


def test_single_process_is_identity():
    assert ranks.max_over_ranks(3.25) == 3.25

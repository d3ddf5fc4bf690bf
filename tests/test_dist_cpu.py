"""Channel sharding and the max-over-ranks timing reduction, on CPU with gloo
(world size 2): ranks hold disjoint channels and agree on the slowest time."""
import os
import socket

import pytest

from paper_1702_04728_gb300 import dist as D

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    chans = D.rank_channels(rank, world)
    times = [1.0 + rank, 10.0 - rank]
    mx = D.max_over_ranks(times)
    gathered = [None] * world
    dist.all_gather_object(gathered, chans)
    q.put((rank, chans, mx, gathered))
    dist.destroy_process_group()


def test_two_ranks_disjoint_channels_and_max_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    all_chans = [c for _, chans, _, _ in res for c in chans]
    assert len(set(all_chans)) == 8                          # disjoint
    for rank, chans, mx, gathered in res:
        assert mx == [2.0, 10.0]                              # slowest rank decides
        assert gathered[rank] == chans
    assert res[0][1] == list(D.NODE_SLICE_HZ)


def test_rank_channels_single_and_bounds():
    assert D.rank_channels(0, 1) == list(D.NODE_SLICE_HZ)
    with pytest.raises(ValueError):
        D.rank_channels(2, 2)
    assert D.max_over_ranks([3.0]) == [3.0]

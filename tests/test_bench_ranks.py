"""The multi-rank path of bench.py on CPU: two gloo ranks agree on the
slowest rank's time and report the whole-job throughput (no GPU involved)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [2.0, 3.5][rank]  # rank 1 is the slower one
    slowest = bench.max_over_ranks(ms, world)
    value = bench.job_throughput(1000000, world, slowest)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, slowest, value))


def test_two_gloo_ranks_take_the_slowest_time():
    import multiprocessing as mp
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, value in res:
        assert slowest == 3.5
        assert value == pytest.approx(2 * 1000000 / 3.5e-3 / 1e6)


def _shard_rank(rank, world, port, q):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    from paper_1606_07414_gb300 import shard, synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    Hs, Ws = synth.uneven_sizes(9, 500)
    blocks = [int(h) // 16 * (int(w) // 16) for h, w in zip(Hs, Ws)]
    mine = shard.rank_images(blocks, rank, world)
    # every rank's list, gathered: each image must be coded exactly once
    n = torch.tensor([len(mine)])
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n)
    m = int(max(s.item() for s in sizes))
    padded = torch.full((m,), -1, dtype=torch.int64)
    padded[:len(mine)] = torch.tensor(mine, dtype=torch.int64)
    lists = [torch.zeros(m, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(lists, padded)
    dist.barrier()
    dist.destroy_process_group()
    got = [[int(x) for x in t.tolist() if x >= 0] for t in lists]
    q.put((rank, got, blocks))


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_images_are_coded_exactly_once(world):
    """Ranks computing their shards of one image list on their own (no
    communication) cover every image exactly once, and the busiest rank holds
    at most the mean plus the largest image."""
    import multiprocessing as mp
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    got, blocks = res[0][1], res[0][2]
    for _, g, _ in res:
        assert g == got  # every rank gathered the same lists
    flat = sorted(i for lst in got for i in lst)
    assert flat == list(range(len(blocks)))
    loads = [sum(blocks[i] for i in lst) for lst in got]
    assert max(loads) <= sum(blocks) / world + max(blocks)


def test_shard_images_host_rules():
    sys.path.insert(0, ROOT)
    from paper_1606_07414_gb300 import shard

    assert shard.shard_images([], 3) == [[], [], []]
    assert shard.shard_images([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]
    assert shard.shard_images([1, 9, 4], 1) == [[0, 1, 2]]
    assert shard.shard_images([7, 0, 3, 3], 2) == [[0], [1, 2, 3]]
    with pytest.raises(ValueError):
        shard.shard_images([1], 0)
    with pytest.raises(ValueError):
        shard.rank_images([1, 2], 2, 2)

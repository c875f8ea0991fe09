"""Multi-rank host logic on CPU (gloo, world size 2): latent sharding covers
every latent exactly once with no exchange, and the benchmark's timing
reduction takes the maximum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2509_18815_gb300.dist import shard


def test_shard_partitions_items():
    for n in [0, 1, 5, 64, 65]:
        for world in [1, 2, 3, 8]:
            seen = []
            for r in range(world):
                seen.extend(shard(n, r, world))
            assert seen == list(range(n))
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2509_18815_gb300.dist import max_over_ranks, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = list(shard(64, rank, world))
    # each rank reports a different per-step time; all must see the max
    vals = max_over_ranks([1.0 + rank, 10.0 - rank])
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mine, vals))


def test_two_rank_gloo_timing_and_sharding():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert out[0][1] + out[1][1] == list(range(64))
    for _, _, vals in out:
        assert vals == [2.0, 10.0]

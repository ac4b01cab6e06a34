"""The N > 1 bench path on CPU: two gloo ranks (no GPU).  Views are sharded
round-robin with no data-path collective; the only collectives are the barrier
and the max-over-ranks of the timed region."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        poses = bench.shard_poses(64, rank, world)
        dist.barrier()
        t = bench.max_over_ranks(10.0 + rank, dist, "cpu")
        out.put((rank, poses, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_views_and_take_the_max():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    all_poses = sorted(res[0][1] + res[1][1])
    assert all_poses == list(range(64))
    assert not set(res[0][1]) & set(res[1][1])
    assert res[0][2] == res[1][2] == 11.0


@pytest.mark.parametrize("n,world", [(64, 1), (64, 3), (8, 8), (2, 4)])
def test_shard_poses_cover_once(n, world):
    shards = [bench.shard_poses(n, r, world) for r in range(world)]
    assert all(shards)
    if world <= n:
        flat = sorted(k for s in shards for k in s)
        assert flat == list(range(n))

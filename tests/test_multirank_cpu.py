"""The multi-rank bench path on CPU: gloo, world size 2, 127.0.0.1 rendezvous.

Replicas (one domain per rank, or a share of an ensemble's scenarios) exchange no
data; the only collective is the maximum of the ranks' timed seconds, from which
the whole-job throughput is computed.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local = [0.5, 0.8][rank]
    value, slowest = bench.whole_job_throughput(1000.0, local, world)
    idx = list(bench.shard(257, rank, world))
    sizes = torch.tensor([len(idx)], dtype=torch.int64)
    dist.all_reduce(sizes)
    out[rank] = (value, slowest, idx[0], idx[-1], int(sizes.item()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_and_sharding(repo_root):
    import sys

    sys.path.insert(0, repo_root)
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    v0, s0, a0, b0, tot = out[0]
    v1, s1, a1, b1, _ = out[1]
    assert s0 == s1 == 0.8  # slowest rank
    assert abs(v0 - 2 * 1000.0 / 0.8) < 1e-9 and v0 == v1
    assert (a0, b0, a1, b1) == (0, 128, 129, 256) and tot == 257


def test_shard_covers_every_item_once():
    import bench

    for n in (0, 1, 7, 256, 1000):
        for world in (1, 2, 3, 8):
            seen = [i for r in range(world) for i in bench.shard(n, r, world)]
            assert seen == list(range(n))

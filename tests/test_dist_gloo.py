"""Multi-process host logic on CPU (gloo, world size 2): the J sharding, the maximum of
the per-rank timings that bench.py reports, and the gather of per-J results."""
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


def _worker(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2412_10167_gb300 import dist as mdist
    try:
        assert mdist.rank_world() == (rank, world)
        Js = list(range(0, 31, 5))                       # 7 J values over 2 ranks
        mine = mdist.shard(Js, rank, world)
        everything = mdist.gather_by_key({J: J * 10 for J in mine})
        assert sorted(everything) == Js and all(v == J * 10 for J, v in everything.items())
        # the slowest rank sets the job time
        assert mdist.max_over_ranks(1.0 + rank) == float(world)
        mdist.barrier()
    finally:
        dist.destroy_process_group()


def test_shard_covers_each_item_once():
    from paper_2412_10167_gb300 import dist as mdist
    for n in range(0, 12):
        for world in range(1, 5):
            parts = [mdist.shard(range(n), r, world) for r in range(world)]
            assert sum(parts, []) == list(range(n))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1


def test_two_rank_gloo_gather_and_timing():
    mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)

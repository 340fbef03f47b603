"""The N > 1 path of the bench, on CPU with two gloo ranks: the evaluator
runs replicas (orders and instances are independent, no exchange on the
data path), so what crosses ranks is the instance sharding and the timing
and work reduction of the JSON line (max over ranks of the timed region,
sum of the solves).  127.0.0.1 rendezvous."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    mine = bench.shard(64, rank, world)
    # each rank's timed region and work differ; the line takes the max time
    # and the summed work
    t, (conv, iters) = bench.reduce_over_ranks(1.5 + rank, [100 * (rank + 1), 7 + rank], "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    out[rank] = (t, conv, iters, gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, conv, iters, gathered = res[rank]
        assert t == 2.5                       # max over ranks
        assert conv == 300 and iters == 15    # sums
        # replicas: every instance taken by exactly one rank
        allv = sorted(i for g in gathered for i in g)
        assert allv == list(range(64))
        assert gathered[0] == list(range(0, 64, 2)) and gathered[1] == list(range(1, 64, 2))


def test_single_process_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(0.25, [3, 4], "cpu") == (0.25, [3, 4])
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]

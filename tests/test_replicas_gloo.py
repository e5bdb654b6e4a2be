"""The multi-GPU path is independent replicas (pairs do not interact); its host
logic runs here as two gloo ranks on the CPU: every rank gets its own pairs,
and the job time is the maximum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ids = [i for s in range(3) for i in bench.pair_ids(rank, s, 8)]
    gathered = [None] * world
    dist.all_gather_object(gathered, ids)
    elapsed = 1.0 + rank  # a slower rank 1
    job = bench.reduce_max(dist, elapsed, "cpu")
    out[rank] = (gathered, job)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_pairs_and_take_the_max_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    gathered, job0 = res[0]
    _, job1 = res[1]
    assert job0 == job1 == 2.0
    a, b = set(gathered[0]), set(gathered[1])
    assert len(a) == 24 and len(b) == 24 and not (a & b)

"""The multi-GPU host logic (replicas, one process per GPU) on CPU: two gloo ranks shard events
without overlap, take the maximum of their times, and form the whole-job rate from it."""
import os
import socket

import pytest

from paper_1310_7556_gb300 import replicas


def test_event_indices_are_disjoint_and_cover_the_range():
    world, per = 4, 7
    shards = [replicas.event_indices(r, world, per, base=100) for r in range(world)]
    flat = [i for s in shards for i in s]
    assert flat == list(range(100, 100 + world * per))
    with pytest.raises(ValueError):
        replicas.event_indices(4, 4, 1)


def test_job_rate_is_units_over_the_slowest_rank():
    assert replicas.job_rate(10, 2, 0.5) == 40.0
    with pytest.raises(ValueError):
        replicas.job_rate(1, 1, 0.0)
    assert replicas.backend_for(False) == "gloo" and replicas.backend_for(True) == "nccl"


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group(replicas.backend_for(False), rank=rank, world_size=world)
    try:
        mine = replicas.event_indices(rank, world, 3)
        seconds = 0.25 * (rank + 1)            # rank 1 is the slower one
        slowest = replicas.max_over_ranks(dist, seconds)
        dist.barrier()
        out[rank] = (mine, slowest, replicas.job_rate(len(mine), world, slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_rate():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    port = _free_port()
    with mp.Manager() as manager:
        out = manager.dict()
        procs = [mp.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    assert res[0][0] == [0, 1, 2] and res[1][0] == [3, 4, 5]
    assert res[0][1] == res[1][1] == 0.5
    assert res[0][2] == res[1][2] == 3 * 2 / 0.5

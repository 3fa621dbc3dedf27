"""The multi-rank plumbing of bench.py on CPU: two gloo ranks agree on the
maximum of their step times and on the whole-job rate (all ranks' elements
over the slowest rank's time), as `bench.py --gpus N` computes them."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, results):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    seconds = 1.0 + rank            # rank 1 is the slow one
    slowest = bench.max_over_ranks(seconds, w)
    rate = bench.whole_job_rate(1000, w, slowest)
    dist.barrier()
    dist.destroy_process_group()
    results[rank] = (r, w, slowest, rate)


def test_two_gloo_ranks_take_the_slowest():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    results = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, results)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert results[0][:2] == (0, 2) and results[1][:2] == (1, 2)
    for r in range(world):
        assert results[r][2] == pytest.approx(2.0)
        assert results[r][3] == pytest.approx(1000 * 2 / 2.0)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0

"""The multi-GPU bench path is replicas only (no collective on the data path):
each rank segments its own field and the job is timed by its slowest rank.
Its host logic -- the max over ranks and the whole-job rate -- runs here as
two gloo ranks on the CPU."""
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


def _rank_main(rank, world, port, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        assert (ws, r, local) == (world, rank, rank)
        elapsed = 10.0 + 5.0 * rank  # the slower rank sets the time
        t = bench.max_over_ranks(elapsed, dist)
        rate = bench.whole_job_rate(1000.0, ws, t)
        out[rank] = (t, rate)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        t, rate = out[r]
        assert t == 15.0
        assert rate == pytest.approx(2 * 1000.0 / 15.0)


def test_single_process_is_its_own_max():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(100.0, 1, 2.0) == 50.0

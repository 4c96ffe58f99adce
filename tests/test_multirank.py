"""The multi-GPU bench path on CPU: two gloo ranks, each standing for one GPU
with its own volume (independent problems, weak scaling).  Checks the
whole-job reduction (slowest rank's time, sum of all ranks' updates) and that
the ranks get distinct problems.  No data-path collective exists to test."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = [1.5, 2.25, 0.5][rank]
        upd = [100, 250, 40][rank]
        s, u = bench.reduce_over_ranks(dist, world, secs, upd, "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(rank))
        out.put((rank, s, u, seeds))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_whole_job_reduction_over_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    secs = [1.5, 2.25, 0.5][:world]
    upd = [100, 250, 40][:world]
    for rank, s, u, seeds in res:
        assert s == max(secs)
        assert u == sum(upd)
        assert len(set(seeds)) == world       # every rank has its own problem


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks(None, 1, 3.0, 7, "cpu") == (3.0, 7.0)

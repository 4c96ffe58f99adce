"""Multi-rank paths on CPU (gloo ranks standing for GPUs).

- bench.py's path: one volume per rank (independent problems, weak scaling).
  The test checks the whole-job reduction (the slowest rank's time, the sum
  of all ranks' updates) and that every rank gets a distinct problem.
- One swarm split across ranks (paper_2002_01981_gb300.distributed): each
  rank evaluates its particles, the fitness values are all-gathered, and
  every rank steps the whole swarm.  The fitness and step functions here are
  the oracle's, so the host logic (partition, gather order, identical steps)
  is tested without a GPU."""
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


# ----------------------------------------------- one swarm split across ranks
def _split_worker(rank, world, port, out, P, gens):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import numpy as np
    from oracle import pso as OP
    from paper_2002_01981_gb300 import distributed as D
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x, U0, C0 = _tiny_problem()
        sw = OP.Swarm(P, seed=7)

        def fitness_fn(lo, hi):
            f, _ = OP.fitness_batch(x, U0, C0, sw.x[lo:hi], max_iter=4, eps=0.0)
            return torch.from_numpy(np.asarray(f, dtype=np.float64))

        def step_fn(f_all):
            OP.pso_step(sw, f_all.numpy())

        D.split_swarm(fitness_fn, step_fn, P, gens)
        out.put((rank, sw.x.copy(), sw.v.copy(), sw.pbest_x.copy(), sw.pbest_f.copy(), sw.gen))
    finally:
        dist.destroy_process_group()


def _tiny_problem():
    import numpy as np
    from oracle import ifcm as O
    from paper_2002_01981_gb300 import phantoms
    x = O.normalize(phantoms.brain_phantom((4, 6, 7), seed=3, sigma=0.05))
    U0, C0, _, _ = O.fcm_init(x, 3, max_iter=20)
    return x, U0, C0


def test_particle_slices_cover_the_swarm():
    from paper_2002_01981_gb300.distributed import particle_slice
    for P in (1, 5, 20, 33):
        for world in (1, 2, 3, 8):
            sl = [particle_slice(P, world, r) for r in range(world)]
            assert sl[0][0] == 0 and sl[-1][1] == P
            assert all(a[1] == b[0] for a, b in zip(sl, sl[1:]))
            sizes = [hi - lo for lo, hi in sl]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world", [2, 3])
def test_split_swarm_over_gloo_ranks_equals_one_process(world):
    # every rank evaluates its slice, the fitness values are all-gathered and
    # every rank steps the whole swarm: the swarms must equal a one-process
    # run bit for bit (the fitness values are the same FP64 numbers)
    import numpy as np
    from oracle import pso as OP
    P, gens = 7, 3
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_worker, args=(r, world, port, out, P, gens))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([out.get(timeout=300) for _ in range(world)], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    x, U0, C0 = _tiny_problem()
    ref = OP.Swarm(P, seed=7)
    for _ in range(gens):
        f, _ = OP.fitness_batch(x, U0, C0, ref.x, max_iter=4, eps=0.0)
        OP.pso_step(ref, f)
    for _, sx, sv, pbx, pbf, gen in res:
        assert np.array_equal(sx, ref.x) and np.array_equal(sv, ref.v)
        assert np.array_equal(pbx, ref.pbest_x) and np.array_equal(pbf, ref.pbest_f)
        assert gen == ref.gen

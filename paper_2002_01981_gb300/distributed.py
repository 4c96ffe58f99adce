"""One particle swarm split across the ranks of a torch.distributed group.

Algorithm 1 step 4 evaluates P independent fitnesses per generation.  With
one GPU per rank, each rank evaluates a contiguous slice of the particles
(``pso_fitness_batch`` on its slice).  The P fitness values are then
all-gathered, which is the only exchange of a generation.  Every rank then
runs the same swarm step (Algorithm 1 steps 5-8) on the whole swarm.  The
step draws p1 and p2 from Philox4x32-10, keyed by (seed, generation,
particle, dimension), so the swarms stay bit-identical on all ranks without
exchanging any other state.  Memberships never cross ranks: each rank holds
the volume and its own particles' buffers.

``split_swarm`` is the host loop, written against two callables so that it
runs the same way with the library's kernels (``pifcm3d_split``) and with any
other fitness and step functions.  ``allgather_fitness`` is the exchange:
NCCL tensors on GPUs, gloo on CPU.
"""
import torch

from . import ifcm as G


def particle_slice(P, world, rank):
    """Contiguous particles [lo, hi) of `rank`: sizes differ by at most one,
    and the lower ranks take the extra ones."""
    base, extra = divmod(int(P), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def allgather_fitness(local, P, group=None):
    """All ranks' fitness slices (float64, 1-D) joined in particle order."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    cap = -(-int(P) // world)
    buf = torch.zeros(cap, dtype=torch.float64, device=local.device)
    buf[:local.numel()] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([parts[r][:particle_slice(P, world, r)[1] - particle_slice(P, world, r)[0]]
                      for r in range(world)])


def split_swarm(fitness_fn, step_fn, P, generations, group=None):
    """Run `generations` of Algorithm 1 steps 4-8 with the particles split
    across the group.  fitness_fn(lo, hi) returns the fitness (float64, 1-D)
    of particles lo..hi-1 at their current positions; step_fn(f) takes the
    fitness of all P particles and advances the swarm.  Returns the last
    generation's full fitness vector."""
    import torch.distributed as dist
    if group is None and not (dist.is_available() and dist.is_initialized()):
        world, rank = 1, 0
    else:
        world, rank = dist.get_world_size(group), dist.get_rank(group)
    lo, hi = particle_slice(P, world, rank)
    f_all = None
    for _ in range(generations):
        f_local = fitness_fn(lo, hi)
        f_all = f_local if world == 1 else allgather_fitness(f_local, P, group)
        step_fn(f_all)
    return f_all


def pifcm3d_split(vol, params, options, nx=None, group=None):
    """Algorithm 1 with the swarm split across the ranks of `group` (or the
    default group; one rank without torch.distributed).  Every rank
    normalises the same volume, computes the same FCM start (the plain kernel,
    as pifcm3d does) and, after the swarm, runs the final IFCM at the best
    personal best.  With one rank the result equals pifcm3d's.  Returns
    (U, result dict); `updates` counts this rank's share."""
    if options.fitness != "restart":
        raise ValueError("the split swarm evaluates restart fitnesses (reading R5)")
    x = G.ifcm_normalize(vol, nx=nx)
    if options.slice_z >= 0:
        x = x[options.slice_z:options.slice_z + 1].contiguous()
    nvox = int(x.shape[0]) * int(x.shape[1]) * int(nx if nx is not None else x.shape[2])
    start = G.Params(c=params.c, m=params.m, max_iter=options.init_max_iter,
                     eps_u=params.eps_u, dist_floor=params.dist_floor, V=params.V,
                     h=params.h)
    U0, C0, _, it0 = G.ifcm_fit(x, start, (0.0, 0.0), nx=nx, plain=True)
    sw = G.Swarm(options.P, seed=options.seed, vmax=options.vmax, radius=options.radius,
                 device=x.device).init()
    updates = [it0 * nvox]

    def fitness_fn(lo, hi):
        if hi <= lo:
            return torch.empty(0, dtype=torch.float64, device=x.device)
        fit, its, _ = G.pso_fitness_batch(x, params, sw.x[lo:hi].contiguous(), U0, C0, nx=nx)
        updates.append(int(its.sum()) * nvox)
        return fit

    split_swarm(fitness_fn, sw.step, options.P, options.generations, group)
    best = int(torch.argmin(sw.pbest_f))
    lam_xi = sw.pbest_x[best].contiguous()
    U, Cc, J, it = G.ifcm_fit(x, params, lam_xi, nx=nx, u_init=U0, c_init=C0)
    updates.append(it * nvox)
    lx = lam_xi.cpu().numpy()
    return U, {"lambda": float(lx[0]), "xi": float(lx[1]), "J": float(J),
               "centres": Cc.cpu().numpy(), "iters_final": int(it), "iters_init": int(it0),
               "best_fitness": float(sw.pbest_f.min()), "best_particle": best,
               "updates": int(sum(updates))}

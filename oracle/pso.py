"""FP64 reference of the particle swarm over (lambda, xi) and of Algorithm 1.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Algorithm 1 steps 3-9: a swarm of P particles in D = 2 dimensions
(lambda, xi in [0, 1], Alg 2 step 3); fitness = J_m of an IFCM run (step 4);
personal best (step 5); best over the topological neighbours (step 6);
v <- v + p1 (x_pbest - x) + p2 (x_lbest - x) with p1, p2 ~ U[0, 1) (step 7);
x <- x + v (step 8).

Readings (R9; the paper fixes none of these): the topological neighbours of
particle i are the ring {i - r, ..., i + r} (wrapping, r = 1 by default) and
ties in the ring go to the lowest particle index; pbest is replaced only on a
strict improvement; initial x ~ U[0,1)^2, v ~ U[-vmax, vmax)^2 with
vmax = 0.2; after step 7 each velocity component is clamped to
[-vmax, vmax] and after step 8 each position is clipped to [0, 1]; p1 and p2
are drawn per particle, per dimension and per generation from Philox4x32-10
(``oracle.philox``); the loop runs a fixed number of generations in place of
"small changes to J" (step 9).  Each arithmetic operation below is one
rounded FP64 operation, in the order written, with no fused multiply-add.
"""
import numpy as np

from . import ifcm
from .philox import (STREAM_INIT_V, STREAM_INIT_X, STREAM_P1, STREAM_P2,
                     swarm_uniform)

D = 2  # (lambda, xi)


class Swarm:
    """Swarm state: positions, velocities, personal bests, generation."""

    def __init__(self, P, seed, vmax=0.2, radius=1):
        self.P = int(P)
        self.seed = int(seed)
        self.vmax = float(vmax)
        self.radius = int(radius)
        self.gen = 0
        i = np.arange(self.P)[:, None]
        d = np.arange(D)[None, :]
        # Alg 1 step 3: random swarm
        self.x = swarm_uniform(seed, 0, i, d, STREAM_INIT_X)
        u = swarm_uniform(seed, 0, i, d, STREAM_INIT_V)
        self.v = self.vmax * (2.0 * u - 1.0)
        self.pbest_x = self.x.copy()
        self.pbest_f = np.full(self.P, np.inf)

    def copy(self):
        s = Swarm.__new__(Swarm)
        s.__dict__ = {k: (v.copy() if isinstance(v, np.ndarray) else v)
                      for k, v in self.__dict__.items()}
        return s


def lbest_index(pbest_f, radius=1):
    """Index of the best personal best in each particle's ring (step 6)."""
    P = len(pbest_f)
    out = np.empty(P, dtype=np.int64)
    for i in range(P):
        members = sorted({(i + o) % P for o in range(-radius, radius + 1)})
        best = members[0]
        for k in members[1:]:
            if pbest_f[k] < pbest_f[best]:
                best = k
        out[i] = best
    return out


def pso_step(s, fitness):
    """Algorithm 1 steps 5-8 for one generation, given f(x_i(t)) (step 4)."""
    f = np.asarray(fitness, dtype=np.float64)
    better = f < s.pbest_f                              # step 5 (strict)
    s.pbest_f = np.where(better, f, s.pbest_f)
    s.pbest_x = np.where(better[:, None], s.x, s.pbest_x)
    lb = lbest_index(s.pbest_f, s.radius)               # step 6
    lbest_x = s.pbest_x[lb]
    i = np.arange(s.P)[:, None]
    d = np.arange(D)[None, :]
    p1 = swarm_uniform(s.seed, s.gen, i, d, STREAM_P1)
    p2 = swarm_uniform(s.seed, s.gen, i, d, STREAM_P2)
    a = p1 * (s.pbest_x - s.x)                          # step 7
    b = p2 * (lbest_x - s.x)
    v = (s.v + a) + b
    s.v = np.minimum(np.maximum(v, -s.vmax), s.vmax)
    s.x = np.minimum(np.maximum(s.x + s.v, 0.0), 1.0)   # step 8
    s.gen += 1
    return s


def best_particle(s):
    """Particle with the lowest personal best (ties to the lowest index)."""
    return int(np.argmin(s.pbest_f))


def fitness_batch(x, U0, C0, lam_xi, m=2.0, max_iter=50, eps=1e-5, V=1, h=1.0,
                  dist_floor=1e-12):
    """Step 4 for every particle: J of an IFCM run from (U0, C0) (R5)."""
    out = []
    iters = []
    for lam, xi in np.asarray(lam_xi, dtype=np.float64):
        _, _, J, it = ifcm.ifcm_fit(x, U0, C0, lam, xi, m, max_iter, eps, V, h,
                                    dist_floor)
        out.append(J)
        iters.append(it)
    return np.array(out), np.array(iters)


def fitness_onestep(x, states, lam_xi, m=2.0, V=1, h=1.0, dist_floor=1e-12):
    """Step 4 in the paper's one-step reading of Algorithm 2 (steps 6-11):
    each particle carries its own (U, C) from generation to generation and
    advances it by one IFCM iteration at its current (lambda, xi); the
    fitness is that iteration's J.  ``states`` is a list of (U, C), updated
    in place."""
    out = []
    for p, (lam, xi) in enumerate(np.asarray(lam_xi, dtype=np.float64)):
        U, C = states[p]
        U, C, J, _ = ifcm.ifcm_iteration(x, U, C, lam, xi, m, V, h, dist_floor)
        states[p] = (U, C)
        out.append(J)
    return np.array(out)


def pifcm3d(vol, c, P, generations, seed, m=2.0, max_iter=50, eps=1e-5,
            init_max_iter=300, vmax=0.2, radius=1, V=1, h=1.0, z=None,
            dist_floor=1e-12, fitness="restart"):
    """Algorithm 1 end to end: normalise (Alg 2 step 1), optional slice z
    (Alg 1 step 1), FCM start (step 2), swarm (steps 3-9), final IFCM at the
    best particle (step 11).  ``fitness`` is "restart" (reading R5: an IFCM
    run from (U0, C0) per evaluation) or "onestep" (``fitness_onestep``).
    Returns a dict with U, C, lambda, xi, J."""
    x = ifcm.normalize(vol)
    if z is not None:
        x = x[z:z + 1]
    U0, C0, _, init_iters = ifcm.fcm_init(x, c, m, init_max_iter, eps, dist_floor)
    s = Swarm(P, seed, vmax, radius)
    states = [(U0, C0)] * P
    for _ in range(generations):
        if fitness == "onestep":
            f = fitness_onestep(x, states, s.x, m, V, h, dist_floor)
        else:
            f, _ = fitness_batch(x, U0, C0, s.x, m, max_iter, eps, V, h, dist_floor)
        pso_step(s, f)
    b = best_particle(s)
    lam, xi = s.pbest_x[b]
    U, C, J, it = ifcm.ifcm_fit(x, U0, C0, lam, xi, m, max_iter, eps, V, h,
                                dist_floor)
    return {"U": U, "C": C, "lambda": lam, "xi": xi, "J": J, "iters": it,
            "pbest_f": s.pbest_f.copy(), "init_iters": init_iters, "swarm": s}

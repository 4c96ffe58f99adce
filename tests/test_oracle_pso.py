"""Pins for the oracle's particle swarm (Algorithm 1 steps 3-9) and driver."""
import numpy as np
import pytest

from oracle import pso
from paper_2002_01981_gb300 import phantoms


def _bowl(xy, target=(0.3, 0.7)):
    return (xy[:, 0] - target[0]) ** 2 + (xy[:, 1] - target[1]) ** 2


def test_swarm_reaches_bowl_minimum():
    s = pso.Swarm(16, seed=11)
    f0 = _bowl(s.x).min()
    for _ in range(80):
        pso.pso_step(s, _bowl(s.x))
    b = pso.best_particle(s)
    # no inertia weight (Alg 1 step 7): the swarm stalls near, not at, the minimum
    assert np.allclose(s.pbest_x[b], [0.3, 0.7], atol=1e-2)
    assert s.pbest_f[b] < 1e-4 and s.pbest_f[b] < f0 / 10


def test_minimum_on_the_box_edge_is_reached():
    # the target lies outside [0,1]^2: the clipped swarm must sit on the edge
    s = pso.Swarm(12, seed=3)
    for _ in range(60):
        pso.pso_step(s, _bowl(s.x, (1.4, -0.2)))
    b = pso.best_particle(s)
    assert np.allclose(s.pbest_x[b], [1.0, 0.0], atol=1e-6)


def test_positions_and_velocities_stay_bounded():
    s = pso.Swarm(9, seed=5, vmax=0.15)
    rng = np.random.default_rng(0)
    assert np.all(np.abs(s.v) <= 0.15) and np.all((s.x >= 0) & (s.x < 1))
    for _ in range(30):
        pso.pso_step(s, rng.random(9))
        assert np.all(np.abs(s.v) <= 0.15)
        assert np.all((s.x >= 0) & (s.x <= 1))


def test_lbest_ring_by_hand():
    f = np.array([5.0, 1.0, 7.0, 7.0, 0.5, 9.0])
    # rings (radius 1, wrapping): {5,0,1},{0,1,2},{1,2,3},{2,3,4},{3,4,5},{4,5,0}
    assert list(pso.lbest_index(f)) == [1, 1, 1, 4, 4, 4]
    g = np.array([2.0, 2.0, 2.0, 2.0])          # ties go to the lowest index
    assert list(pso.lbest_index(g)) == [0, 0, 1, 0]
    assert list(pso.lbest_index(np.array([3.0]))) == [0]
    assert list(pso.lbest_index(f, radius=2)) == [4, 1, 4, 4, 4, 4]


def test_pbest_needs_strict_improvement():
    s = pso.Swarm(3, seed=2)
    pso.pso_step(s, np.array([1.0, 2.0, 3.0]))
    keep = s.pbest_x.copy()
    pso.pso_step(s, np.array([1.0, 2.0, 3.0]))    # equal fitness: no update
    assert np.array_equal(s.pbest_x, keep)
    x_now = s.x.copy()
    pso.pso_step(s, np.array([0.5, 2.0, np.nan]))  # strict improvement / NaN
    assert np.array_equal(s.pbest_x[0], x_now[0])
    assert np.array_equal(s.pbest_x[2], keep[2]) and s.pbest_f[2] == 3.0


def test_zero_attraction_keeps_velocity():
    # with x = pbest = lbest the update is v <- v (clamped), x <- x + v
    s = pso.Swarm(4, seed=9)
    s.pbest_f = np.full(4, -np.inf)      # nothing can improve
    s.pbest_x = s.x.copy()
    s.pbest_x[:] = s.x
    s.pbest_x = np.tile(s.x[:1], (4, 1))
    s.x = s.pbest_x.copy()
    v0, x0 = s.v.copy(), s.x.copy()
    pso.pso_step(s, np.zeros(4))
    assert np.array_equal(s.v, v0)
    assert np.array_equal(s.x, np.clip(x0 + v0, 0, 1))


def test_resume_is_bit_identical():
    rng = np.random.default_rng(1)
    fits = [rng.random(7) for _ in range(10)]
    a = pso.Swarm(7, seed=42)
    for f in fits:
        pso.pso_step(a, f)
    b = pso.Swarm(7, seed=42)
    for f in fits[:4]:
        pso.pso_step(b, f)
    saved = b.copy()
    for f in fits[4:]:
        pso.pso_step(saved, f)
    assert np.array_equal(a.x, saved.x) and np.array_equal(a.v, saved.v)
    assert np.array_equal(a.pbest_f, saved.pbest_f) and a.gen == saved.gen == 10


@pytest.mark.slow
def test_pifcm3d_small_end_to_end():
    vol = phantoms.ellipse_slice(16, seed=1, sigma=0.05)
    out = pso.pifcm3d(vol, c=4, P=4, generations=3, seed=1, max_iter=10)
    U, C = out["U"], out["C"]
    assert np.allclose(U.sum(axis=0), 1.0, atol=1e-13)
    assert np.all(np.diff(np.sort(C)) > 0.1)          # four distinct grey levels
    assert 0 <= out["lambda"] <= 1 and 0 <= out["xi"] <= 1
    assert out["J"] <= out["pbest_f"].min() * (1 + 1e-12) + 1e-15



def test_onestep_fitness_carries_each_particle_state():
    # with positions held fixed, generation g of the one-step reading is
    # iteration g of an IFCM run from the shared start
    from oracle import ifcm
    rng = np.random.default_rng(21)
    x = np.clip(np.repeat([0.1, 0.5, 0.9], 24).reshape(3, 4, 6) +
                0.04 * rng.standard_normal((3, 4, 6)), 0, 1)
    U0, C0, _, _ = ifcm.fcm_init(x, 3, max_iter=20)
    lam_xi = np.array([[0.3, 0.2], [0.6, 0.1]])
    states = [(U0, C0)] * 2
    for g in range(4):
        f = pso.fitness_onestep(x, states, lam_xi)
        for p in range(2):
            J = ifcm.ifcm_fit(x, U0, C0, lam_xi[p, 0], lam_xi[p, 1], 2.0, g + 1, 0.0)[2]
            assert f[p] == J


def test_one_step_computed_by_hand(monkeypatch):
    # Alg 1 steps 5-8 on three particles with given draws p1, p2 (stream 2 and
    # 3 of the generator), every value worked out by hand:
    # step 5: particle 1 improves (0.5 < 1.0) and takes its position as pbest;
    #         particles 0 (4.0 > 3.0) and 2 (2.5 > 2.0) keep theirs;
    # step 6: every ring of three holds all three, so lbest = particle 1,
    #         lbest_x = (0.60, 0.40);
    # step 7: v <- v + p1 (pbest_x - x) + p2 (lbest_x - x), clamped to +-0.2;
    # step 8: x <- clip(x + v, 0, 1).
    p1 = np.array([[0.25, 0.5], [0.75, 0.125], [0.5, 0.375]])
    p2 = np.array([[0.5, 0.25], [0.375, 0.625], [0.125, 0.75]])

    def draws(seed, gen, i, d, stream):
        assert stream in (pso.STREAM_P1, pso.STREAM_P2)
        return np.broadcast_to(p1 if stream == pso.STREAM_P1 else p2, (3, 2)).copy()

    s = pso.Swarm(3, seed=1)
    s.x = np.array([[0.50, 0.50], [0.60, 0.40], [0.90, 0.10]])
    s.v = np.array([[0.01, -0.02], [0.05, 0.0], [-0.03, 0.04]])
    s.pbest_x = np.array([[0.55, 0.45], [0.70, 0.30], [0.85, 0.20]])
    s.pbest_f = np.array([3.0, 1.0, 2.0])
    monkeypatch.setattr(pso, "swarm_uniform", draws)
    pso.pso_step(s, np.array([4.0, 0.5, 2.5]))
    # particle 0: pbest - x = (0.05, -0.05), lbest - x = (0.10, -0.10)
    #   v = (0.01 + 0.25*0.05 + 0.5*0.10, -0.02 + 0.5*(-0.05) + 0.25*(-0.10))
    #     = (0.0725, -0.07); x = (0.5725, 0.43)
    # particle 1: both differences are 0: v = (0.05, 0.0); x = (0.65, 0.40)
    # particle 2: pbest - x = (-0.05, 0.10), lbest - x = (-0.30, 0.30)
    #   v = (-0.03 - 0.025 - 0.0375, 0.04 + 0.0375 + 0.225) = (-0.0925, 0.3025)
    #   -> clamped (-0.0925, 0.2); x = (0.8075, 0.30)
    v_hand = np.array([[0.0725, -0.07], [0.05, 0.0], [-0.0925, 0.2]])
    x_hand = np.array([[0.5725, 0.43], [0.65, 0.40], [0.8075, 0.30]])
    assert np.allclose(s.v, v_hand, rtol=0, atol=1e-15)
    assert np.allclose(s.x, x_hand, rtol=0, atol=1e-15)
    assert np.array_equal(s.pbest_f, [3.0, 0.5, 2.0])
    assert np.allclose(s.pbest_x, [[0.55, 0.45], [0.60, 0.40], [0.85, 0.20]], rtol=0, atol=0)
    assert s.gen == 1

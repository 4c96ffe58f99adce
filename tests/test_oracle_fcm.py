"""Pins for the oracle's membership (Eq 2), objective (Eq 1), centres (Eq 3),
normalisation (Alg 2 step 1) and the iteration loop."""
import itertools
import math

import numpy as np
import pytest

from oracle import ifcm
from paper_2002_01981_gb300 import phantoms


# ------------------------------------------------------- Alg 2 step 1
def test_normalize_maps_min_max_to_0_1_affinely():
    rng = np.random.default_rng(0)
    v = (rng.random((3, 4, 5)) * 7 - 2).astype(np.float32)
    x = ifcm.normalize(v)
    assert x.min() == 0.0 and x.max() == 1.0
    i, j = np.unravel_index(np.argmin(v), v.shape), np.unravel_index(np.argmax(v), v.shape)
    assert x[i] == 0.0 and x[j] == 1.0
    # affine: equal differences stay equal
    a = v.astype(np.float64).ravel()
    assert np.allclose(np.diff(x.ravel()) * (a.max() - a.min()), np.diff(a), atol=1e-12)


@pytest.mark.parametrize("bad", [np.full((2, 2, 2), 3.0), np.array([[[1.0, np.nan]]]),
                                 np.array([[[1.0, np.inf]]])])
def test_normalize_rejects_degenerate(bad):
    with pytest.raises(ValueError):
        ifcm.normalize(bad)


# --------------------------------------------------------------- Eq 2
def test_membership_two_clusters_closed_form():
    d2 = np.array([0.2, 0.05]).reshape(2, 1)
    u = ifcm.membership(d2, 2.0)
    # m = 2, c = 2: u_1 = d2_2 / (d2_1 + d2_2)
    assert abs(u[0, 0] - 0.05 / 0.25) < 1e-15 and abs(u[1, 0] - 0.2 / 0.25) < 1e-15
    u3 = ifcm.membership(d2, 3.0)
    # m = 3: u_1 = 1 / (1 + (d_1 / d_2)) with d = sqrt(d2)
    r = math.sqrt(0.2) / math.sqrt(0.05)
    assert abs(u3[0, 0] - 1 / (1 + r)) < 1e-15


def test_membership_sums_to_one():
    rng = np.random.default_rng(1)
    d2 = rng.random((6, 1000)) + 1e-12
    for m in (1.3, 2.0, 2.5, 4.0):
        u = ifcm.membership(d2, m)
        assert np.allclose(u.sum(axis=0), 1.0, atol=1e-14)
        assert np.all(u > 0)


def test_membership_orders_by_distance():
    rng = np.random.default_rng(2)
    d2 = rng.random((5, 200)) + 1e-6
    u = ifcm.membership(d2, 2.0)
    assert np.array_equal(np.argmax(u, 0), np.argmin(d2, 0))


# --------------------------------------------------------------- Eq 3
def test_centres_of_crisp_memberships_are_class_means():
    rng = np.random.default_rng(3)
    x = rng.random((2, 3, 4))
    lab = rng.integers(0, 3, x.shape)
    U = np.stack([(lab == j).astype(float) for j in range(3)])
    C = ifcm.centres(x, U, 2.0)
    for j in range(3):
        assert abs(C[j] - x[lab == j].mean()) < 1e-15


# ------------------------------------------------------- P1: textbook FCM
def _textbook_fcm(xs, c, m, max_iter, eps):
    """Classic FCM (Bezdek) on a flat list of intensities, pure Python:
    centres first, memberships from unsquared distances with exponent
    2/(m-1), a singularity guard of 1e-6 on the distance."""
    n = len(xs)
    cs = [(j + 0.5) / c for j in range(c)]
    u = [[1.0 / c] * n for _ in range(c)]
    J = None
    it = 0
    for it in range(1, max_iter + 1):
        dist = [[max(abs(xs[i] - cs[j]), 1e-6) for i in range(n)] for j in range(c)]
        new = [[0.0] * n for _ in range(c)]
        for i in range(n):
            for j in range(c):
                s = 0.0
                for k in range(c):
                    s += (dist[j][i] / dist[k][i]) ** (2.0 / (m - 1.0))
                new[j][i] = 1.0 / s
        J = sum(new[j][i] ** m * dist[j][i] ** 2 for j in range(c) for i in range(n))
        delta = max(abs(new[j][i] - u[j][i]) for j in range(c) for i in range(n))
        u = new
        cs = [sum(u[j][i] ** m * xs[i] for i in range(n)) / sum(u[j][i] ** m for i in range(n))
              for j in range(c)]
        if delta < eps:
            break
    return u, cs, J, it


@pytest.mark.parametrize("m", [1.5, 2.0, 3.0])
def test_lambda_xi_zero_is_textbook_fcm(m):
    rng = np.random.default_rng(4)
    x = rng.random((2, 5, 6))
    c = 3
    U, C, J, it = ifcm.fcm_init(x, c, m, max_iter=300, eps=1e-9)
    u_t, c_t, J_t, it_t = _textbook_fcm(list(x.ravel()), c, m, 300, 1e-9)
    assert it == it_t
    assert np.allclose(U.reshape(c, -1), np.array(u_t), atol=1e-12)
    assert np.allclose(C, c_t, rtol=1e-12)
    assert abs(J - J_t) < 1e-12 * abs(J_t)
    # the same through ifcm_fit with lambda = xi = 0 from a given start
    U2, C2, J2, it2 = ifcm.ifcm_fit(x, np.full((c,) + x.shape, 1 / c), (np.arange(c) + 0.5) / c,
                                    0.0, 0.0, m, 300, 1e-9)
    assert it2 == it and np.array_equal(U2, U)


# ----------------------------------------------------- P4: J non-increasing
def test_fcm_objective_is_non_increasing():
    vol = phantoms.ellipse_slice(32, seed=5, sigma=0.08)
    x = ifcm.normalize(vol)
    U = np.full((4,) + x.shape, 0.25)
    C = (np.arange(4) + 0.5) / 4
    _, _, _, _, hist = ifcm.ifcm_fit(x, U, C, 0.0, 0.0, 2.0, 60, 0.0, history=True)
    Js = [h[0] for h in hist]
    assert all(b <= a * (1 + 1e-13) for a, b in zip(Js, Js[1:]))
    assert Js[-1] < Js[0]


# ------------------------------------- P5: fixed point and brute force
def test_noise_free_classes_reach_exact_means():
    vol = phantoms.piecewise_cube(4, levels=(0.1, 0.5, 0.9))
    x = ifcm.normalize(vol)
    U, C, J, it = ifcm.fcm_init(x, 3, 2.0, max_iter=500, eps=1e-14)
    levels = np.unique(x)
    assert np.allclose(np.sort(C), levels, atol=1e-9)
    assert np.all(U.max(axis=0) > 1 - 1e-9)


def _brute_force_partition(values, c):
    """Optimal hard partition of 1-D values into c contiguous intervals of the
    sorted order (minimum within-class sum of squares), by enumeration."""
    order = np.argsort(values, kind="stable")
    v = values[order]
    n = len(v)
    best, best_cuts = np.inf, None
    for cuts in itertools.combinations(range(1, n), c - 1):
        bounds = (0,) + cuts + (n,)
        sse = sum(np.sum((v[a:b] - v[a:b].mean()) ** 2) for a, b in zip(bounds, bounds[1:]))
        if sse < best:
            best, best_cuts = sse, bounds
    lab = np.empty(n, dtype=int)
    for j, (a, b) in enumerate(zip(best_cuts, best_cuts[1:])):
        lab[order[a:b]] = j
    return lab


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_noisy_separated_classes_match_brute_force(seed):
    vol = phantoms.piecewise_cube(4, levels=(0.1, 0.5, 0.9), seed=seed, sigma=0.03)
    x = ifcm.normalize(vol)
    U, C, J, it = ifcm.fcm_init(x, 3, 2.0, max_iter=300, eps=1e-10)
    lab = ifcm.labels(U).ravel()
    # relabel clusters by ascending centre to compare with interval order
    rank = np.argsort(np.argsort(C))
    lab = rank[lab]
    assert np.array_equal(lab, _brute_force_partition(x.ravel(), 3))


# --------------------------------------------------- iteration bookkeeping
def test_stop_rule_and_iteration_count():
    rng = np.random.default_rng(6)
    x = rng.random((1, 8, 8))
    U0 = np.full((2, 1, 8, 8), 0.5)
    C0 = np.array([0.25, 0.75])
    _, _, _, it, hist = ifcm.ifcm_fit(x, U0, C0, 0.3, 0.2, 2.0, 50, 1e-5, history=True)
    deltas = [h[1] for h in hist]
    assert len(hist) == it
    assert all(d >= 1e-5 for d in deltas[:-1])
    assert deltas[-1] < 1e-5 or it == 50
    _, _, _, it3 = ifcm.ifcm_fit(x, U0, C0, 0.3, 0.2, 2.0, 3, 0.0)
    assert it3 == 3


def test_ifcm_memberships_sum_to_one():
    vol = phantoms.ellipse_slice(16, seed=3)
    x = ifcm.normalize(vol)
    U0, C0, _, _ = ifcm.fcm_init(x, 4)
    U, C, J, it = ifcm.ifcm_fit(x, U0, C0, 0.6, 0.4, 2.0, 10, 1e-5)
    assert np.allclose(U.sum(axis=0), 1.0, atol=1e-14)
    assert np.all((C > 0) & (C < 1))

"""Pins of the FP64 adjoint (oracle/adjoint.py): dJ^{K-1}/d(lambda, xi)
through K unrolled IFCM iterations.

- K = 1: J^0 = sum_ij u_ij^m d2_ij with u minimising J over the simplex for
  fixed d2 (Eq 2 is that minimiser), so by the envelope theorem
  dJ/dlambda = sum_ij u^m d(d2)/dlambda = -sum u^m D H over the voxels where
  neither clamp of reading R2 is active (likewise xi with F).  The adjoint
  chain must reproduce this, with no contribution from the U feedback.
- Any K: FP64 central differences of the oracle's forward J, h = 1e-6
  (truncation ~h^2, rounding ~1e-16 J / h: both far below the 1e-6 bar).
- Reading R8: for fixed U the derivatives are <= 0.
"""
import numpy as np
import pytest

from oracle import adjoint as A
from oracle import ifcm as O
from paper_2002_01981_gb300 import phantoms


def unit_volume(shape, seed, sigma=0.06):
    return np.clip(phantoms.brain_phantom(shape, seed=seed, sigma=sigma), 0.0, 1.0).astype(
        np.float64)


def fd(x, U0, C0, lam, xi, m, K, h=1e-6):
    f = lambda a, b: O.ifcm_fit(x, U0, C0, a, b, m, K, 0.0)[2]   # noqa: E731
    return ((f(lam + h, xi) - f(lam - h, xi)) / (2 * h),
            (f(lam, xi + h) - f(lam, xi - h)) / (2 * h))


@pytest.mark.parametrize("m", [2.0, 3.0, 1.5])
def test_envelope_closed_form_at_one_iteration(m):
    x = unit_volume((4, 6, 7), seed=5)
    c = 3
    U0 = phantoms.random_memberships(x.shape, c, seed=6).astype(np.float64)
    C0 = np.array([0.15, 0.5, 0.85])
    lam, xi = 0.35, 0.3
    J, gl, gx = A.ifcm_grad(x, U0, C0, lam, xi, m, K=1)
    H, F = O.neighbour_terms(x, U0)
    D = (x[None] - C0[:, None, None, None]) ** 2
    f = 1.0 - lam * H - xi * F
    d2 = O.modified_distance(x, C0, H, F, lam, xi)
    u = O.membership(d2, m)
    live = (f > 0) & (D * np.maximum(f, 0) > 1e-12)
    assert abs(J - O.objective(u, d2, m)) <= 1e-14 * J
    assert gl == pytest.approx(float(np.sum(np.where(live, -u ** m * D * H, 0.0))), rel=1e-12)
    assert gx == pytest.approx(float(np.sum(np.where(live, -u ** m * D * F, 0.0))), rel=1e-12)
    assert gl <= 0.0 and gx <= 0.0                       # reading R8


CASES = [
    # shape, c, m, lambda, xi, K
    ((4, 6, 7), 3, 2.0, 0.3, 0.25, 3),
    ((4, 6, 7), 3, 2.0, 0.3, 0.25, 8),
    ((5, 5, 6), 4, 1.5, 0.2, 0.4, 4),
    ((3, 7, 5), 5, 3.0, 0.4, 0.1, 3),
    ((1, 9, 11), 4, 2.0, 0.5, 0.3, 5),        # 2D
    ((6, 5, 4), 2, 2.0, 0.0, 0.0, 4),         # at plain FCM
    ((1, 1, 6), 3, 2.0, 0.4, 0.4, 3),         # a line
    ((4, 6, 7), 3, 2.0, 0.9, 0.8, 2),         # clamp regime (factor <= 0 at some voxels)
]


@pytest.mark.parametrize("shape,c,m,lam,xi,K", CASES)
def test_matches_central_differences(shape, c, m, lam, xi, K):
    x = unit_volume(shape, seed=7)
    U0 = phantoms.random_memberships(shape, c, seed=8).astype(np.float64)
    C0 = np.linspace(0.1, 0.9, c)
    J, gl, gx = A.ifcm_grad(x, U0, C0, lam, xi, m, K)
    assert J == pytest.approx(O.ifcm_fit(x, U0, C0, lam, xi, m, K, 0.0)[2], rel=1e-14)
    fl, fx = fd(x, U0, C0, lam, xi, m, K)
    assert gl == pytest.approx(fl, rel=1e-6, abs=1e-9)
    assert gx == pytest.approx(fx, rel=1e-6, abs=1e-9)


def test_flat_neighbourhoods_match_central_differences():
    # constant slabs along z (three levels, two clusters, so d^2 stays away
    # from the floor) with noise on the columns x >= 4: the middle plane of a
    # slab at x <= 2 sees 26 equal neighbours, so sum_k g_ik = 0 there and H
    # is the plain neighbour mean (reading R3)
    lv = np.array([0.2, 0.2, 0.2, 0.55, 0.55, 0.55, 0.9, 0.9])
    x = np.repeat(lv[:, None, None], 6 * 7, axis=1).reshape(8, 6, 7)
    x[:, :, 4:] += 0.05 * np.random.default_rng(14).standard_normal((8, 6, 3))
    x = np.clip(x, 0.0, 1.0)
    U0 = phantoms.random_memberships(x.shape, 2, seed=9).astype(np.float64)
    C0 = np.array([0.3, 0.7])
    _, _, aux = O.neighbour_terms(x, U0, return_aux=True)
    assert np.sum(aux["G"][0] == 0.0) >= 40
    J, gl, gx = A.ifcm_grad(x, U0, C0, 0.4, 0.3, 2.0, K=3)
    fl, fx = fd(x, U0, C0, 0.4, 0.3, 2.0, 3)
    assert gl == pytest.approx(fl, rel=1e-6, abs=1e-9)
    assert gx == pytest.approx(fx, rel=1e-6, abs=1e-9)


def test_gradient_of_a_longer_run_from_the_fcm_start():
    # the shape of the differentiation workload: FCM start, then K = 12
    x = unit_volume((6, 8, 9), seed=10, sigma=0.09)
    U0, C0, _, _ = O.fcm_init(x, 4, max_iter=60)
    J, gl, gx = A.ifcm_grad(x, U0, C0, 0.3, 0.2, 2.0, K=12)
    fl, fx = fd(x, U0, C0, 0.3, 0.2, 2.0, 12)
    assert gl == pytest.approx(fl, rel=1e-6, abs=1e-9)
    assert gx == pytest.approx(fx, rel=1e-6, abs=1e-9)

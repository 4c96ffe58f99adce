"""Pins for the oracle's neighbourhood terms (Eqs 5-10) and distance (Eq 4)."""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from conftest import read_golden
from oracle import ifcm


def fr(s):
    return float(Fraction(s))


# ---------------------------------------------------------------- Eq 9, Eq 10
def test_neighbourhood_L3_is_the_26_cube():
    nb = ifcm.neighbourhood(3)
    cube = {o for o in itertools.product((-1, 0, 1), repeat=3) if o != (0, 0, 0)}
    assert len(nb) == 26 and set(nb) == cube


def test_neighbourhood_L2_is_the_6_faces():
    # 0 < |d|^2 < 2 keeps only the face neighbours
    assert sorted(ifcm.neighbourhood(2)) == sorted(
        [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)])


def test_shell_weights():
    assert np.allclose(ifcm.shell_weights(1, 0.7), [1.0])
    W = ifcm.shell_weights(3, 2.0)
    assert abs(W.sum() - 1.0) < 1e-15
    assert np.allclose(W[1:] / W[:-1], np.exp(-1 / 2.0))   # exponential decay


# ------------------------------------------------------ hand-worked fixtures
def _mixed_fixture():
    g = read_golden("hand_3x3x3_mixed.txt")
    x = np.empty((3, 3, 3))
    U = np.zeros((3, 3, 3, 3))
    for z, y, xx in itertools.product(range(3), repeat=3):
        nnz = (z != 1) + (y != 1) + (xx != 1)
        kind = {0: "centre", 1: "face", 2: "edge", 3: "corner"}[nnz]
        x[z, y, xx] = fr(g[f"x_{kind}"][0])
        if kind == "centre":
            U[:, z, y, xx] = 1.0 / 3.0
        else:
            U[int(g[f"cluster_{kind}"][0]), z, y, xx] = 1.0
    return g, x, U


def test_hand_fixture_H_F_G_Q():
    g, x, U = _mixed_fixture()
    H, F, aux = ifcm.neighbour_terms(x, U, return_aux=True)
    assert aux["G"][0][1, 1, 1] == fr(g["G"][0])
    assert aux["Q"][0][1, 1, 1] == fr(g["Q"][0])
    assert np.allclose(H[:, 1, 1, 1], [fr(v) for v in g["H"]], rtol=0, atol=1e-15)
    assert np.allclose(F[:, 1, 1, 1], [fr(v) for v in g["F"]], rtol=0, atol=1e-15)


def test_hand_fixture_distance_membership_objective():
    g, x, U = _mixed_fixture()
    C = np.array([fr(v) for v in g["C"]])
    lam, xi = fr(g["lambda"][0]), fr(g["xi"][0])
    H, F = ifcm.neighbour_terms(x, U)
    d2 = ifcm.modified_distance(x, C, H, F, lam, xi)
    assert np.allclose(d2[:, 1, 1, 1], [fr(v) for v in g["d2"]], rtol=1e-14, atol=0)
    u = ifcm.membership(d2, 2.0)
    assert np.allclose(u[:, 1, 1, 1], [fr(v) for v in g["u"]], rtol=1e-14, atol=0)
    share = np.sum(u[:, 1, 1, 1] ** 2 * d2[:, 1, 1, 1])
    assert abs(share - fr(g["J_centre"][0])) < 1e-15


def test_boundary_counts_and_Q():
    rows = read_golden("hand_boundary.txt")["_rows"]
    for row in rows:
        _, nz, ny, nx, z, y, xx, count, Q = row
        shape = (int(nz), int(ny), int(nx))
        x = np.random.default_rng(0).random(shape)
        U = np.full((2,) + shape, 0.5)
        _, _, aux = ifcm.neighbour_terms(x, U, return_aux=True)
        assert aux["count"][0][int(z), int(y), int(xx)] == int(count), row
        assert aux["Q"][0][int(z), int(y), int(xx)] == int(Q), row


# ------------------------------------------------------------- invariants
def _random_case(shape, c, seed):
    rng = np.random.default_rng(seed)
    x = rng.random(shape)
    U = rng.random((c,) + shape)
    U /= U.sum(axis=0, keepdims=True)
    return x, U


@pytest.mark.parametrize("shape", [(5, 6, 7), (1, 9, 8), (2, 3, 4), (1, 1, 5)])
def test_H_sums_to_one_and_ranges(shape):
    x, U = _random_case(shape, 4, 1)
    H, F = ifcm.neighbour_terms(x, U)
    assert np.allclose(H.sum(axis=0), 1.0, atol=1e-14)
    assert H.min() >= 0 and H.max() <= 1
    assert F.min() >= 0 and F.max() <= 1
    assert np.all(F.sum(axis=0) <= 1 + 1e-14)     # sum_j u^2 <= (sum_j u)^2 = 1


@pytest.mark.parametrize("shape", [(4, 5, 6), (1, 7, 7)])
def test_uniform_memberships(shape):
    c = 5
    x, _ = _random_case(shape, c, 2)
    U = np.full((c,) + shape, 1.0 / c)
    H, F = ifcm.neighbour_terms(x, U)
    assert np.allclose(H, 1.0 / c, atol=1e-15)
    assert np.allclose(F, 1.0 / c ** 2, atol=1e-15)


def test_interior_Q_3d_and_2d():
    x, U = _random_case((5, 5, 5), 2, 3)
    _, _, aux = ifcm.neighbour_terms(x, U, return_aux=True)
    assert np.all(aux["Q"][0][1:-1, 1:-1, 1:-1] == 54)
    x, U = _random_case((1, 5, 5), 2, 3)
    _, _, aux = ifcm.neighbour_terms(x, U, return_aux=True)
    assert np.all(aux["Q"][0][0, 1:-1, 1:-1] == 12)


def test_flat_neighbourhood_uses_plain_mean():
    # every neighbour equals the centre: G = 0, H falls back to the mean of u_kj
    x = np.full((3, 3, 3), 0.25)
    rng = np.random.default_rng(4)
    U = rng.random((3, 3, 3, 3))
    U /= U.sum(axis=0, keepdims=True)
    H, _, aux = ifcm.neighbour_terms(x, U, return_aux=True)
    assert aux["G"][0][1, 1, 1] == 0
    mask = np.ones((3, 3, 3), bool)
    mask[1, 1, 1] = False
    expect = U[:, mask].mean(axis=1)
    assert np.allclose(H[:, 1, 1, 1], expect, atol=1e-15)


def test_single_voxel_has_no_terms():
    H, F = ifcm.neighbour_terms(np.array([[[0.3]]]), np.full((2, 1, 1, 1), 0.5))
    assert np.all(H == 0) and np.all(F == 0)


# --------------------------------------------------- brute-force voxel loops
def _brute_terms(x, U):
    """Per-voxel loops over the 26 offsets with explicit bounds checks."""
    c = U.shape[0]
    nz, ny, nx = x.shape
    H = np.zeros_like(U)
    F = np.zeros_like(U)
    for z, y, xx in itertools.product(range(nz), range(ny), range(nx)):
        G = Q = 0.0
        n = 0
        h = np.zeros(c)
        f = np.zeros(c)
        s = np.zeros(c)
        for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
            if (dz, dy, dx) == (0, 0, 0):
                continue
            kz, ky, kx = z + dz, y + dy, xx + dx
            if not (0 <= kz < nz and 0 <= ky < ny and 0 <= kx < nx):
                continue
            gk = abs(x[z, y, xx] - x[kz, ky, kx])
            qk = dx * dx + dy * dy + dz * dz
            for j in range(c):
                h[j] += U[j, kz, ky, kx] * gk
                f[j] += U[j, kz, ky, kx] ** 2 * qk
                s[j] += U[j, kz, ky, kx]
            G += gk
            Q += qk
            n += 1
        if n:
            H[:, z, y, xx] = h / G if G > 0 else s / n
            F[:, z, y, xx] = f / Q
    return H, F


@pytest.mark.parametrize("shape", [(3, 4, 5), (1, 4, 6), (2, 5, 3)])
def test_matches_brute_force_loops(shape):
    x, U = _random_case(shape, 3, 5)
    H, F = ifcm.neighbour_terms(x, U)
    Hb, Fb = _brute_terms(x, U)
    assert np.allclose(H, Hb, atol=1e-14)
    assert np.allclose(F, Fb, atol=1e-14)


def test_slice_of_3d_is_2d_8_neighbourhood():
    # nz = 1 with the 26-neighbourhood equals the 8-neighbourhood in 2D (R4)
    x, U = _random_case((1, 6, 7), 3, 6)
    H, F = ifcm.neighbour_terms(x, U)
    c, _, ny, nx = U.shape
    for y, xx in itertools.product(range(ny), range(nx)):
        G = Q = 0.0
        h = np.zeros(c)
        f = np.zeros(c)
        for dy, dx in itertools.product((-1, 0, 1), repeat=2):
            if (dy, dx) == (0, 0) or not (0 <= y + dy < ny and 0 <= xx + dx < nx):
                continue
            gk = abs(x[0, y, xx] - x[0, y + dy, xx + dx])
            h += U[:, 0, y + dy, xx + dx] * gk
            f += U[:, 0, y + dy, xx + dx] ** 2 * (dx * dx + dy * dy)
            G += gk
            Q += dx * dx + dy * dy
        assert np.allclose(H[:, 0, y, xx], h / G, atol=1e-14)
        assert np.allclose(F[:, 0, y, xx], f / Q, atol=1e-14)


# ------------------------------------------------------------ equivariance
def test_axis_flips_transpose_and_cluster_permutation():
    x, U = _random_case((4, 5, 5), 3, 7)
    C = np.array([0.2, 0.5, 0.8])
    ref = ifcm.ifcm_iteration(x, U, C, 0.4, 0.3)
    for ax in (0, 1, 2):
        out = ifcm.ifcm_iteration(np.flip(x, ax), np.flip(U, ax + 1), C, 0.4, 0.3)
        assert np.allclose(out[0], np.flip(ref[0], ax + 1), atol=1e-13)
        assert np.allclose(out[1], ref[1], atol=1e-13)
        assert abs(out[2] - ref[2]) < 1e-12
    xt, Ut = np.swapaxes(x, 1, 2), np.swapaxes(U, 2, 3)
    out = ifcm.ifcm_iteration(xt, Ut, C, 0.4, 0.3)
    assert np.allclose(out[0], np.swapaxes(ref[0], 2, 3), atol=1e-13)
    perm = [2, 0, 1]
    out = ifcm.ifcm_iteration(x, U[perm], C[perm], 0.4, 0.3)
    assert np.allclose(out[0], ref[0][perm], atol=1e-13)
    assert np.allclose(out[1], ref[1][perm], atol=1e-13)


# ------------------------------------------------------------------- Eq 4
def test_distance_clamp_and_floor():
    x = np.array([[[0.5, 0.3]]])
    C = np.array([0.5, 0.0])
    H = np.array([[[[0.0, 1.0]]], [[[1.0, 0.0]]]])
    F = np.zeros_like(H)
    d2 = ifcm.modified_distance(x, C, H, F, 1.0, 0.0)
    # voxel 0, cluster 0: x == c -> floor; cluster 1: factor 1 - 1*1 = 0 -> floor
    assert d2[0, 0, 0, 0] == 1e-12 and d2[1, 0, 0, 0] == 1e-12
    # voxel 1, cluster 0: factor 1 - 1 = 0 -> floor; cluster 1: 0.09 * 1
    assert d2[0, 0, 0, 1] == 1e-12 and abs(d2[1, 0, 0, 1] - 0.09) < 1e-16


def test_lambda_xi_signs():
    # larger H (or F) for a cluster lowers its distance: Eq 4 subtracts them
    x = np.array([[[0.4]]])
    C = np.array([0.1, 0.9])
    H = np.array([0.8, 0.2]).reshape(2, 1, 1, 1)
    F = np.array([0.1, 0.6]).reshape(2, 1, 1, 1)
    d0 = ifcm.modified_distance(x, C, H, F, 0.0, 0.0)
    dl = ifcm.modified_distance(x, C, H, F, 0.5, 0.0)
    dx_ = ifcm.modified_distance(x, C, H, F, 0.0, 0.5)
    assert abs(dl[0, 0, 0, 0] - 0.09 * 0.6) < 1e-16 and abs(dl[1, 0, 0, 0] - 0.25 * 0.9) < 1e-16
    assert abs(dx_[0, 0, 0, 0] - 0.09 * 0.95) < 1e-16 and abs(dx_[1, 0, 0, 0] - 0.25 * 0.7) < 1e-16
    assert np.allclose(d0[:, 0, 0, 0], [0.09, 0.25])


# ----------------------------------------------- V > 1 shells (Eq 10, R17)
def test_cube_L_and_shell_sizes():
    assert [ifcm.cube_L(v) for v in (1, 2, 3, 4)] == [3, 5, 6, 7]
    for V in (1, 2, 3):
        sh = ifcm.shells(V)
        assert [len(s) for s in sh] == [(2 * r + 1) ** 3 - (2 * r - 1) ** 3
                                        for r in range(1, V + 1)]
        for r, s in enumerate(sh, start=1):
            assert all(max(abs(a) for a in o) == r for o in s)
    # with Eq 9's L = 3 the second shell is empty (the ball holds distance 1 only)
    assert len(ifcm.shells(2, L=3)[1]) == 0


def test_interior_Q_of_the_second_shell():
    # sum of dx^2 + dy^2 + dz^2 over the 5^3 cube is 3 * 10 * 25 = 750; the
    # inner 3^3 cube contributes 3 * 2 * 9 = 54; so Q_2 = 696 at an interior voxel
    x = np.random.default_rng(0).random((5, 5, 5))
    U = np.full((2, 5, 5, 5), 0.5)
    _, _, aux = ifcm.neighbour_terms(x, U, V=2, return_aux=True)
    assert aux["Q"][0][2, 2, 2] == 54 and aux["Q"][1][2, 2, 2] == 696
    assert aux["count"][1][2, 2, 2] == 98


def _brute_terms_V(x, U, V, h):
    """Per-voxel loops over the cube of radius V, shell by shell, with the
    weights of Eq 10 renormalised over the shells that hold an in-volume voxel."""
    c = U.shape[0]
    nz, ny, nx = x.shape
    W = np.array([np.exp(-r / h) for r in range(1, V + 1)])
    W = W / W.sum()
    H = np.zeros_like(U)
    F = np.zeros_like(U)
    rng = range(-V, V + 1)
    for z, y, xx in itertools.product(range(nz), range(ny), range(nx)):
        hs, fs, ws = np.zeros(c), np.zeros(c), 0.0
        for r in range(1, V + 1):
            G = Q = 0.0
            n = 0
            hh, ff, ss = np.zeros(c), np.zeros(c), np.zeros(c)
            for dz, dy, dx in itertools.product(rng, rng, rng):
                if max(abs(dz), abs(dy), abs(dx)) != r:
                    continue
                kz, ky, kx = z + dz, y + dy, xx + dx
                if not (0 <= kz < nz and 0 <= ky < ny and 0 <= kx < nx):
                    continue
                gk = abs(x[z, y, xx] - x[kz, ky, kx])
                qk = dx * dx + dy * dy + dz * dz
                hh += U[:, kz, ky, kx] * gk
                ff += U[:, kz, ky, kx] ** 2 * qk
                ss += U[:, kz, ky, kx]
                G += gk
                Q += qk
                n += 1
            if n:
                hs += W[r - 1] * (hh / G if G > 0 else ss / n)
                fs += W[r - 1] * ff / Q
                ws += W[r - 1]
        if ws > 0:
            H[:, z, y, xx] = hs / ws
            F[:, z, y, xx] = fs / ws
    return H, F


@pytest.mark.parametrize("shape,V,h", [((5, 6, 7), 2, 1.0), ((1, 8, 9), 2, 0.5),
                                       ((4, 7, 7), 3, 2.0), ((2, 3, 9), 2, 1.0)])
def test_shells_match_brute_force_loops(shape, V, h):
    x, U = _random_case(shape, 3, 6)
    H, F = ifcm.neighbour_terms(x, U, V=V, h=h)
    Hb, Fb = _brute_terms_V(x, U, V, h)
    assert np.allclose(H, Hb, atol=1e-14)
    assert np.allclose(F, Fb, atol=1e-14)
    assert np.allclose(H.sum(axis=0), 1.0, atol=1e-13)


def test_shells_uniform_memberships():
    x = np.random.default_rng(1).random((4, 6, 5))
    U = np.full((4,) + x.shape, 0.25)
    H, F = ifcm.neighbour_terms(x, U, V=3, h=1.5)
    assert np.allclose(H, 0.25, atol=1e-15) and np.allclose(F, 0.0625, atol=1e-15)

"""GPU (C ABI) vs FP64 oracle, element by element, on seeded inputs.

Tolerances: memberships <= 1e-5 max-abs (FP32 path), centres <= 1e-6
relative, J <= 1e-5 relative, hard labels identical on >= 99.99% of voxels.
Iteration counts are fixed (eps = 0) wherever a stop decision could fall on
either side of the threshold in FP32 vs FP64.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ifcm as O          # noqa: E402
from oracle import pso as OP          # noqa: E402
from paper_2002_01981_gb300 import phantoms  # noqa: E402

pytestmark = pytest.mark.gpu

U_TOL = 1e-5
C_RTOL = 1e-6
J_RTOL = 1e-5


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_01981_gb300 import build
    build.build()
    from paper_2002_01981_gb300 import ifcm
    return ifcm


def dev_vol(a):
    """(nz, ny, nx) float32 -> padded CUDA tensor (nz, ny, pitch)."""
    return torch.from_numpy(phantoms.pad_pitch(np.asarray(a, np.float32))).cuda()


def dev_u(u):
    """(c, nz, ny, nx) float32 -> padded CUDA tensor."""
    c, nz, ny, nx = u.shape
    out = np.zeros((c, nz, ny, phantoms.pitch_for(nx)), np.float32)
    out[..., :nx] = u
    return torch.from_numpy(out).cuda()


def unpad(t, nx):
    return t[..., :nx].cpu().numpy().astype(np.float64)


def unit_volume(shape, seed, sigma=0.06):
    """Seeded phantom already inside [0, 1] (input of the fit entry points)."""
    raw = phantoms.brain_phantom(shape, seed=seed, sigma=sigma)
    return np.clip(raw, 0.0, 1.0).astype(np.float32)


def labels_agree(Ug, Uo):
    return np.mean(np.argmax(Ug, 0) == np.argmax(Uo, 0))


# ------------------------------------------------------------ normalise
@pytest.mark.parametrize("shape", [(7, 13, 29), (1, 64, 64), (3, 1, 5), (33, 41, 37)])
def test_normalize_matches_oracle(G, shape):
    raw = phantoms.brain_phantom(shape, seed=3) * 3.7 - 0.4
    raw = raw.astype(np.float32)
    x = G.ifcm_normalize(dev_vol(raw), nx=shape[2])
    ref = O.normalize(raw)
    got = unpad(x, shape[2])
    assert np.max(np.abs(got - ref)) <= 2.0 ** -23
    assert got.min() == 0.0 and got.max() == 1.0


def test_normalize_flags_constant_and_nonfinite(G):
    from paper_2002_01981_gb300.native import IfcmError
    with pytest.raises(IfcmError):
        G.ifcm_normalize(dev_vol(np.full((4, 5, 6), 0.3, np.float32)), nx=6)
    bad = np.random.default_rng(0).random((4, 5, 6)).astype(np.float32)
    bad[2, 3, 1] = np.nan
    with pytest.raises(IfcmError):
        G.ifcm_normalize(dev_vol(bad), nx=6)


# ----------------------------------------------------- one IFCM iteration
CASES_ONE = [
    # shape (nz, ny, nx), c, m, lambda, xi
    ((9, 14, 21), 4, 2.0, 0.4, 0.3),
    ((5, 17, 70), 3, 2.0, 0.8, 0.6),      # three x tiles, ragged
    ((40, 9, 33), 4, 2.0, 0.5, 0.5),      # two z-chunks, ragged
    ((1, 37, 45), 4, 2.0, 0.7, 0.2),      # 2D: 8-neighbourhood
    ((3, 3, 3), 2, 2.0, 0.9, 0.9),
    ((2, 2, 2), 5, 2.0, 0.3, 0.6),
    ((1, 1, 7), 3, 2.0, 0.5, 0.5),        # a line
    ((1, 1, 1), 2, 2.0, 0.5, 0.5),        # no neighbours: H = F = 0
    ((6, 11, 13), 8, 2.0, 0.6, 0.4),
    ((6, 11, 13), 6, 1.5, 0.6, 0.4),      # general m
    ((4, 10, 12), 4, 3.0, 0.2, 0.7),
    ((7, 12, 10), 4, 2.0, 0.0, 0.0),      # plain FCM step
]


@pytest.mark.parametrize("shape,c,m,lam,xi", CASES_ONE)
def test_one_iteration(G, shape, c, m, lam, xi):
    x = unit_volume(shape, seed=11)
    U = phantoms.random_memberships(shape, c, seed=12)
    C = np.linspace(0.1, 0.9, c)
    prm = G.Params(c=c, m=m, max_iter=1, eps_u=0.0)
    Ug, Cg, Jg, itg = G.ifcm_fit(dev_vol(x), prm, (lam, xi), nx=shape[2], u_init=dev_u(U),
                                 c_init=C)
    Uo, Co, Jo, ito = O.ifcm_fit(x.astype(np.float64), U.astype(np.float64), C, lam, xi, m, 1,
                                 0.0)
    assert itg == ito == 1
    assert np.max(np.abs(unpad(Ug, shape[2]) - Uo)) <= U_TOL
    assert np.allclose(Cg.cpu().numpy(), Co, rtol=C_RTOL, atol=0)
    assert abs(Jg - Jo) <= J_RTOL * abs(Jo)


def test_flat_neighbourhoods(G):
    # noise-free piecewise-constant volume: many voxels have sum_k g_ik = 0
    x = phantoms.piecewise_cube(6, levels=(0.1, 0.5, 0.9), nz=5)
    U = phantoms.random_memberships(x.shape, 3, seed=4)
    C = np.array([0.2, 0.5, 0.8])
    prm = G.Params(c=3, max_iter=1, eps_u=0.0)
    Ug, Cg, Jg, _ = G.ifcm_fit(dev_vol(x), prm, (0.6, 0.3), nx=6, u_init=dev_u(U), c_init=C)
    Uo, Co, Jo, _ = O.ifcm_fit(x.astype(np.float64), U.astype(np.float64), C, 0.6, 0.3, 2.0, 1,
                               0.0)
    assert np.max(np.abs(unpad(Ug, 6) - Uo)) <= U_TOL
    assert np.allclose(Cg.cpu().numpy(), Co, rtol=C_RTOL)


# --------------------------------------------------------- whole runs
@pytest.mark.parametrize("shape,c,lam,xi,iters", [((12, 20, 36), 4, 0.5, 0.4, 20),
                                                  ((1, 64, 64), 4, 0.7, 0.3, 30),
                                                  ((21, 18, 40), 3, 0.45, 0.5, 25)])
def test_fixed_iteration_runs(G, shape, c, lam, xi, iters):
    x = unit_volume(shape, seed=21)
    U = phantoms.random_memberships(shape, c, seed=22)
    C = np.linspace(0.15, 0.85, c)
    prm = G.Params(c=c, max_iter=iters, eps_u=0.0)
    Ug, Cg, Jg, itg = G.ifcm_fit(dev_vol(x), prm, (lam, xi), nx=shape[2], u_init=dev_u(U),
                                 c_init=C)
    Uo, Co, Jo, ito = O.ifcm_fit(x.astype(np.float64), U.astype(np.float64), C, lam, xi, 2.0,
                                 iters, 0.0)
    Ugn = unpad(Ug, shape[2])
    assert itg == ito == iters
    assert np.max(np.abs(Ugn - Uo)) <= U_TOL
    assert np.allclose(Cg.cpu().numpy(), Co, rtol=C_RTOL)
    assert abs(Jg - Jo) <= J_RTOL * abs(Jo)
    assert labels_agree(Ugn, Uo) >= 0.9999


def fp32_floor(x, U, C, lam, xi, iters):
    """How far the FP64 oracle's U moves after a run's iterations when it
    rounds to FP32 in every iteration (a) only its U and C, (b) also its H and
    F: the larger of the two.  That is the part of the GPU-oracle gap that FP32
    storage and the FP32 rounding of the neighbourhood terms alone explain."""
    f32 = lambda a: np.asarray(a).astype(np.float32).astype(np.float64)
    Ua, Ca, Ub, Cb, Uc, Cc = U, C, U, C, U, C
    for _ in range(iters):
        Ua, Ca, _, _ = O.ifcm_iteration(x, Ua, Ca, lam, xi)
        Ub, Cb, _, _ = O.ifcm_iteration(x, Ub, Cb, lam, xi)
        Ub, Cb = f32(Ub), f32(Cb)
        H, F = O.neighbour_terms(x, Uc)
        Uc = O.membership(O.modified_distance(x, Cc, f32(H), f32(F), lam, xi), 2.0)
        Cc = f32(O.centres(x, Uc, 2.0))
        Uc = f32(Uc)
    return max(float(np.max(np.abs(Ua - Ub))), float(np.max(np.abs(Ua - Uc))))


def u_bound(x, U, C, lam, xi, iters):
    """U tolerance of a run: 1e-5, except in the clamp regime (lambda + xi > 1,
    reading R2 of Eq 4), where 1 - lambda H - xi F sits near 0 at many voxels
    and the iteration amplifies FP32 rounding: four times the oracle's own
    FP32 floor (fp32_floor).  The GPU's U error measured 0.93-2.85x the
    storage part of that floor on test_clamp_regime_runs' cases (lean 3D
    kernel) and 3.3x the floor on the 24 x 24 Algorithm 1 run (lean 2D
    kernel: 1.6e-5 against a bound of 2.0e-5)."""
    if lam + xi <= 1.0:
        return U_TOL
    return max(U_TOL, 4.0 * fp32_floor(x, U, C, lam, xi, iters))


@pytest.mark.parametrize("lam,xi", [(0.9, 0.8), (1.0, 1.0), (0.7, 0.6)])
def test_clamp_regime_runs(G, lam, xi):
    # lambda + xi > 1: two clusters can reach 1 - lambda H - xi F <= 0 at once
    # (reading R2), where the iteration amplifies FP32 rounding ~1000x.  The
    # GPU must stay within the oracle's own FP32-storage sensitivity, keep the
    # hard labels, and match centres and J.
    shape, c, iters = (21, 18, 40), 3, 25
    x = unit_volume(shape, seed=21).astype(np.float64)
    U = phantoms.random_memberships(shape, c, seed=22)
    C = np.linspace(0.15, 0.85, c)
    prm = G.Params(c=c, max_iter=iters, eps_u=0.0)
    Ug, Cg, Jg, _ = G.ifcm_fit(dev_vol(x.astype(np.float32)), prm, (lam, xi), nx=shape[2],
                               u_init=dev_u(U), c_init=C)
    Uo, Co, Jo, _ = O.ifcm_fit(x, U.astype(np.float64), C, lam, xi, 2.0, iters, 0.0)
    bound = u_bound(x, U.astype(np.float64), C, lam, xi, iters)
    Ugn = unpad(Ug, shape[2])
    assert np.max(np.abs(Ugn - Uo)) <= bound
    assert labels_agree(Ugn, Uo) >= 0.9999
    # measured on a GB300: C within 3.9e-8, J within 1.4e-7 (relative)
    assert np.allclose(Cg.cpu().numpy(), Co, rtol=C_RTOL)
    assert abs(Jg - Jo) <= J_RTOL * abs(Jo)


def test_plain_form_matches_oracle(G):
    shape = (10, 16, 23)
    x = unit_volume(shape, seed=31)
    U = phantoms.random_memberships(shape, 4, seed=32)
    C = np.linspace(0.1, 0.9, 4)
    prm = G.Params(c=4, max_iter=12, eps_u=0.0)
    Ug, Cg, Jg, itg = G.ifcm_fit(dev_vol(x), prm, (0.6, 0.5), nx=shape[2], u_init=dev_u(U),
                                 c_init=C, plain=True)
    Uo, Co, Jo, ito = O.ifcm_fit(x.astype(np.float64), U.astype(np.float64), C, 0.6, 0.5, 2.0,
                                 12, 0.0)
    assert itg == ito
    assert np.max(np.abs(unpad(Ug, shape[2]) - Uo)) <= U_TOL
    assert np.allclose(Cg.cpu().numpy(), Co, rtol=C_RTOL)


def test_fcm_start_and_stop_rule(G):
    shape = (1, 48, 52)
    raw = phantoms.ellipse_slice(64, seed=1)[:, :48, :52]
    x = O.normalize(raw)
    xg = G.ifcm_normalize(dev_vol(raw), nx=52)
    prm = G.Params(c=4, max_iter=300, eps_u=1e-5)
    Ug, Cg, Jg, itg = G.ifcm_fit(xg, prm, (0.0, 0.0), nx=52)
    Uo, Co, Jo, ito = O.fcm_init(x, 4, 2.0, 300, 1e-5)
    # the stop test is taken in FP32 on the GPU and FP64 in the oracle
    assert abs(itg - ito) <= 1
    assert np.max(np.abs(unpad(Ug, 52) - Uo)) <= 1e-4
    assert np.allclose(Cg.cpu().numpy(), Co, rtol=1e-5)
    # the oracle replaying the GPU's run (its normalised volume, its
    # iteration count) meets the parity bars
    xs = xg.cpu().numpy()[..., :52].astype(np.float64)
    Ur, Cr, Jr, itr = O.fcm_init(xs, 4, 2.0, int(itg), 0.0)
    assert itr == itg
    assert np.max(np.abs(unpad(Ug, 52) - Ur)) <= U_TOL
    assert np.allclose(Cg.cpu().numpy(), Cr, rtol=C_RTOL)
    assert abs(Jg - Jr) <= J_RTOL * abs(Jr)


# ------------------------------------------------------- particle batch
def test_fitness_batch_matches_independent_runs(G):
    shape = (14, 22, 30)
    x = unit_volume(shape, seed=41)
    U0 = phantoms.random_memberships(shape, 4, seed=42)
    C0 = np.array([0.05, 0.3, 0.55, 0.85])
    lam_xi = np.random.default_rng(43).random((7, 2))
    prm = G.Params(c=4, max_iter=15, eps_u=0.0)
    fit, its, cout = G.pso_fitness_batch(dev_vol(x), prm, lam_xi, dev_u(U0), C0, nx=shape[2],
                                         want_centres=True)
    fit, its, cout = fit.cpu().numpy(), its.cpu().numpy(), cout.cpu().numpy()
    for p in range(7):
        _, Co, Jo, ito = O.ifcm_fit(x.astype(np.float64), U0.astype(np.float64), C0,
                                    lam_xi[p, 0], lam_xi[p, 1], 2.0, 15, 0.0)
        assert its[p] == ito
        assert abs(fit[p] - Jo) <= J_RTOL * abs(Jo)
        assert np.allclose(cout[p], Co, rtol=C_RTOL)


def test_fitness_batch_with_stop_rule(G):
    shape = (8, 16, 20)
    x = unit_volume(shape, seed=51)
    xo = x.astype(np.float64)
    U0o, C0o, _, _ = O.fcm_init(xo, 4)
    xg = dev_vol(x)
    U0g, C0g, _, _ = G.ifcm_fit(xg, G.Params(c=4, max_iter=300, eps_u=1e-5), (0.0, 0.0),
                                nx=shape[2])
    lam_xi = np.random.default_rng(52).random((5, 2))
    prm = G.Params(c=4, max_iter=50, eps_u=1e-5)
    fit, its, cen = G.pso_fitness_batch(xg, prm, lam_xi, U0g, C0g, nx=shape[2],
                                        want_centres=True)
    fit, its, cen = fit.cpu().numpy(), its.cpu().numpy(), cen.cpu().numpy()
    U0s, C0s = unpad(U0g, shape[2]), C0g.cpu().numpy().astype(np.float64)
    for p in range(5):
        _, _, Jo, ito = O.ifcm_fit(xo, U0o, C0o, lam_xi[p, 0], lam_xi[p, 1], 2.0, 50, 1e-5)
        assert abs(int(its[p]) - ito) <= 1
        assert abs(fit[p] - Jo) <= 1e-4 * abs(Jo)
        # the oracle replaying each run from the GPU's start for the GPU's
        # iteration count meets the parity bars (measured: J 4.3e-8, C 5.4e-8)
        _, Cr, Jr, _ = O.ifcm_fit(xo, U0s, C0s, lam_xi[p, 0], lam_xi[p, 1], 2.0, int(its[p]),
                                  0.0)
        assert abs(fit[p] - Jr) <= J_RTOL * abs(Jr)
        assert np.allclose(cen[p], Cr, rtol=C_RTOL)


# ------------------------------------------------------------- swarm
@pytest.mark.parametrize("P,radius,seed", [(1, 1, 3), (2, 1, 4), (3, 0, 5), (20, 1, 6),
                                           (64, 2, 7), (10, 1, 2**40 + 17)])
def test_swarm_is_bit_identical(G, P, radius, seed):
    sw = G.Swarm(P, seed=seed, radius=radius, vmax=0.2).init()
    ref = OP.Swarm(P, seed=seed, vmax=0.2, radius=radius)
    assert np.array_equal(sw.x.cpu().numpy(), ref.x)
    assert np.array_equal(sw.v.cpu().numpy(), ref.v)
    rng = np.random.default_rng(seed % 1000)
    for g in range(12):
        f = rng.random(P)
        if g == 5:
            f[:] = 0.25          # ties everywhere
        sw.step(torch.tensor(f, device="cuda"))
        OP.pso_step(ref, f)
        assert np.array_equal(sw.x.cpu().numpy(), ref.x)
        assert np.array_equal(sw.v.cpu().numpy(), ref.v)
        assert np.array_equal(sw.pbest_x.cpu().numpy(), ref.pbest_x)
        assert np.array_equal(sw.pbest_f.cpu().numpy(), ref.pbest_f)
    assert int(sw.gen.item()) == ref.gen


# ------------------------------------------------------------ Algorithm 1
def test_pifcm3d_ellipse_slice_full_workload(G):
    # the 64 x 64 ellipse slice at its workload's full parameters: c = 4,
    # 10 particles x 20 generations, <= 50 iterations, stop max|du| < 1e-5.
    # FP32 and FP64 stop tests may end a run an iteration apart, and that can
    # steer the two swarms apart, so the GPU's own result is checked: its
    # final run at the (lambda, xi) it reports, against the oracle's run there
    # from the oracle's FCM start
    raw = phantoms.ellipse_slice(64, seed=1, sigma=0.05)
    prm = G.Params(c=4, max_iter=50, eps_u=1e-5)
    opts = G.Options(P=10, generations=20, seed=1, init_max_iter=300)
    U, res = G.pifcm3d(dev_vol(raw), prm, opts, nx=64)
    assert res["status"] == 0
    assert 0.0 <= res["lambda"] <= 1.0 and 0.0 <= res["xi"] <= 1.0
    x = O.normalize(raw)
    U0, C0, _, it0 = O.fcm_init(x, 4, 2.0, 300, 1e-5)
    assert abs(res["iters_init"] - it0) <= 1
    Uo, Co, Jo, ito = O.ifcm_fit(x, U0, C0, res["lambda"], res["xi"], 2.0, 50, 1e-5)
    assert abs(res["iters_final"] - ito) <= 1
    assert labels_agree(unpad(U, 64), Uo) >= 0.999
    assert np.allclose(res["centres"], Co, rtol=1e-4, atol=0)
    assert abs(res["J"] - Jo) <= 1e-4 * abs(Jo)
    # The same final run replayed by the oracle from the GPU's own normalised
    # volume and FCM start (the same resident launch as pifcm3d's, from
    # u = 1/c and c_j = (j + 1/2)/c), for the GPU's iteration count.  Only
    # FP32 rounding separates the two, so the parity bars apply: U within the
    # clamp-regime conditioning bound (u_bound), labels, C and J.
    xg = G.ifcm_normalize(dev_vol(raw), nx=64)
    U0g, C0g, _, it0g = G.ifcm_fit(xg, G.Params(c=4, max_iter=300, eps_u=1e-5), (0.0, 0.0),
                                   nx=64)
    assert it0g == res["iters_init"]
    xs = xg.cpu().numpy()[..., :64].astype(np.float64)
    U0s = unpad(U0g, 64).astype(np.float64)
    C0s = C0g.cpu().numpy().astype(np.float64)
    lam, xi, its = res["lambda"], res["xi"], res["iters_final"]
    Ur, Cr, Jr, _ = O.ifcm_fit(xs, U0s, C0s, lam, xi, 2.0, its, 0.0)
    assert np.max(np.abs(unpad(U, 64) - Ur)) <= u_bound(xs, U0s, C0s, lam, xi, its)
    assert labels_agree(unpad(U, 64), Ur) >= 0.9999
    # measured at (lambda, xi) = (1, 1), 50 iterations: U 8.6e-8, C 1.2e-8
    assert np.allclose(res["centres"], Cr, rtol=C_RTOL, atol=0)
    assert abs(res["J"] - Jr) <= J_RTOL * abs(Jr)


def test_pifcm3d_small_run_matches_oracle(G):
    raw = phantoms.ellipse_slice(24, seed=1, sigma=0.05)
    prm = G.Params(c=4, max_iter=8, eps_u=0.0)
    opts = G.Options(P=4, generations=3, seed=9, init_max_iter=40)
    U, res = G.pifcm3d(dev_vol(raw), prm, opts, nx=24)
    ref = OP.pifcm3d(raw, c=4, P=4, generations=3, seed=9, max_iter=8, eps=0.0,
                     init_max_iter=40)
    assert res["status"] == 0
    # each swarm is driven by its own fitness values; they agree unless a
    # personal-best comparison is a near tie (none expected at these sizes)
    assert res["lambda"] == ref["lambda"] and res["xi"] == ref["xi"]
    x = O.normalize(raw)
    U0, C0, _, _ = O.fcm_init(x, 4, 2.0, 40, 0.0)
    bound = u_bound(x, U0, C0, ref["lambda"], ref["xi"], 8)
    assert np.max(np.abs(unpad(U, 24) - ref["U"])) <= bound
    assert labels_agree(unpad(U, 24), ref["U"]) >= 0.9999
    assert np.allclose(res["centres"], ref["C"], rtol=1e-5)
    assert abs(res["J"] - ref["J"]) <= J_RTOL * abs(ref["J"])
    assert res["iters_final"] == ref["iters"]
    assert abs(res["best_fitness"] - ref["pbest_f"].min()) <= J_RTOL * ref["pbest_f"].min()


def test_pifcm3d_host_equals_device(G):
    raw = phantoms.brain_phantom((10, 12, 14), seed=5)
    vol = phantoms.pad_pitch(raw)
    prm = G.Params(c=4, max_iter=6, eps_u=0.0)
    opts = G.Options(P=3, generations=2, seed=2, init_max_iter=30)
    Ud, rd = G.pifcm3d(torch.from_numpy(vol).cuda(), prm, opts, nx=14)
    uh = torch.empty((4,) + vol.shape, dtype=torch.float32).pin_memory()
    _, rh = G.pifcm3d_host(torch.from_numpy(vol).pin_memory(), prm, opts, nx=14, u_out=uh)
    assert rd == rh
    assert torch.equal(Ud.cpu()[..., :14], uh[..., :14])


@pytest.mark.parametrize("slice_z", [-1, 2])
def test_split_swarm_on_one_rank_equals_pifcm3d(G, slice_z):
    # the split driver (fitness slices + allgather + identical swarm steps)
    # with a single rank runs exactly pifcm3d's launches
    from paper_2002_01981_gb300 import distributed as D
    raw = phantoms.brain_phantom((6, 20, 22), seed=12, sigma=0.05)
    prm = G.Params(c=3, max_iter=6, eps_u=1e-5)
    opts = G.Options(P=5, generations=3, seed=4, init_max_iter=40, slice_z=slice_z)
    Ua, ra = G.pifcm3d(dev_vol(raw), prm, opts, nx=22)
    Ub, rb = D.pifcm3d_split(dev_vol(raw), prm, opts, nx=22)
    assert (rb["lambda"], rb["xi"]) == (ra["lambda"], ra["xi"])
    assert rb["J"] == ra["J"] and rb["best_fitness"] == ra["best_fitness"]
    assert rb["iters_final"] == ra["iters_final"] and rb["iters_init"] == ra["iters_init"]
    assert np.array_equal(rb["centres"], np.asarray(ra["centres"]))
    assert torch.equal(Ua[..., :22], Ub[..., :22])


def test_pifcm3d_graph_replays_equal_direct_runs(G):
    raw = phantoms.brain_phantom((7, 18, 21), seed=13, sigma=0.05)
    prm = G.Params(c=4, max_iter=6, eps_u=1e-5)
    opts = G.Options(P=4, generations=3, seed=6, init_max_iter=30)
    vol = dev_vol(raw)
    Ud, rd = G.pifcm3d(vol, prm, opts, nx=21)
    graph = G.pifcm3d_graph(vol, prm, opts, nx=21)
    for _ in range(2):
        graph.launch()
        rg = graph.result()
        assert rg == rd
        assert torch.equal(graph.u_out[..., :21], Ud[..., :21])
    # a replay follows the buffer's new contents
    vol.copy_(dev_vol(phantoms.brain_phantom((7, 18, 21), seed=14, sigma=0.05)))
    graph.launch()
    _, rd2 = G.pifcm3d(vol, prm, opts, nx=21)
    assert graph.result() == rd2 and rd2 != rd
    graph.close()


def test_pifcm3d_slice_mode(G):
    raw = phantoms.brain_phantom((6, 20, 22), seed=8)
    prm = G.Params(c=3, max_iter=5, eps_u=0.0)
    opts = G.Options(P=3, generations=2, seed=4, init_max_iter=30, slice_z=2)
    U, res = G.pifcm3d(dev_vol(raw), prm, opts, nx=22)
    ref = OP.pifcm3d(raw, c=3, P=3, generations=2, seed=4, max_iter=5, eps=0.0,
                     init_max_iter=30, z=2)
    assert U.shape[1] == 1
    assert res["lambda"] == ref["lambda"]
    x = O.normalize(raw)[2:3]
    U0, C0, _, _ = O.fcm_init(x, 3, 2.0, 30, 0.0)
    bound = u_bound(x, U0, C0, ref["lambda"], ref["xi"], 5)
    assert np.max(np.abs(unpad(U, 22) - ref["U"])) <= bound
    # measured on a GB300: C within 4.9e-8, J within 4.2e-7 (relative)
    assert np.allclose(res["centres"], ref["C"], rtol=C_RTOL)
    assert abs(res["J"] - ref["J"]) <= J_RTOL * abs(ref["J"])


# ------------------------------------------- many volumes in one launch
MULTI_SPECS = [((9, 14, 21), 3, 3), ((16, 12, 33), 4, 5), ((5, 30, 17), 3, 1),
               ((12, 12, 12), 6, 4), ((20, 9, 40), 4, 2), ((1, 40, 37), 4, 3)]


def _multi_inputs(G, specs, seed, scale=1.0):
    # scale <= 0.5 keeps lambda + xi <= 1, out of the clamp regime
    vols, host = [], []
    for k, (shape, c, P) in enumerate(specs):
        x = unit_volume(shape, seed=seed + k)
        U0 = phantoms.random_memberships(shape, c, seed=seed + 100 + k)
        C0 = np.sort(np.random.default_rng(seed + 200 + k).random(c))
        lam_xi = np.random.default_rng(seed + 300 + k).random((P, 2)) * scale
        vols.append(G.BatchVolume(dev_vol(x), c, lam_xi, dev_u(U0), C0, nx=shape[2]))
        host.append((x, U0, C0, lam_xi))
    return vols, host


@pytest.mark.parametrize("eps", [0.0, 1e-5])
def test_fitness_multi_equals_single_volume_runs(G, eps):
    vols, _ = _multi_inputs(G, MULTI_SPECS, seed=61)
    prm = G.Params(max_iter=12, eps_u=eps)
    outs = G.pso_fitness_multi(vols, prm)
    for v, (fit, its) in zip(vols, outs):
        f1, i1 = _single_call(G, v, G.Params(c=v.c, max_iter=12, eps_u=eps))
        # same arithmetic per (particle, tile) and a fixed reduction order
        assert _same_fitness(fit, f1, len(fit), flat=v.x.shape[0] == 1)
        assert torch.equal(its, i1)


def test_fitness_multi_matches_oracle(G):
    vols, host = _multi_inputs(G, MULTI_SPECS, seed=71)
    outs = G.pso_fitness_multi(vols, G.Params(max_iter=8, eps_u=0.0))
    for (x, U0, C0, lam_xi), (fit, its) in zip(host, outs):
        fo, io = OP.fitness_batch(x.astype(np.float64), U0.astype(np.float64), C0, lam_xi,
                                  max_iter=8, eps=0.0)
        assert np.array_equal(its.cpu().numpy(), io)
        assert np.all(np.abs(fit.cpu().numpy() - fo) <= J_RTOL * np.abs(fo))


def test_fitness_batch_at_the_particle_limit(G):
    # the most particles one batch takes (1024): every particle's J and C
    # against the oracle (lambda + xi <= 1, out of the clamp regime, where the
    # parity bars apply); one more is rejected before anything is launched
    from paper_2002_01981_gb300.native import IfcmError
    shape, c, P = (3, 4, 5), 3, 1024
    x = unit_volume(shape, seed=41)
    U0 = phantoms.random_memberships(shape, c, seed=42)
    C0 = np.array([0.2, 0.5, 0.8])
    lam_xi = np.random.default_rng(43).random((P, 2)) * 0.5
    prm = G.Params(c=c, max_iter=3, eps_u=0.0)
    fit, its, cen = G.pso_fitness_batch(dev_vol(x), prm, lam_xi, dev_u(U0), C0, nx=shape[2],
                                        want_centres=True)
    fit, its, cen = fit.cpu().numpy(), its.cpu().numpy(), cen.cpu().numpy()
    assert np.all(its == 3)
    x64, U64 = x.astype(np.float64), U0.astype(np.float64)
    for p in range(P):
        _, Co, Jo, _ = O.ifcm_fit(x64, U64, C0, lam_xi[p, 0], lam_xi[p, 1], 2.0, 3, 0.0)
        assert abs(fit[p] - Jo) <= J_RTOL * abs(Jo), p
        assert np.allclose(cen[p], Co, rtol=C_RTOL), p
    with pytest.raises(IfcmError):
        G.pso_fitness_batch(dev_vol(x), prm, np.full((P + 1, 2), 0.5), dev_u(U0), C0,
                            nx=shape[2])


def test_fitness_multi_at_the_launch_limits(G):
    # 70 volumes of 64 particles: the first wave fills one launch's 64 volumes
    # and 4096 particles at once, the second takes the other 6 volumes
    specs = [((2 + k % 3, 3 + k % 4, 4 + k % 5), 3, 64) for k in range(70)]
    vols, host = _multi_inputs(G, specs, seed=91, scale=0.5)
    prm = G.Params(max_iter=3, eps_u=0.0)
    ws_bytes = G.pso_fitness_multi_workspace_bytes(vols, prm)
    assert G.pso_fitness_multi_waves(vols, prm, ws_bytes) == 2
    outs = G.pso_fitness_multi(vols, prm)
    for (x, U0, C0, lam_xi), (fit, its) in zip(host, outs):
        fo, io = OP.fitness_batch(x.astype(np.float64), U0.astype(np.float64), C0, lam_xi,
                                  max_iter=3, eps=0.0)
        assert np.array_equal(its.cpu().numpy(), io)
        assert np.all(np.abs(fit.cpu().numpy() - fo) <= J_RTOL * np.abs(fo))


def test_fitness_multi_in_workspace_sized_waves(G):
    # the smallest workspace runs one volume per wave; results do not change
    vols, _ = _multi_inputs(G, MULTI_SPECS, seed=81)
    prm = G.Params(max_iter=6, eps_u=1e-5)
    full = G.pso_fitness_multi(vols, prm)
    lo = G.pso_fitness_multi_workspace_bytes(vols, prm, minimum=True)
    assert lo < G.pso_fitness_multi_workspace_bytes(vols, prm)
    small = G.pso_fitness_multi(vols, prm, ws=G.workspace(lo))
    for v, (fa, ia), (fb, ib) in zip(vols, full, small):
        assert _same_fitness(fa, fb, len(fa), flat=v.x.shape[0] == 1) and torch.equal(ia, ib)


def _same_fitness(fit, f1, P, flat=False):
    """Multi-volume fitness against the single-volume call (_single_call).
    Bit-equal when both launches cut the volume alike.  A 2D image (flat) is
    cut into runs of tiles whose length follows the launch's plan, and a
    thread's FP32 sums run over its run of tiles, so it uses the J bar (1e-5
    relative)."""
    if flat:
        return torch.allclose(fit, f1, rtol=J_RTOL, atol=0)
    return torch.equal(fit, f1)


def _single_call(G, v, prm):
    """The single-volume call a multi-volume volume is compared with.  In a
    multi-volume launch a volume's particles run in pairs; a lone particle
    shares its pair with a copy of itself.  So a one-particle volume is
    compared with a two-particle call on two copies of it, which runs the same
    kernel with the same arithmetic, not with a one-particle call (a different
    kernel, with its clusters paired in the packed lanes)."""
    lx = np.asarray(v.lam_xi, np.float64).reshape(-1, 2)
    if len(lx) == 1:
        lx = np.concatenate([lx, lx])
    f1, i1, _ = G.pso_fitness_batch(v.x, prm, lx, v.u0, v.c0, nx=v.nx)
    n = len(np.asarray(v.lam_xi).reshape(-1, 2))
    return f1[:n], i1[:n]


def test_fitness_multi_beyond_one_launch(G):
    # 70 volumes (more than one launch holds) and 5000 particles on 5 volumes
    # (more particles than one launch holds) split into several launches
    specs = [((3 + k % 5, 4 + k % 3, 5 + k % 7), 2 + k % 3, 1 + k % 2) for k in range(70)]
    vols, _ = _multi_inputs(G, specs, seed=91)
    prm = G.Params(max_iter=4, eps_u=0.0)
    outs = G.pso_fitness_multi(vols, prm)
    for v, (fit, its) in zip(vols, outs):
        f1, i1 = _single_call(G, v, G.Params(c=v.c, max_iter=4, eps_u=0.0))
        assert _same_fitness(fit, f1, len(fit), flat=v.x.shape[0] == 1) and torch.equal(its, i1)
    big = [((4, 6, 8), 3, 1000), ((5, 5, 9), 3, 1000), ((6, 4, 7), 3, 1000),
           ((3, 7, 8), 3, 1000), ((4, 4, 4), 3, 1000)]
    vols, _ = _multi_inputs(G, big, seed=95)
    outs = G.pso_fitness_multi(vols, prm)
    for v, (fit, its) in zip(vols, outs):
        f1, i1, _ = G.pso_fitness_batch(v.x, G.Params(c=3, max_iter=4, eps_u=0.0), v.lam_xi,
                                        v.u0, v.c0, nx=v.nx)
        assert torch.equal(fit, f1) and torch.equal(its, i1)


# ------------------------------------------------ work decomposition plans
@pytest.mark.parametrize("c,np_,chunks", [(4, 1, 1), (4, 2, 1), (4, 1, 3), (4, 2, 100),
                                          (3, 1, 2), (5, 2, 1), (5, 2, 3), (5, 1, 2),
                                          (6, 1, 1), (6, 1, 100), (2, 2, 4)])
def test_every_plan_matches_oracle(G, c, np_, chunks):
    # z = 37 planes: up to five chunks (the last one ragged), x and y tails too
    shape = (37, 30, 70)
    x = unit_volume(shape, seed=121)
    U0 = phantoms.random_memberships(shape, c, seed=122)
    C0 = np.sort(np.random.default_rng(123).random(c))
    lam_xi = np.random.default_rng(124).random((3, 2)) * 0.6
    G.force_plan(np_, chunks)
    try:
        fit, its, cout = G.pso_fitness_batch(dev_vol(x), G.Params(c=c, max_iter=6, eps_u=0.0),
                                             lam_xi, dev_u(U0), C0, nx=shape[2],
                                             want_centres=True)
    finally:
        G.force_plan(0)
    fo, io = OP.fitness_batch(x.astype(np.float64), U0.astype(np.float64), C0, lam_xi,
                              max_iter=6, eps=0.0)
    assert np.array_equal(its.cpu().numpy(), io)
    assert np.all(np.abs(fit.cpu().numpy() - fo) <= J_RTOL * np.abs(fo))


@pytest.mark.parametrize("chunks", [0, 1, 3, 10])
def test_2d_runs_of_tiles_match_oracle(G, chunks):
    # a 2D image of 100 rows (10 tiles of 11 rows, the last with one row: lanes
    # outside the image in the masked form) and 45 columns (a ragged x tile);
    # chunks cut each column of tiles into runs: the rule (0), whole columns
    # (1), runs of 4, 4 and 2 tiles (3), one tile per item (10)
    shape = (1, 100, 45)
    x = unit_volume(shape, seed=141)
    U0 = phantoms.random_memberships(shape, 4, seed=142)
    C0 = np.sort(np.random.default_rng(143).random(4))
    lam_xi = np.random.default_rng(144).random((6, 2)) * 0.6
    if chunks:
        G.force_plan(2, chunks)
    try:
        fit, its, _ = G.pso_fitness_batch(dev_vol(x), G.Params(c=4, max_iter=6, eps_u=0.0),
                                          lam_xi, dev_u(U0), C0, nx=shape[2])
    finally:
        G.force_plan(0)
    fo, io = OP.fitness_batch(x.astype(np.float64), U0.astype(np.float64), C0, lam_xi,
                              max_iter=6, eps=0.0)
    assert np.array_equal(its.cpu().numpy(), io)
    assert np.all(np.abs(fit.cpu().numpy() - fo) <= J_RTOL * np.abs(fo))


@pytest.mark.parametrize("c,P", [(4, 4), (3, 3), (6, 2)])
def test_lean_2d_kernel_on_the_largest_sweep_slice(G, c, P):
    # the 854 x 854 slice of the 2D sweep: iteration 1 from a shared random
    # start runs the general kernel, iteration 2 (U^t from Eq 2) the lean 2D
    # kernel -- two particles per item for c <= 5, one for c = 6.  J, C of
    # every particle against the oracle, and U of one particle (ifcm_fit, the
    # one-particle form) on every pixel
    n = 854
    raw = phantoms.brain_slice(n, seed=2, sigma=0.07)
    x = O.normalize(raw).astype(np.float32)
    U0 = phantoms.random_memberships(x.shape, c, seed=151)
    C0 = np.linspace(0.1, 0.9, c)
    lam_xi = np.random.default_rng(152).random((P, 2)) * 0.5
    prm = G.Params(c=c, max_iter=2, eps_u=0.0)
    G.profile_read(G.PROF_STENCIL)
    G.profile_enable(True)
    try:
        fit, its, cen = G.pso_fitness_batch(dev_vol(x), prm, lam_xi, dev_u(U0), C0, nx=n,
                                            want_centres=True)
        Ug, Cg, Jg, _ = G.ifcm_fit(dev_vol(x), prm, tuple(lam_xi[0]), nx=n, u_init=dev_u(U0),
                                   c_init=C0)
        torch.cuda.synchronize()
    finally:
        G.profile_enable(False)
    assert G.profile_read(G.PROF_STENCIL)[1] == 4           # two launches per call
    assert np.all(its.cpu().numpy() == 2)
    fit, cen = fit.cpu().numpy(), cen.cpu().numpy()
    x64 = x.astype(np.float64)
    for p in range(P):
        Uo, Co, Jo, _ = O.ifcm_fit(x64, U0.astype(np.float64), C0, lam_xi[p, 0], lam_xi[p, 1],
                                   2.0, 2, 0.0)
        assert abs(fit[p] - Jo) <= J_RTOL * abs(Jo), p
        assert np.allclose(cen[p], Co, rtol=C_RTOL, atol=0), p
        if p == 0:
            assert np.max(np.abs(unpad(Ug, n) - Uo)) <= U_TOL
            assert np.allclose(Cg.cpu().numpy(), Co, rtol=C_RTOL)
            assert abs(Jg - Jo) <= J_RTOL * abs(Jo)


def test_autotuned_plan_is_cached_and_matches_oracle(G):
    shape = (24, 40, 70)
    x = unit_volume(shape, seed=131)
    U0 = phantoms.random_memberships(shape, 4, seed=132)
    C0 = np.array([0.1, 0.35, 0.6, 0.85])
    lam_xi = np.random.default_rng(133).random((5, 2)) * 0.6
    xg = dev_vol(x)
    G.autotune_reset()
    G.autotune(1)
    try:
        fit, its, _ = G.pso_fitness_batch(xg, G.Params(c=4, max_iter=5, eps_u=0.0), lam_xi,
                                          dev_u(U0), C0, nx=shape[2])
        npp, tz, tuned = G.stencil_plan(G.shape_of(xg, shape[2]), 4, 5)
    finally:
        G.autotune(0)
        G.autotune_reset()
    assert tuned and npp in (1, 2) and 8 <= tz <= 24
    fo, io = OP.fitness_batch(x.astype(np.float64), U0.astype(np.float64), C0, lam_xi,
                              max_iter=5, eps=0.0)
    assert np.array_equal(its.cpu().numpy(), io)
    assert np.all(np.abs(fit.cpu().numpy() - fo) <= J_RTOL * np.abs(fo))


def test_fitness_graph_replays_follow_the_inputs(G):
    vols, _ = _multi_inputs(G, MULTI_SPECS, seed=141)
    for v in vols:
        v.lam_xi = torch.tensor(v.lam_xi, dtype=torch.float64, device="cuda")
    prm = G.Params(max_iter=7, eps_u=1e-5)
    graph = G.pso_fitness_multi_graph(vols, prm)
    try:
        for trial in range(2):
            if trial:
                for k, v in enumerate(vols):       # the swarm moves: new values, same buffers
                    v.lam_xi.copy_(torch.rand(v.lam_xi.shape, dtype=torch.float64,
                                              generator=torch.Generator().manual_seed(k))
                                   .cuda())
            graph.launch()
            graph.check()
            direct = G.pso_fitness_multi(vols, prm)
            for (fg, ig), (fd, id_) in zip(graph.outputs, direct):
                assert torch.equal(fg, fd) and torch.equal(ig, id_)
    finally:
        graph.close()

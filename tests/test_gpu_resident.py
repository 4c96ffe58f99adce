"""Resident runs (ifcm_resident_enable, on by default) against the FP64 oracle:
batches whose every volume fits one CTA's shared memory run every particle's
whole IFCM run (Alg 1 step 4, reading R5) in one launch, and pifcm3d's FCM
start (Alg 1 step 2) likewise.  The arithmetic per voxel is that of the plain
kernel, so the FP32 bars of the parity suite apply unchanged: memberships
<= 1e-5 max-abs, centres <= 1e-6 relative, J <= 1e-5 relative, iteration
counts equal at fixed counts and within one where the stop rule decides in
FP32 on the GPU and FP64 in the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ifcm as O          # noqa: E402
from oracle import pso as OP          # noqa: E402
from paper_2002_01981_gb300 import phantoms  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.resident]

U_TOL = 1e-5
C_RTOL = 1e-6
J_RTOL = 1e-5
SMEM = 225 * 1024                      # shared-memory bound of a resident run


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_01981_gb300 import build
    build.build()
    from paper_2002_01981_gb300 import ifcm
    return ifcm


def dev_vol(a):
    return torch.from_numpy(phantoms.pad_pitch(np.asarray(a, np.float32))).cuda()


def dev_u(u):
    c, nz, ny, nx = u.shape
    out = np.zeros((c, nz, ny, phantoms.pitch_for(nx)), np.float32)
    out[..., :nx] = u
    return torch.from_numpy(out).cuda()


def unpad(t, nx):
    return t[..., :nx].cpu().numpy().astype(np.float64)


def unit_volume(shape, seed, sigma=0.06):
    raw = phantoms.brain_phantom(shape, seed=seed, sigma=sigma)
    return np.clip(raw, 0.0, 1.0).astype(np.float32)


def u_bound(x, U, C, lam, xi, iters):
    """U tolerance of a run: 1e-5, except in the clamp regime (lambda + xi > 1,
    reading R2 of Eq 4).  There 1 - lambda H - xi F sits near 0 at many voxels
    and the iteration amplifies FP32 rounding, so the bound is four times the
    FP64 oracle's own FP32 sensitivity: how far it moves, at worst over the
    run's iterations, when its U, C, H and F are rounded to FP32 in every
    iteration.  (The resident form rounds H, F and the factor of Eq 4 in
    another order than the stencil kernels; on the 24 x 24 Algorithm 1 run
    its final U error measured 2.5e-5, where this sensitivity peaks at 1.5e-5
    during the run and ends at 5e-6.)"""
    if lam + xi <= 1.0:
        return U_TOL
    f32 = lambda a: np.asarray(a).astype(np.float32).astype(np.float64)
    Ua, Ca, Ub, Cb = U, C, U, C
    worst = 0.0
    for _ in range(iters):
        Ua, Ca, _, _ = O.ifcm_iteration(x, Ua, Ca, lam, xi)
        H, F = O.neighbour_terms(x, Ub)
        d2 = O.modified_distance(x, Cb, f32(H), f32(F), lam, xi)
        Ub = O.membership(d2, 2.0)
        Cb = f32(O.centres(x, Ub, 2.0))
        Ub = f32(Ub)
        worst = max(worst, float(np.max(np.abs(Ua - Ub))))
    return max(U_TOL, 4.0 * worst)


def stencil_launches(G, fn):
    """Runs fn and returns how many stencil launches it made (0 for a
    resident run)."""
    G.profile_read(G.PROF_STENCIL)
    G.profile_enable(True)
    try:
        out = fn()
        torch.cuda.synchronize()
    finally:
        G.profile_enable(False)
    return out, G.profile_read(G.PROF_STENCIL)[1]


# shapes: 2D and 3D, a line, one voxel, ragged sizes, the largest volume that
# fits at c = 4 (80 x 80 = 6400 voxels) and at c = 8 (3388 voxels)
CASES = [((1, 32, 32), 4, 2.0), ((9, 14, 21), 4, 2.0), ((1, 1, 7), 3, 2.0), ((1, 1, 1), 2, 2.0),
         ((5, 11, 13), 8, 2.0), ((1, 80, 80), 4, 2.0), ((2, 41, 41), 8, 2.0),
         ((6, 10, 12), 3, 1.5), ((4, 9, 11), 5, 3.0)]


@pytest.mark.parametrize("shape,c,m", CASES)
def test_batch_matches_oracle(G, shape, c, m):
    assert (1 + 2 * c) * 4 * int(np.prod(shape)) <= SMEM
    x = unit_volume(shape, seed=11)
    U0 = phantoms.random_memberships(shape, c, seed=12)
    C0 = np.linspace(0.1, 0.9, c)
    lam_xi = np.random.default_rng(13).random((5, 2)) * 0.6
    prm = G.Params(c=c, m=m, max_iter=12, eps_u=0.0)
    (fit, its, cout), n_st = stencil_launches(
        G, lambda: G.pso_fitness_batch(dev_vol(x), prm, lam_xi, dev_u(U0), C0, nx=shape[2],
                                       want_centres=True))
    assert n_st == 0                     # one resident launch, no stencil launch
    fit, its, cout = fit.cpu().numpy(), its.cpu().numpy(), cout.cpu().numpy()
    for p in range(5):
        _, Co, Jo, ito = O.ifcm_fit(x.astype(np.float64), U0.astype(np.float64), C0,
                                    lam_xi[p, 0], lam_xi[p, 1], m, 12, 0.0)
        assert its[p] == ito == 12
        assert abs(fit[p] - Jo) <= J_RTOL * abs(Jo)
        assert np.allclose(cout[p], Co, rtol=C_RTOL, atol=0)


@pytest.mark.parametrize("shape,c,lam,xi", [((1, 48, 48), 4, 0.5, 0.3), ((7, 12, 15), 3, 0.2, 0.6),
                                            ((1, 1, 1), 4, 0.4, 0.4)])
def test_fit_memberships_match_oracle(G, shape, c, lam, xi):
    x = unit_volume(shape, seed=21)
    U = phantoms.random_memberships(shape, c, seed=22)
    C = np.linspace(0.15, 0.85, c)
    prm = G.Params(c=c, max_iter=15, eps_u=0.0)
    (Ug, Cg, Jg, itg), n_st = stencil_launches(
        G, lambda: G.ifcm_fit(dev_vol(x), prm, (lam, xi), nx=shape[2], u_init=dev_u(U),
                              c_init=C))
    assert n_st == 0
    Uo, Co, Jo, ito = O.ifcm_fit(x.astype(np.float64), U.astype(np.float64), C, lam, xi, 2.0, 15,
                                 0.0)
    assert itg == ito == 15
    assert np.max(np.abs(unpad(Ug, shape[2]) - Uo)) <= U_TOL
    assert np.allclose(Cg.cpu().numpy(), Co, rtol=C_RTOL)
    assert abs(Jg - Jo) <= J_RTOL * abs(Jo)


@pytest.mark.parametrize("lam,xi", [(0.9, 0.8), (1.0, 1.0), (0.7, 0.6)])
def test_clamp_regime_runs(G, lam, xi):
    # lambda + xi > 1 (reading R2): labels, centres and J at the parity
    # suite's bars; U within the conditioning bound of u_bound
    shape, c, iters = (6, 18, 40), 3, 25
    x = unit_volume(shape, seed=21).astype(np.float64)
    U = phantoms.random_memberships(shape, c, seed=22).astype(np.float64)
    C = np.linspace(0.15, 0.85, c)
    prm = G.Params(c=c, max_iter=iters, eps_u=0.0)
    (Ug, Cg, Jg, _), n_st = stencil_launches(
        G, lambda: G.ifcm_fit(dev_vol(x.astype(np.float32)), prm, (lam, xi), nx=shape[2],
                              u_init=dev_u(U.astype(np.float32)), c_init=C))
    assert n_st == 0
    Uo, Co, Jo, _ = O.ifcm_fit(x, U, C, lam, xi, 2.0, iters, 0.0)
    Ugn = unpad(Ug, shape[2])
    assert np.max(np.abs(Ugn - Uo)) <= u_bound(x, U, C, lam, xi, iters)
    assert np.mean(np.argmax(Ugn, 0) == np.argmax(Uo, 0)) >= 0.9999
    # measured on a GB300: C within 5.8e-8, J within 1.4e-6 (relative)
    assert np.allclose(Cg.cpu().numpy(), Co, rtol=C_RTOL)
    assert abs(Jg - Jo) <= J_RTOL * abs(Jo)


def test_flat_neighbourhoods(G):
    # noise-free piecewise-constant volume: many voxels have sum_k g_ik = 0
    # (reading R3: the plain mean of the in-volume neighbours)
    x = phantoms.piecewise_cube(6, levels=(0.1, 0.5, 0.9), nz=5)
    U = phantoms.random_memberships(x.shape, 3, seed=4)
    C = np.array([0.2, 0.5, 0.8])
    prm = G.Params(c=3, max_iter=3, eps_u=0.0)
    Ug, Cg, Jg, _ = G.ifcm_fit(dev_vol(x), prm, (0.6, 0.3), nx=6, u_init=dev_u(U), c_init=C)
    Uo, Co, Jo, _ = O.ifcm_fit(x.astype(np.float64), U.astype(np.float64), C, 0.6, 0.3, 2.0, 3,
                               0.0)
    assert np.max(np.abs(unpad(Ug, 6) - Uo)) <= U_TOL
    assert np.allclose(Cg.cpu().numpy(), Co, rtol=C_RTOL)
    assert abs(Jg - Jo) <= J_RTOL * abs(Jo)


def test_stop_rule(G):
    shape = (1, 40, 40)
    x = unit_volume(shape, seed=51)
    xo = x.astype(np.float64)
    U0o, C0o, _, _ = O.fcm_init(xo, 4)
    xg = dev_vol(x)
    U0g, C0g, _, it0 = G.ifcm_fit(xg, G.Params(c=4, max_iter=300, eps_u=1e-5), (0.0, 0.0),
                                  nx=shape[2])
    lam_xi = np.random.default_rng(52).random((6, 2)) * 0.5
    prm = G.Params(c=4, max_iter=50, eps_u=1e-5)
    fit, its, cen = G.pso_fitness_batch(xg, prm, lam_xi, U0g, C0g, nx=shape[2],
                                        want_centres=True)
    fit, its, cen = fit.cpu().numpy(), its.cpu().numpy(), cen.cpu().numpy()
    assert np.all(its < 50)             # every run stopped on its own rule
    U0s, C0s = unpad(U0g, shape[2]), C0g.cpu().numpy().astype(np.float64)
    for p in range(6):
        _, _, Jo, ito = O.ifcm_fit(xo, U0o, C0o, lam_xi[p, 0], lam_xi[p, 1], 2.0, 50, 1e-5)
        assert abs(int(its[p]) - ito) <= 1
        assert abs(fit[p] - Jo) <= 1e-4 * abs(Jo)
        # the oracle replaying the run from the GPU's start for the GPU's
        # iteration count meets the parity bars (measured: J 3.1e-8, C 5.9e-8)
        _, Cr, Jr, _ = O.ifcm_fit(xo, U0s, C0s, lam_xi[p, 0], lam_xi[p, 1], 2.0, int(its[p]),
                                  0.0)
        assert abs(fit[p] - Jr) <= J_RTOL * abs(Jr)
        assert np.allclose(cen[p], Cr, rtol=C_RTOL)


def test_resident_equals_stencil_form(G):
    # the same batch through both forms: iteration counts equal at fixed
    # counts, fitness to FP32 rounding of differently grouped sums
    shape = (6, 20, 24)
    x = unit_volume(shape, seed=31)
    U0 = phantoms.random_memberships(shape, 4, seed=32)
    C0 = np.array([0.1, 0.35, 0.6, 0.85])
    lam_xi = np.random.default_rng(33).random((9, 2)) * 0.6
    prm = G.Params(c=4, max_iter=10, eps_u=0.0)
    args = (dev_vol(x), prm, lam_xi, dev_u(U0), C0)
    (f_res, i_res, _), n_res = stencil_launches(G, lambda: G.pso_fitness_batch(*args, nx=24))
    G.resident_enable(False)
    try:
        (f_st, i_st, _), n_st = stencil_launches(G, lambda: G.pso_fitness_batch(*args, nx=24))
    finally:
        G.resident_enable(True)
    assert n_res == 0 and n_st == 10
    assert torch.equal(i_res, i_st)
    assert torch.allclose(f_res, f_st, rtol=2e-6, atol=0)


def test_larger_volumes_keep_the_stencil_kernels(G):
    # one voxel past the bound at c = 4 runs the stencil kernels, same results
    shape = (1, 71, 91)                 # 6461 voxels: (1 + 8) x 4 x 6461 > 225 KB
    assert 9 * 4 * 71 * 91 > SMEM
    x = unit_volume(shape, seed=61)
    U0 = phantoms.random_memberships(shape, 4, seed=62)
    C0 = np.array([0.1, 0.35, 0.6, 0.85])
    lam_xi = np.array([[0.3, 0.2], [0.5, 0.4]])
    prm = G.Params(c=4, max_iter=5, eps_u=0.0)
    (fit, its, _), n_st = stencil_launches(
        G, lambda: G.pso_fitness_batch(dev_vol(x), prm, lam_xi, dev_u(U0), C0, nx=91))
    assert n_st == 5
    fo, io = OP.fitness_batch(x.astype(np.float64), U0.astype(np.float64), C0, lam_xi,
                              max_iter=5, eps=0.0)
    assert np.array_equal(its.cpu().numpy(), io)
    assert np.all(np.abs(fit.cpu().numpy() - fo) <= J_RTOL * np.abs(fo))


def test_multi_volume_batch_matches_oracle(G):
    # small volumes of uneven size and c: one resident launch per c group
    specs = [((1, 30, 30), 4, 5), ((4, 9, 13), 4, 3), ((1, 17, 40), 5, 4), ((3, 8, 8), 6, 2)]
    vols, host = [], []
    for k, (shape, c, P) in enumerate(specs):
        x = unit_volume(shape, seed=70 + k)
        U0 = phantoms.random_memberships(shape, c, seed=80 + k)
        C0 = np.sort(np.random.default_rng(90 + k).random(c))
        lam_xi = np.random.default_rng(100 + k).random((P, 2)) * 0.6
        vols.append(G.BatchVolume(dev_vol(x), c, lam_xi, dev_u(U0), C0, nx=shape[2]))
        host.append((x, U0, C0, lam_xi))
    outs, n_st = stencil_launches(G, lambda: G.pso_fitness_multi(vols, G.Params(max_iter=8,
                                                                                eps_u=0.0)))
    assert n_st == 0
    for (x, U0, C0, lam_xi), (fit, its) in zip(host, outs):
        fo, io = OP.fitness_batch(x.astype(np.float64), U0.astype(np.float64), C0, lam_xi,
                                  max_iter=8, eps=0.0)
        assert np.array_equal(its.cpu().numpy(), io)
        assert np.all(np.abs(fit.cpu().numpy() - fo) <= J_RTOL * np.abs(fo))


def test_pifcm3d_small_run_matches_oracle(G):
    # Algorithm 1 on a 24 x 24 slice: resident FCM start and fitness batches
    raw = phantoms.ellipse_slice(24, seed=1, sigma=0.05)
    prm = G.Params(c=4, max_iter=8, eps_u=0.0)
    opts = G.Options(P=4, generations=3, seed=9, init_max_iter=40)
    (U, res), n_st = stencil_launches(G, lambda: G.pifcm3d(dev_vol(raw), prm, opts, nx=24))
    assert n_st == 0
    ref = OP.pifcm3d(raw, c=4, P=4, generations=3, seed=9, max_iter=8, eps=0.0,
                     init_max_iter=40)
    assert res["status"] == 0
    assert res["lambda"] == ref["lambda"] and res["xi"] == ref["xi"]
    assert res["iters_init"] == 40 and res["iters_final"] == ref["iters"]
    x = O.normalize(raw)
    U0, C0, _, _ = O.fcm_init(x, 4, 2.0, 40, 0.0)
    bound = u_bound(x, U0, C0, ref["lambda"], ref["xi"], 8)
    assert np.max(np.abs(unpad(U, 24) - ref["U"])) <= bound
    assert np.allclose(res["centres"], ref["C"], rtol=1e-5)
    assert abs(res["J"] - ref["J"]) <= J_RTOL * abs(ref["J"])
    assert abs(res["best_fitness"] - ref["pbest_f"].min()) <= J_RTOL * ref["pbest_f"].min()
    assert res["updates"] == 24 * 24 * (40 + 4 * 3 * 8 + 8)


def test_pifcm3d_ellipse_slice_full_workload(G):
    # the 64 x 64 ellipse slice at its workload's full parameters (c = 4,
    # 10 particles x 20 generations, <= 50 iterations, stop max|du| < 1e-5),
    # resident; the final run at the reported (lambda, xi) against the
    # oracle's run there from the oracle's FCM start
    raw = phantoms.ellipse_slice(64, seed=1, sigma=0.05)
    prm = G.Params(c=4, max_iter=50, eps_u=1e-5)
    opts = G.Options(P=10, generations=20, seed=1, init_max_iter=300)
    (U, res), n_st = stencil_launches(G, lambda: G.pifcm3d(dev_vol(raw), prm, opts, nx=64))
    assert n_st == 0
    assert res["status"] == 0
    x = O.normalize(raw)
    U0, C0, _, it0 = O.fcm_init(x, 4, 2.0, 300, 1e-5)
    assert abs(res["iters_init"] - it0) <= 1
    Uo, Co, Jo, ito = O.ifcm_fit(x, U0, C0, res["lambda"], res["xi"], 2.0, 50, 1e-5)
    assert abs(res["iters_final"] - ito) <= 1
    lab = np.mean(np.argmax(unpad(U, 64), 0) == np.argmax(Uo, 0))
    assert lab >= 0.9999
    assert np.allclose(res["centres"], Co, rtol=1e-5, atol=0)
    assert abs(res["J"] - Jo) <= 1e-4 * abs(Jo)
    # the oracle replaying the final run from the GPU's own normalised volume
    # and FCM start, for the GPU's iteration count, meets the parity bars
    # (measured at (lambda, xi) = (1, 1), 50 iterations: U 8.6e-8, C 1.8e-8)
    xg = G.ifcm_normalize(dev_vol(raw), nx=64)
    U0g, C0g, _, it0g = G.ifcm_fit(xg, G.Params(c=4, max_iter=300, eps_u=1e-5), (0.0, 0.0),
                                   nx=64)
    assert it0g == res["iters_init"]
    xs = xg.cpu().numpy()[..., :64].astype(np.float64)
    U0s, C0s = unpad(U0g, 64), C0g.cpu().numpy().astype(np.float64)
    lam, xi, its = res["lambda"], res["xi"], res["iters_final"]
    Ur, Cr, Jr, _ = O.ifcm_fit(xs, U0s, C0s, lam, xi, 2.0, its, 0.0)
    assert np.max(np.abs(unpad(U, 64) - Ur)) <= u_bound(xs, U0s, C0s, lam, xi, its)
    assert np.mean(np.argmax(unpad(U, 64), 0) == np.argmax(Ur, 0)) >= 0.9999
    assert np.allclose(res["centres"], Cr, rtol=C_RTOL, atol=0)
    assert abs(res["J"] - Jr) <= J_RTOL * abs(Jr)


def test_graph_capture_of_a_resident_run(G):
    # pifcm3d captured into one CUDA graph takes the resident form as well
    raw = phantoms.ellipse_slice(32, seed=2, sigma=0.05)
    prm = G.Params(c=4, max_iter=10, eps_u=1e-5)
    opts = G.Options(P=6, generations=4, seed=3, init_max_iter=100)
    U1, r1 = G.pifcm3d(dev_vol(raw), prm, opts, nx=32)
    g = G.pifcm3d_graph(dev_vol(raw), prm, opts, nx=32)
    g.launch()
    r2 = g.result()
    U2 = g.u_out.clone()
    g.close()
    assert r1["lambda"] == r2["lambda"] and r1["xi"] == r2["xi"]
    assert r1["J"] == r2["J"] and r1["iters_final"] == r2["iters_final"]
    assert torch.equal(U1, U2)


def test_slice_mode_runs_resident(G):
    # Algorithm 1 step 1 (one slice of a volume): the slice fits a CTA's shared
    # memory, so its FCM start and fitness batches run resident
    raw = phantoms.brain_phantom((6, 20, 22), seed=8)
    prm = G.Params(c=3, max_iter=5, eps_u=0.0)
    opts = G.Options(P=3, generations=2, seed=4, init_max_iter=30, slice_z=2)
    (U, res), n_st = stencil_launches(G, lambda: G.pifcm3d(dev_vol(raw), prm, opts, nx=22))
    assert n_st == 0
    ref = OP.pifcm3d(raw, c=3, P=3, generations=2, seed=4, max_iter=5, eps=0.0,
                     init_max_iter=30, z=2)
    assert U.shape[1] == 1
    assert res["lambda"] == ref["lambda"] and res["xi"] == ref["xi"]
    x = O.normalize(raw)[2:3]
    U0, C0, _, _ = O.fcm_init(x, 3, 2.0, 30, 0.0)
    bound = u_bound(x, U0, C0, ref["lambda"], ref["xi"], 5)
    assert np.max(np.abs(unpad(U, 22) - ref["U"])) <= bound
    # measured on a GB300: C within 3.4e-8, J within 3.1e-7 (relative)
    assert np.allclose(res["centres"], ref["C"], rtol=C_RTOL)
    assert abs(res["J"] - ref["J"]) <= J_RTOL * abs(ref["J"])


def test_bf16_batches_keep_the_stencil_kernels(G):
    # resident runs hold FP32 memberships only: a bf16 batch of a small volume
    # runs the stencil kernels and stores bf16
    shape = (4, 9, 11)
    x = unit_volume(shape, seed=91)
    U0 = phantoms.random_memberships(shape, 4, seed=92)
    C0 = np.array([0.1, 0.35, 0.6, 0.85])
    lam_xi = np.array([[0.3, 0.2], [0.4, 0.1]])
    prm = G.Params(c=4, max_iter=3, eps_u=0.0, u_dtype="bf16")
    (fit, its, _), n_st = stencil_launches(
        G, lambda: G.pso_fitness_batch(dev_vol(x), prm, lam_xi, dev_u(U0), C0, nx=11))
    assert n_st == 3
    assert np.all(its.cpu().numpy() == 3)

"""Parity at the benchmark's full size (181x217x181, c = 4, 20 particles), in
the launch configuration bench.py times: float2 pair words, two particles per
work item, whole-column z-chunks (tz = 181), 32x11 tiles, 152 persistent CTAs.

The oracle cannot afford 20 whole IFCM runs at this size, so the check uses
one iteration from a shared seeded start (U0, C0).  H and F (Eqs 5-8) depend
only on U0, so the oracle computes them once.  Then:
- every particle's J^0 (Eq 1, a sum over all 7.1 M voxels) and C^1 (Eq 3)
  against the oracle: 1e-5 and 1e-6 relative;
- U^1 of one particle (ifcm_fit) on 20,000 sampled voxels plus every voxel
  of the volume's faces, element by element against the oracle: 1e-5;
- sum_j u_ij = 1 on every voxel (an invariant at any size).

Those two tests start from a seeded random field, so their one iteration runs
the general kernel.  The kernel the bench times, the lean 3D kernel, runs every
iteration whose start comes from Eq 2: a second iteration from the same start
(two particles, and one particle with U on every voxel), and a whole pifcm3d
run of one generation from a two-iteration FCM start.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ifcm as O                     # noqa: E402
from paper_2002_01981_gb300 import phantoms      # noqa: E402

pytestmark = pytest.mark.gpu

SHAPE = (181, 217, 181)
C, P = 4, 20


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_01981_gb300 import build
    build.build()
    from paper_2002_01981_gb300 import ifcm
    return ifcm


@pytest.fixture(scope="module")
def case(G):
    raw = phantoms.brain_phantom(SHAPE, seed=2, sigma=0.07)
    x64 = O.normalize(raw)
    U0 = phantoms.random_memberships(SHAPE, C, seed=17)
    C0 = np.array([0.1, 0.3, 0.6, 0.85])
    lam_xi = G.Swarm(P, seed=2).init().x.cpu().numpy()          # the bench's first swarm
    nz, ny, nx = SHAPE
    pitch = phantoms.pitch_for(nx)
    vol = torch.from_numpy(phantoms.pad_pitch(raw)).cuda()
    x = G.ifcm_normalize(vol, nx=nx)
    u0 = np.zeros((C, nz, ny, pitch), np.float32)
    u0[..., :nx] = U0
    u0 = torch.from_numpy(u0).cuda()
    H, F = O.neighbour_terms(x64, U0.astype(np.float64))           # Eqs 5-8, once
    return dict(x64=x64, U0=U0.astype(np.float64), C0=C0, lam_xi=lam_xi, x=x, u0=u0, H=H, F=F)


def oracle_step(case, lam, xi):
    d2 = O.modified_distance(case["x64"], case["C0"], case["H"], case["F"], lam, xi)
    U1 = O.membership(d2, 2.0)
    return U1, O.objective(U1, d2, 2.0), O.centres(case["x64"], U1, 2.0)


def test_batch_in_the_bench_configuration(G, case):
    np_, tz, _ = G.stencil_plan(G.shape_of(case["x"], SHAPE[2]), C, P)
    assert (np_, tz) == (2, SHAPE[0])                  # the plan bench.py runs
    prm = G.Params(c=C, max_iter=1, eps_u=0.0)
    fit, its, cen = G.pso_fitness_batch(case["x"], prm, case["lam_xi"], case["u0"], case["C0"],
                                        nx=SHAPE[2], want_centres=True)
    fit, cen = fit.cpu().numpy(), cen.cpu().numpy()
    assert np.all(its.cpu().numpy() == 1)
    for p in range(P):
        _, J, C1 = oracle_step(case, *case["lam_xi"][p])
        assert abs(fit[p] - J) <= 1e-5 * abs(J), p
        assert np.allclose(cen[p], C1, rtol=1e-6, atol=0), p


def test_sampled_memberships_of_one_particle(G, case):
    lam, xi = case["lam_xi"][0]
    prm = G.Params(c=C, max_iter=1, eps_u=0.0)
    Ug, _, _, _ = G.ifcm_fit(case["x"], prm, (lam, xi), nx=SHAPE[2], u_init=case["u0"],
                             c_init=case["C0"])
    ug = Ug[..., :SHAPE[2]].cpu().numpy().astype(np.float64)
    U1, _, _ = oracle_step(case, lam, xi)
    nz, ny, nx = SHAPE
    rng = np.random.default_rng(5)
    idx = rng.integers(0, nz * ny * nx, 20000)
    z, r = np.divmod(idx, ny * nx)
    y, xx = np.divmod(r, nx)
    assert np.max(np.abs(ug[:, z, y, xx] - U1[:, z, y, xx])) <= 1e-5
    for sl in [(0,), (nz - 1,), (slice(None), 0), (slice(None), ny - 1),
               (slice(None), slice(None), 0), (slice(None), slice(None), nx - 1)]:
        face = (slice(None),) + sl
        assert np.max(np.abs(ug[face] - U1[face])) <= 1e-5
    assert np.max(np.abs(ug.sum(axis=0) - 1.0)) <= 1e-5


def test_lean_kernel_two_iterations(G, case):
    # the kernel the bench times, stencil3d_kernel, at full size in the bench's
    # plan (two particles per item, whole-column z-chunks): it runs every
    # iteration whose U^t comes from Eq 2, here the second one.  (lambda, xi)
    # away from the clamp of reading R2, so that U is compared everywhere.
    lam_xi = np.array([[0.3, 0.2], [0.45, 0.25]])
    prm = G.Params(c=C, max_iter=2, eps_u=0.0)
    G.profile_read(G.PROF_STENCIL3D)
    G.profile_enable(True)
    try:
        G.force_plan(2, 1)
        try:
            fit, its, cen = G.pso_fitness_batch(case["x"], prm, lam_xi, case["u0"], case["C0"],
                                                nx=SHAPE[2], want_centres=True)
            torch.cuda.synchronize()
        finally:
            G.force_plan(0)
        n3 = G.profile_read(G.PROF_STENCIL3D)[1]
        Ug, Cg, Jg, _ = G.ifcm_fit(case["x"], prm, tuple(lam_xi[0]), nx=SHAPE[2],
                                   u_init=case["u0"], c_init=case["C0"])
        torch.cuda.synchronize()
        n3_fit = G.profile_read(G.PROF_STENCIL3D)[1]
    finally:
        G.profile_enable(False)
    assert n3 == 1 and n3_fit == 1            # iteration 2 of each call ran the lean kernel
    assert np.all(its.cpu().numpy() == 2)
    fit, cen = fit.cpu().numpy(), cen.cpu().numpy()
    x64 = case["x64"]
    for p in range(2):
        lam, xi = lam_xi[p]
        U1, _, C1 = oracle_step(case, lam, xi)
        H, F = O.neighbour_terms(x64, U1)
        d2 = O.modified_distance(x64, C1, H, F, lam, xi)
        U2 = O.membership(d2, 2.0)
        J, C2 = O.objective(U2, d2, 2.0), O.centres(x64, U2, 2.0)
        assert abs(fit[p] - J) <= 1e-5 * abs(J), p
        assert np.allclose(cen[p], C2, rtol=1e-6, atol=0), p
        if p == 0:                            # the one-particle form, every voxel
            ug = Ug[..., :SHAPE[2]].cpu().numpy().astype(np.float64)
            assert np.max(np.abs(ug - U2)) <= 1e-5
            assert np.allclose(Cg.cpu().numpy(), C2, rtol=1e-6, atol=0)
            assert abs(Jg - J) <= 1e-5 * abs(J)


def test_lean_kernel_in_a_whole_run(G, case):
    # what the bench runs: pifcm3d, whose batches start from the FCM start, so
    # every iteration runs stencil3d_kernel -- two particles per item for the
    # 20-particle batch, one for the final run.  One generation, one iteration
    # per fitness, two FCM-start iterations.  The swarm's best lies in the
    # clamp regime (reading R8), where FP32 and FP64 may put a voxel whose Eq 4
    # factor is within rounding of 0 on different sides of the clamp: U is
    # held to 1e-5 on 99.99 % of the voxels (measured: the 99.99th percentile
    # 2.0e-6, the largest 4.2e-4), labels, centres and J to the parity bars
    # (measured: labels all equal, C 2.6e-8, J 1.3e-7).
    assert G.stencil_plan(G.shape_of(case["x"], SHAPE[2]), C, P)[:2] == (2, SHAPE[0])
    raw = phantoms.brain_phantom(SHAPE, seed=2, sigma=0.07)
    vol = torch.from_numpy(phantoms.pad_pitch(raw)).cuda()
    prm = G.Params(c=C, max_iter=1, eps_u=0.0)
    opts = G.Options(P=P, generations=1, seed=2, init_max_iter=2)
    G.profile_read(G.PROF_STENCIL3D)
    G.profile_enable(True)
    try:
        U, res = G.pifcm3d(vol, prm, opts, nx=SHAPE[2])
        torch.cuda.synchronize()
    finally:
        G.profile_enable(False)
    assert G.profile_read(G.PROF_STENCIL3D)[1] == 2      # the batch and the final run
    assert res["status"] == 0 and res["iters_init"] == 2 and res["iters_final"] == 1
    x64 = case["x64"]
    U0, C0, _, _ = O.fcm_init(x64, C, 2.0, 2, 0.0)
    H, F = O.neighbour_terms(x64, U0)
    lam, xi = res["lambda"], res["xi"]
    d2 = O.modified_distance(x64, C0, H, F, lam, xi)
    U1 = O.membership(d2, 2.0)
    J, C1 = O.objective(U1, d2, 2.0), O.centres(x64, U1, 2.0)
    ug = U[..., :SHAPE[2]].cpu().numpy().astype(np.float64)
    assert np.mean(np.argmax(ug, 0) == np.argmax(U1, 0)) >= 0.9999
    assert np.mean(np.abs(ug - U1) <= 1e-5) >= 0.9999
    assert np.max(np.abs(ug.sum(axis=0) - 1.0)) <= 1e-5
    assert np.allclose(res["centres"], C1, rtol=1e-6, atol=0)
    assert abs(res["J"] - J) <= 1e-5 * abs(J)
    # the batch's J of the best particle: the same run on the two-particle kernel
    assert abs(res["best_fitness"] - J) <= 1e-5 * abs(J)

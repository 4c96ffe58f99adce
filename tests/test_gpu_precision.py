"""Membership storage and reduction precision on the GPU (C ABI) against the
FP64 oracle.

BF16 storage (u_dtype "bf16") rounds U^t to bfloat16 once per iteration and
keeps FP32 arithmetic.  Two references:
- the plain FP64 oracle: U within 1e-2 max-abs;
- the FP64 oracle with the same storage model (``oracle.precision.round_bf16``
  applied to U after every iteration): the GPU's FP32 arithmetic differs from
  FP64 by ~1e-6 relative, so the two round the same value differently only
  where it lies that close to a rounding boundary; each such flip is one
  bfloat16 ulp (<= 2^-8 below 1) in that element and perturbs its neighbours'
  H and F by a small fraction of that.  Bound: U within 2^-8 (one ulp below
  1), centres and J within 1e-5 relative, labels >= 99.99 %.
Compensated FP32 sums ("comp32") keep the FP32-path bars: U 1e-5, C 1e-6
relative, J 1e-5 relative.
The batched BF16 forms are compared bit for bit with single runs under the
same forced work decomposition (each particle's lane computes the same IEEE
operations wherever it sits).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ifcm as O                     # noqa: E402
from oracle.precision import round_bf16          # noqa: E402
from paper_2002_01981_gb300 import phantoms      # noqa: E402

pytestmark = pytest.mark.gpu

U_TOL_BF16 = 1e-2          # vs the plain FP64 oracle
U_TOL_MODEL = 2.0 ** -8    # vs the FP64 oracle with bf16 storage
C_RTOL_MODEL = 1e-5
J_RTOL_MODEL = 1e-5
LABELS_MODEL = 0.9999


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_01981_gb300 import build
    build.build()
    from paper_2002_01981_gb300 import ifcm
    yield ifcm
    ifcm.force_plan(0)


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


def labels_agree(Ug, Uo):
    return np.mean(np.argmax(Ug, 0) == np.argmax(Uo, 0))


CASES = [
    # shape (nz, ny, nx), c, m, lambda, xi, iterations, forced np (0: default)
    ((9, 14, 21), 4, 2.0, 0.4, 0.3, 8, 0),
    ((5, 17, 70), 3, 2.0, 0.5, 0.4, 8, 0),     # np = 2, odd c
    ((5, 17, 70), 3, 2.0, 0.5, 0.4, 8, 1),     # np = 1, odd c: padded pair word
    ((40, 9, 33), 4, 2.0, 0.5, 0.3, 6, 1),     # cluster pairs for c = 4
    ((1, 37, 45), 4, 2.0, 0.6, 0.2, 10, 0),    # 2D
    ((6, 11, 13), 5, 2.0, 0.4, 0.4, 8, 0),     # c = 5, np = 1
    ((6, 11, 13), 8, 2.0, 0.3, 0.3, 6, 0),
    ((6, 11, 13), 6, 1.5, 0.4, 0.3, 6, 0),     # general m
    ((1, 1, 1), 2, 2.0, 0.5, 0.5, 3, 0),       # no neighbours
    ((1, 1, 7), 3, 2.0, 0.5, 0.5, 4, 0),       # a line
]


@pytest.mark.parametrize("shape,c,m,lam,xi,iters,np_", CASES)
def test_bf16_run_vs_oracle(G, shape, c, m, lam, xi, iters, np_):
    x = unit_volume(shape, seed=21)
    U = phantoms.random_memberships(shape, c, seed=22)
    C = np.linspace(0.1, 0.9, c)
    G.force_plan(np_, 1)
    try:
        prm = G.Params(c=c, m=m, max_iter=iters, eps_u=0.0, u_dtype="bf16")
        Ug, Cg, Jg, itg = G.ifcm_fit(dev_vol(x), prm, (lam, xi), nx=shape[2],
                                     u_init=dev_u(U), c_init=C)
    finally:
        G.force_plan(0)
    x64, U64 = x.astype(np.float64), U.astype(np.float64)
    Um, Cm, Jm, _ = O.ifcm_fit(x64, U64, C, lam, xi, m, iters, 0.0, store=round_bf16)
    Uo, Co, Jo, _ = O.ifcm_fit(x64, U64, C, lam, xi, m, iters, 0.0)
    u = unpad(Ug, shape[2])
    assert itg == iters
    assert np.array_equal(round_bf16(u), u)              # the stored values are bf16
    assert np.max(np.abs(u - Uo)) <= U_TOL_BF16
    assert np.max(np.abs(u - Um)) <= U_TOL_MODEL
    assert np.allclose(Cg.cpu().numpy(), Cm, rtol=C_RTOL_MODEL, atol=0)
    assert abs(Jg - Jm) <= J_RTOL_MODEL * abs(Jm)
    assert labels_agree(u, Um) >= LABELS_MODEL


def test_bf16_flat_neighbourhoods(G):
    # noise-free piecewise-constant volume: sum_k g_ik = 0 at many voxels
    x = phantoms.piecewise_cube(6, levels=(0.1, 0.5, 0.9), nz=5)
    U = phantoms.random_memberships(x.shape, 3, seed=4)
    C = np.array([0.2, 0.45, 0.8])
    for np_ in (2, 1):
        G.force_plan(np_, 1)
        try:
            prm = G.Params(c=3, max_iter=5, eps_u=0.0, u_dtype="bf16")
            Ug, Cg, Jg, _ = G.ifcm_fit(dev_vol(x), prm, (0.6, 0.5), nx=x.shape[2],
                                       u_init=dev_u(U), c_init=C)
        finally:
            G.force_plan(0)
        Um, Cm, Jm, _ = O.ifcm_fit(x.astype(np.float64), U.astype(np.float64), C, 0.6, 0.5,
                                   2.0, 5, 0.0, store=round_bf16)
        assert np.max(np.abs(unpad(Ug, x.shape[2]) - Um)) <= U_TOL_MODEL
        assert abs(Jg - Jm) <= J_RTOL_MODEL * abs(Jm)


@pytest.mark.parametrize("c,np_,eps", [(4, 2, 2e-3), (3, 2, 2e-3), (4, 1, 2e-3), (5, 2, 1e-2),
                                       (6, 1, 1e-2)])
def test_bf16_batch_equals_single_runs(G, c, np_, eps):
    # odd P (the last pair has one particle) and eps > 0 (particles of a pair
    # stop at different iterations): each particle's fitness and iteration
    # count must equal its run alone, bit for bit, under the same plan
    shape = (12, 23, 40)
    x = dev_vol(unit_volume(shape, seed=31))
    U0 = dev_u(phantoms.random_memberships(shape, c, seed=32))
    C0 = np.linspace(0.15, 0.85, c)
    lam_xi = np.random.default_rng(33).random((5, 2)) * 0.7
    prm = G.Params(c=c, max_iter=25, eps_u=eps, u_dtype="bf16")
    G.force_plan(np_, 2)
    try:
        fit, its, cen = G.pso_fitness_batch(x, prm, lam_xi, U0, C0, nx=shape[2],
                                            want_centres=True)
        fit, its, cen = fit.cpu().numpy(), its.cpu().numpy(), cen.cpu().numpy()
        assert len(set(its.tolist())) > 1, "want particles stopping at different iterations"
        for p in range(5):
            f1, i1, c1 = G.pso_fitness_batch(x, prm, lam_xi[p:p + 1], U0, C0, nx=shape[2],
                                             want_centres=True)
            assert int(i1[0]) == int(its[p])
            assert float(f1[0]) == float(fit[p])
            assert np.array_equal(c1.cpu().numpy()[0], cen[p])
    finally:
        G.force_plan(0)


def test_bf16_multi_equals_per_volume(G):
    vols, specs = [], [((9, 20, 35), 4, 3), ((14, 13, 50), 4, 6), ((7, 30, 21), 5, 4)]
    prm = G.Params(max_iter=12, eps_u=1e-3, u_dtype="bf16")
    for k, (shape, c, P) in enumerate(specs):
        x = dev_vol(unit_volume(shape, seed=40 + k))
        U0 = dev_u(phantoms.random_memberships(shape, c, seed=50 + k))
        C0 = np.linspace(0.1, 0.9, c)
        lx = np.random.default_rng(60 + k).random((P, 2)) * 0.6
        vols.append(G.BatchVolume(x=x, c=c, lam_xi=lx, u0=U0, c0=C0, nx=shape[2]))
    G.force_plan(0)
    outs = G.pso_fitness_multi(vols, prm)
    for v, (fit, its) in zip(vols, outs):
        pv = G.Params(c=v.c, max_iter=12, eps_u=1e-3, u_dtype="bf16")
        f1, i1, _ = G.pso_fitness_batch(v.x, pv, v.lam_xi, v.u0, v.c0, nx=v.nx)
        assert np.array_equal(i1.cpu().numpy(), its.cpu().numpy())
        # the multi-volume launch may cut the volume into other z-chunks (the
        # plan is chosen for the whole launch): FP64 record sums in another order
        assert np.allclose(f1.cpu().numpy(), fit.cpu().numpy(), rtol=1e-9, atol=0)


@pytest.mark.parametrize("shape,c,lam,xi", [((9, 14, 21), 4, 0.4, 0.3),
                                            ((20, 30, 41), 6, 0.5, 0.2),
                                            ((1, 37, 45), 3, 0.6, 0.2)])
def test_comp32_reduction_vs_oracle(G, shape, c, lam, xi):
    x = unit_volume(shape, seed=71)
    U = phantoms.random_memberships(shape, c, seed=72)
    C = np.linspace(0.1, 0.9, c)
    prm = G.Params(c=c, max_iter=8, eps_u=0.0, reduce="comp32")
    Ug, Cg, Jg, _ = G.ifcm_fit(dev_vol(x), prm, (lam, xi), nx=shape[2], u_init=dev_u(U),
                               c_init=C)
    Uo, Co, Jo, _ = O.ifcm_fit(x.astype(np.float64), U.astype(np.float64), C, lam, xi, 2.0, 8,
                               0.0)
    assert np.max(np.abs(unpad(Ug, shape[2]) - Uo)) <= 1e-5
    assert np.allclose(Cg.cpu().numpy(), Co, rtol=1e-6, atol=0)
    assert abs(Jg - Jo) <= 1e-5 * abs(Jo)


def test_bf16_whole_algorithm(G):
    raw = phantoms.brain_phantom((10, 24, 30), seed=81, sigma=0.06)
    vol = dev_vol(raw)
    opts = G.Options(P=6, generations=3, seed=9, init_max_iter=60)
    U32, r32 = G.pifcm3d(vol, G.Params(c=4, max_iter=20), opts, nx=30)
    U16, r16 = G.pifcm3d(vol, G.Params(c=4, max_iter=20, u_dtype="bf16", reduce="comp32"),
                         opts, nx=30)
    assert r16["status"] == 0 and r16["updates"] > 0
    u16, u32 = unpad(U16, 30), unpad(U32, 30)
    assert np.allclose(u16.sum(0), 1.0, atol=2e-2)
    assert np.array_equal(round_bf16(u16), u16)
    # each run reaches its own best (lambda, xi); the segmentations still agree
    assert labels_agree(u16, u32) >= 0.99


def test_plain_form_rejects_bf16(G):
    from paper_2002_01981_gb300.native import IfcmError
    x = dev_vol(unit_volume((4, 5, 6), seed=1))
    with pytest.raises(IfcmError):
        G.ifcm_fit(x, G.Params(c=3, max_iter=2, u_dtype="bf16"), (0.2, 0.2), nx=6, plain=True)


def test_c6_workload_slab_vs_oracle(G):
    """16 planes of the 256^3 six-class workload (Rician sigma 0.1), each side
    from its own FCM start (30 iterations), then 10 IFCM iterations at
    (0.4, 0.3): FP32 at the FP32 bars; bf16 storage (FP64 or compensated FP32
    sums) at the bf16 bars against the plain FP64 oracle."""
    raw = phantoms.multi_tissue((256, 256, 256), seed=5, sigma=0.1)[120:136].copy()
    nz, ny, nx = raw.shape
    c, lam, xi = 6, 0.4, 0.3
    xo = O.normalize(raw)
    U0o, C0o, _, _ = O.fcm_init(xo, c, max_iter=30, eps=0.0)
    Uo, Co, Jo, _ = O.ifcm_fit(xo, U0o, C0o, lam, xi, 2.0, 10, 0.0)
    x = G.ifcm_normalize(dev_vol(raw), nx=nx)
    U0, C0, _, _ = G.ifcm_fit(x, G.Params(c=c, max_iter=30, eps_u=0.0), (0.0, 0.0), nx=nx)
    for d, r, utol, ctol, jtol, lab in [("fp32", "fp64", 1e-5, 1e-6, 1e-5, 0.9999),
                                        ("fp32", "comp32", 1e-5, 1e-6, 1e-5, 0.9999),
                                        ("bf16", "fp64", 1e-2, 1e-4, 1e-3, 0.999),
                                        ("bf16", "comp32", 1e-2, 1e-4, 1e-3, 0.999)]:
        prm = G.Params(c=c, max_iter=10, eps_u=0.0, u_dtype=d, reduce=r)
        Ug, Cg, Jg, _ = G.ifcm_fit(x, prm, (lam, xi), nx=nx, u_init=U0, c_init=C0)
        u = unpad(Ug, nx)
        eu = np.max(np.abs(u - Uo))
        ec = np.max(np.abs(Cg.cpu().numpy() / Co - 1.0))
        ej = abs(Jg / Jo - 1.0)
        la = labels_agree(u, Uo)
        print(f"c6 slab {d}/{r}: U {eu:.2e} C {ec:.2e} J {ej:.2e} labels {la:.6f}")
        assert eu <= utol and ec <= ctol and ej <= jtol and la >= lab, (d, r, eu, ec, ej, la)

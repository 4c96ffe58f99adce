"""dJ^{K-1}/d(lambda, xi) on the GPU (C ABI: ifcm_grad, ifcm_polish) against
the FP64 oracle adjoint, and the autograd wrapper.

Tolerance: 1e-5 relative on each derivative and on J (FP32 forward and reverse
passes against FP64, K up to 20; measured on a GB300 within 5.8e-7 and 1.7e-7).  Starts are seeded random
memberships from the shared input generator, so both sides begin from the
same (U^0, C^0).  Points are chosen with 1 - lambda H - xi F > 0 almost
everywhere (lambda + xi < 1), away from the clamp of reading R2 whose kink
would make the derivative jump.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint as A                  # noqa: E402
from oracle import ifcm as O                     # noqa: E402
from paper_2002_01981_gb300 import phantoms      # noqa: E402

pytestmark = pytest.mark.gpu

G_RTOL = 1e-5
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
    return torch.from_numpy(phantoms.pad_pitch(np.asarray(a, np.float32))).cuda()


def dev_u(u):
    c, nz, ny, nx = u.shape
    out = np.zeros((c, nz, ny, phantoms.pitch_for(nx)), np.float32)
    out[..., :nx] = u
    return torch.from_numpy(out).cuda()


def unit_volume(shape, seed, sigma=0.06):
    raw = phantoms.brain_phantom(shape, seed=seed, sigma=sigma)
    return np.clip(raw, 0.0, 1.0).astype(np.float32)


CASES = [
    # shape (nz, ny, nx), c, m, lambda, xi, K
    ((9, 14, 21), 4, 2.0, 0.4, 0.3, 5),
    ((20, 37, 70), 4, 2.0, 0.3, 0.25, 8),     # several tiles, ragged tails
    ((5, 17, 40), 3, 2.0, 0.5, 0.2, 6),
    ((1, 37, 45), 4, 2.0, 0.35, 0.3, 8),      # 2D
    ((6, 11, 13), 6, 2.0, 0.3, 0.3, 4),
    ((6, 11, 13), 5, 1.5, 0.3, 0.2, 4),       # general m
    ((4, 10, 12), 3, 3.0, 0.2, 0.4, 4),
    ((7, 12, 10), 2, 2.0, 0.0, 0.0, 5),       # at plain FCM
    ((1, 1, 9), 3, 2.0, 0.4, 0.3, 3),         # a line
    ((2, 2, 2), 8, 2.0, 0.3, 0.3, 2),
]


@pytest.mark.parametrize("shape,c,m,lam,xi,K", CASES)
def test_gradient_matches_oracle_adjoint(G, shape, c, m, lam, xi, K):
    x = unit_volume(shape, seed=91)
    U0 = phantoms.random_memberships(shape, c, seed=92)
    C0 = np.linspace(0.1, 0.9, c)
    J, g = G.ifcm_grad(dev_vol(x), G.Params(c=c, m=m), (lam, xi), dev_u(U0), C0, K,
                       nx=shape[2])
    Jo, glo, gxo = A.ifcm_grad(x.astype(np.float64), U0.astype(np.float64), C0, lam, xi, m, K)
    g = g.cpu().numpy()
    assert abs(float(J) - Jo) <= J_RTOL * abs(Jo)
    scale = max(abs(glo), abs(gxo))          # both derivatives share J's scale
    assert abs(g[0] - glo) <= G_RTOL * max(abs(glo), 1e-3 * scale)
    assert abs(g[1] - gxo) <= G_RTOL * max(abs(gxo), 1e-3 * scale)


def test_flat_neighbourhoods(G):
    lv = np.array([0.2, 0.2, 0.2, 0.55, 0.55, 0.55, 0.9, 0.9])
    x = np.repeat(lv[:, None, None], 6 * 7, axis=1).reshape(8, 6, 7)
    x[:, :, 4:] += 0.05 * np.random.default_rng(14).standard_normal((8, 6, 3))
    x = np.clip(x, 0.0, 1.0).astype(np.float32)
    U0 = phantoms.random_memberships(x.shape, 2, seed=9)
    C0 = np.array([0.3, 0.7])
    J, g = G.ifcm_grad(dev_vol(x), G.Params(c=2), (0.4, 0.3), dev_u(U0), C0, 3, nx=7)
    Jo, glo, gxo = A.ifcm_grad(x.astype(np.float64), U0.astype(np.float64), C0, 0.4, 0.3,
                               2.0, 3)
    g = g.cpu().numpy()
    assert g[0] == pytest.approx(glo, rel=G_RTOL)
    assert g[1] == pytest.approx(gxo, rel=G_RTOL)


def test_twenty_unrolled_iterations(G):
    # the differentiation workload's shape (Gaussian sigma 0.09, c = 4, K = 20)
    # on a 48^3 piece
    x = np.clip(phantoms.gaussian_phantom((48, 48, 48), seed=4, sigma=0.09), 0, 1)
    U0 = phantoms.random_memberships(x.shape, 4, seed=5)
    C0 = np.array([0.1, 0.3, 0.55, 0.85])
    J, g = G.ifcm_grad(dev_vol(x), G.Params(c=4), (0.3, 0.2), dev_u(U0), C0, 20, nx=48)
    Jo, glo, gxo = A.ifcm_grad(x.astype(np.float64), U0.astype(np.float64), C0, 0.3, 0.2, 2.0,
                               20)
    g = g.cpu().numpy()
    assert float(J) == pytest.approx(Jo, rel=J_RTOL)
    assert g[0] == pytest.approx(glo, rel=G_RTOL)
    assert g[1] == pytest.approx(gxo, rel=G_RTOL)


def test_central_differences_of_the_gpu_forward(G):
    # FP32 forward: J carries ~1e-7 relative rounding, so with h = 1e-3 the
    # central difference is good to ~1e-3 relative
    shape = (10, 20, 30)
    x = dev_vol(unit_volume(shape, seed=93))
    U0 = dev_u(phantoms.random_memberships(shape, 4, seed=94))
    C0 = np.linspace(0.1, 0.9, 4)
    prm = G.Params(c=4)
    _, g = G.ifcm_grad(x, prm, (0.35, 0.25), U0, C0, 6, nx=shape[2])
    f = lambda a, b: float(G.ifcm_grad(x, prm, (a, b), U0, C0, 6, nx=shape[2])[0])  # noqa
    h = 1e-3
    fl = (f(0.35 + h, 0.25) - f(0.35 - h, 0.25)) / (2 * h)
    fx = (f(0.35, 0.25 + h) - f(0.35, 0.25 - h)) / (2 * h)
    g = g.cpu().numpy()
    assert g[0] == pytest.approx(fl, rel=1e-2)
    assert g[1] == pytest.approx(fx, rel=1e-2)


def test_autograd_function(G):
    shape = (8, 12, 16)
    x = dev_vol(unit_volume(shape, seed=95))
    U0 = dev_u(phantoms.random_memberships(shape, 3, seed=96))
    C0 = torch.tensor([0.2, 0.5, 0.8], dtype=torch.float64, device="cuda")
    lx = torch.tensor([0.3, 0.2], dtype=torch.float64, device="cuda", requires_grad=True)
    prm = G.Params(c=3)
    J = G.IFCMObjective.apply(lx, x, U0, C0, prm, 4, shape[2])
    (2.5 * J).backward()
    _, g = G.ifcm_grad(x, prm, lx.detach(), U0, C0, 4, nx=shape[2])
    assert torch.equal(lx.grad, 2.5 * g)


def test_polish_follows_the_oracle_rule(G):
    # the same projected, normalised descent rule driven by the oracle's
    # gradient: the GPU path visits the same points (directions agree to
    # ~1e-5) and returns the best
    shape = (6, 12, 14)
    x = unit_volume(shape, seed=97)
    U0 = phantoms.random_memberships(shape, 3, seed=98)
    C0 = np.array([0.2, 0.5, 0.8])
    K, steps, a0, dec = 4, 5, 0.05, 0.7
    lx, Jbest = G.ifcm_polish(dev_vol(x), G.Params(c=3), (0.2, 0.1), dev_u(U0), C0, K,
                              steps=steps, step0=a0, decay=dec, nx=shape[2])
    x64, U64 = x.astype(np.float64), U0.astype(np.float64)
    cur = np.array([0.2, 0.1])
    best, bestJ = cur.copy(), np.inf
    alpha = a0
    for _ in range(steps):
        J, gl, gx = A.ifcm_grad(x64, U64, C0, cur[0], cur[1], 2.0, K)
        if J < bestJ:
            best, bestJ = cur.copy(), J
        g = np.array([gl, gx])
        cur = np.clip(cur - alpha * g / np.linalg.norm(g), 0.0, 1.0)
        alpha *= dec
    J = O.ifcm_fit(x64, U64, C0, cur[0], cur[1], 2.0, K, 0.0)[2]
    if J < bestJ:
        best, bestJ = cur.copy(), J
    assert np.allclose(lx.cpu().numpy(), best, atol=1e-5)
    assert Jbest == pytest.approx(bestJ, rel=J_RTOL)
    J0 = O.ifcm_fit(x64, U64, C0, 0.2, 0.1, 2.0, K, 0.0)[2]
    assert bestJ <= J0


def test_gradient_rejects_bf16(G):
    from paper_2002_01981_gb300.native import IfcmError
    x = dev_vol(unit_volume((4, 5, 6), seed=1))
    U0 = dev_u(phantoms.random_memberships((4, 5, 6), 3, seed=2))
    with pytest.raises(IfcmError):
        G.ifcm_grad(x, G.Params(c=3, u_dtype="bf16"), (0.2, 0.2), U0, [0.2, 0.5, 0.8], 2, nx=6)

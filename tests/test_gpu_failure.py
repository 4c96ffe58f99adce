"""Failure detection on the GPU without a fault: every wait of the stencil
kernels on their shared-memory tiles is bounded.  A bound of 1 ns makes the
waits run out on purpose; the kernels must record IFCM_ERR_TIMEOUT in the
workspace's status word, wait for their own copies in flight, and return, so
that the call returns normally and the GPU context stays usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2002_01981_gb300 import phantoms  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_01981_gb300 import build
    build.build()
    from paper_2002_01981_gb300 import ifcm
    return ifcm


def _inputs(shape, c, P, seed):
    raw = np.clip(phantoms.brain_phantom(shape, seed=seed, sigma=0.06), 0.0, 1.0)
    x = torch.from_numpy(phantoms.pad_pitch(raw.astype(np.float32))).cuda()
    nz, ny, nx = shape
    U = phantoms.random_memberships(shape, c, seed=seed + 1)
    u0 = np.zeros((c, nz, ny, phantoms.pitch_for(nx)), np.float32)
    u0[..., :nx] = U
    lam_xi = np.random.default_rng(seed + 2).random((P, 2)) * 0.6
    return x, torch.from_numpy(u0).cuda(), np.linspace(0.15, 0.85, c), lam_xi, nx


# Every CTA must wait for some tile before it has landed: the volumes have more
# planes (tiles down a 2D image) per CTA than the ring holds, so the producer
# waits for stages to be released.
@pytest.mark.parametrize("shape,c,P", [((24, 40, 48), 4, 6),    # both 3D kernels
                                       ((1, 300, 70), 4, 3),    # the 2D kernel
                                       ((12, 20, 36), 3, 1)])   # one particle
def test_wait_that_runs_out_reports_timeout(G, shape, c, P):
    from paper_2002_01981_gb300.native import IfcmError
    x, u0, c0, lam_xi, nx = _inputs(shape, c, P, seed=41)
    prm = G.Params(c=c, max_iter=4, eps_u=0.0)
    G.force_plan(2 if P > 1 else 1, 1)       # whole columns: many planes per item
    try:
        ref, ref_it, _ = G.pso_fitness_batch(x, prm, lam_xi, u0, c0, nx=nx)
        G.set_wait_limit_ns(1)
        with pytest.raises(IfcmError) as err:
            G.pso_fitness_batch(x, prm, lam_xi, u0, c0, nx=nx)
        assert err.value.status == 4          # IFCM_ERR_TIMEOUT
    finally:
        G.set_wait_limit_ns(0)
        G.force_plan(0)
    torch.cuda.synchronize()
    # the context is usable and the same call gives the same results again
    G.force_plan(2 if P > 1 else 1, 1)
    try:
        fit, its, _ = G.pso_fitness_batch(x, prm, lam_xi, u0, c0, nx=nx)
    finally:
        G.force_plan(0)
    assert torch.equal(fit, ref) and torch.equal(its, ref_it)

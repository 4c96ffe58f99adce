"""ifcm_fit_noalloc: the IFCM run for callers that cannot allocate device
memory (graph capture in global mode, plugins whose host owns every
allocation).  It runs exactly the launches of ifcm_fit, which takes a caller
workspace, so it must give bit-identical results, on consecutive calls that
share the library's static scratch, whatever an earlier call of another
shape left there.  Its device-side failures are reported by
ifcm_fit_noalloc_status.

This file is collected last so that a run stopping at its first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2002_01981_gb300 import phantoms  # noqa: E402

def _lib():
    from paper_2002_01981_gb300 import build, native
    build.build()
    return native.load()


def _call_noalloc(lib, x, nx, prm, lam_xi, u_init, c_init):
    from paper_2002_01981_gb300 import ifcm as G
    from paper_2002_01981_gb300 import native as N
    dev = x.device
    c = prm.c
    u_out = torch.empty((c,) + tuple(x.shape), dtype=torch.float32, device=dev)
    c_out = torch.empty(c, dtype=torch.float64, device=dev)
    J_out = torch.empty(1, dtype=torch.float64, device=dev)
    it_out = torch.empty(1, dtype=torch.int32, device=dev)
    p = prm.native()
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    st = lib.ifcm_fit_noalloc(ptr(x), G.shape_of(x, nx), ctypes.byref(p), ptr(lam_xi),
                              ptr(u_init), ptr(c_init), ptr(u_out), ptr(c_out), ptr(J_out),
                              ptr(it_out), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    N.check(st)
    torch.cuda.synchronize()
    return u_out, c_out, float(J_out.item()), int(it_out.item())


def _volume(shape, seed):
    raw = np.clip(phantoms.brain_phantom(shape, seed=seed, sigma=0.06), 0, 1).astype(np.float32)
    return torch.from_numpy(phantoms.pad_pitch(raw)).cuda()


@pytest.mark.gpu
def test_noalloc_matches_ifcm_fit_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = _lib()
    from paper_2002_01981_gb300 import ifcm as G
    from paper_2002_01981_gb300 import native as N
    shape = (11, 23, 37)
    x = _volume(shape, 61)
    U = torch.from_numpy(phantoms.random_memberships(shape, 4, seed=62,
                                                     padded_pitch=x.shape[2])).cuda()
    C = torch.tensor([0.1, 0.35, 0.6, 0.85], dtype=torch.float64, device="cuda")
    shape3 = (7, 41, 29)      # another shape and c, after the first two
    x3 = _volume(shape3, 63)
    # call 1: a given start; call 2: the uniform start, other (lambda, xi) and
    # a stop threshold, over whatever call 1 left in the shared scratch; call
    # 3: another layout of the scratch (shape, c = 5)
    cases = [(x, 37, G.Params(c=4, max_iter=15, eps_u=0.0), (0.5, 0.4), U, C),
             (x, 37, G.Params(c=4, max_iter=40, eps_u=1e-5), (0.3, 0.6), None, None),
             (x3, 29, G.Params(c=5, max_iter=20, eps_u=1e-5), (0.6, 0.2), None, None)]
    for xv, nx, prm, lx, u0, c0 in cases:
        lam_xi = torch.tensor(lx, dtype=torch.float64, device="cuda")
        Ur, Cr, Jr, itr = G.ifcm_fit(xv, prm, lam_xi, nx=nx, u_init=u0, c_init=c0)
        Un, Cn, Jn, itn = _call_noalloc(lib, xv, nx, prm, lam_xi, u0, c0)
        N.check(lib.ifcm_fit_noalloc_status(
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
        # the same launches on the same inputs: bit-identical results
        assert itn == itr
        assert torch.equal(Un[..., :nx], Ur[..., :nx])
        assert torch.equal(Cn, Cr)
        assert Jn == Jr


@pytest.mark.gpu
def test_noalloc_reports_device_failures():
    # a bounded wait that runs out (see ifcm_set_wait_limit_ns) is recorded in
    # the status word at the start of the static scratch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = _lib()
    from paper_2002_01981_gb300 import ifcm as G
    shape = (11, 23, 37)
    x = _volume(shape, 61)
    prm = G.Params(c=4, max_iter=5, eps_u=0.0)
    lam_xi = torch.tensor((0.5, 0.4), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    G.force_plan(1, 1)             # whole columns: more planes per item than the ring holds
    try:
        G.set_wait_limit_ns(1)
        _call_noalloc(lib, x, 37, prm, lam_xi, None, None)
        assert lib.ifcm_fit_noalloc_status(stream) == 4      # IFCM_ERR_TIMEOUT
    finally:
        G.set_wait_limit_ns(0)
        G.force_plan(0)
    # the next call clears the status and works
    Ur, _, Jr, _ = G.ifcm_fit(x, prm, lam_xi, nx=37)
    Un, _, Jn, _ = _call_noalloc(lib, x, 37, prm, lam_xi, None, None)
    assert lib.ifcm_fit_noalloc_status(stream) == 0
    assert torch.equal(Un[..., :37], Ur[..., :37]) and Jn == Jr


def test_noalloc_rejects_volumes_beyond_its_scratch():
    # refused on the host, before any device work: no GPU needed
    lib = _lib()
    from paper_2002_01981_gb300 import native as N
    shp = N.IfcmShape(112, 112, 112, 112)
    p = N.IfcmParams(4, 2.0, 1, 1.0, 50, 1e-5, 1e-12)
    fake = ctypes.c_void_p(256)
    st = lib.ifcm_fit_noalloc(fake, shp, ctypes.byref(p), fake, None, None, None, None, None,
                              None, None)
    assert st == 2          # IFCM_ERR_NOMEM
    msg = lib.ifcm_last_error().decode()
    assert "64 MiB" in msg and str(lib.ifcm_fit_workspace_bytes(shp, ctypes.byref(p))) in msg

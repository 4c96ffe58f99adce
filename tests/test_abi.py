"""The C ABI library loads, exports every symbol include/pifcm.h declares, and
rejects bad arguments on the host before any CUDA call (no GPU needed)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_2002_01981_gb300 import build, native
    build.build()
    return native.load()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "pifcm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


def test_header_declares_the_path_entry_points():
    names = _declared_functions()
    for n in ("ifcm_fit", "pso_fitness_batch", "pso_step", "pso_init", "ifcm_normalize",
              "pifcm3d", "pifcm3d_host"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2002_01981_gb300 import native
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in native.SIGNATURES, name


def test_struct_sizes_match_the_header_layout():
    from paper_2002_01981_gb300 import native as N
    assert ctypes.sizeof(N.IfcmShape) == 16
    assert ctypes.sizeof(N.IfcmParams) == 64
    assert ctypes.sizeof(N.PsoState) == 64
    assert ctypes.sizeof(N.PifcmOptions) == 48
    assert ctypes.sizeof(N.PifcmResult) == 8 * 8 + 4 * 8 + 8 + 4 * 4


def _params(**kw):
    from paper_2002_01981_gb300 import native as N
    d = dict(c=4, m=2.0, V=1, h=1.0, max_iter=50, eps_u=1e-5, dist_floor=1e-12, u_dtype=0,
             reduce=0)
    d.update(kw)
    return N.IfcmParams(d["c"], d["m"], d["V"], d["h"], d["max_iter"], d["eps_u"],
                        d["dist_floor"], d["u_dtype"], d["reduce"])


@pytest.mark.parametrize("shape,ok", [((181, 217, 181, 184), True), ((5, 1, 1, 8), True),
                                      ((5, 4, 3, 6), False), ((0, 4, 3, 4), False),
                                      ((5, 4, 3, 4), False), ((5, 4, -1, 8), False)])
def test_shape_validation(lib, shape, ok):
    from paper_2002_01981_gb300 import native as N
    nx, ny, nz, pitch = shape
    shp = N.IfcmShape(nx, ny, nz, pitch)
    fake = ctypes.c_void_p(256)          # never dereferenced: checks fail first
    st = lib.ifcm_normalize(fake, fake, shp, fake, 0, None)
    if ok:
        assert st == 2          # passes the checks, then: workspace of 0 bytes
    else:
        assert st == 1
        assert lib.ifcm_last_error()


@pytest.mark.parametrize("kw,status", [(dict(c=1), 1), (dict(c=9), 1), (dict(m=1.0), 1),
                                       (dict(m=float("nan")), 1), (dict(V=5), 6),
                                       (dict(V=0), 6), (dict(V=2, h=0.0), 1),
                                       (dict(V=2, u_dtype=1), 6),
                                       (dict(max_iter=0), 1), (dict(eps_u=-1.0), 1),
                                       (dict(dist_floor=0.0), 1), (dict(u_dtype=2), 1),
                                       (dict(u_dtype=-1), 1), (dict(reduce=2), 1)])
def test_parameter_validation(lib, kw, status):
    from paper_2002_01981_gb300 import native as N
    shp = N.IfcmShape(8, 8, 8, 8)
    p = _params(**kw)
    fake = ctypes.c_void_p(256)
    st = lib.ifcm_fit(fake, shp, ctypes.byref(p), fake, None, None, None, None, None, None,
                      fake, 1 << 40, None)
    assert st == status


def test_misaligned_and_null_pointers(lib):
    from paper_2002_01981_gb300 import native as N
    shp = N.IfcmShape(8, 8, 8, 8)
    p = _params()
    st = lib.ifcm_fit(ctypes.c_void_p(260), shp, ctypes.byref(p), ctypes.c_void_p(256), None,
                      None, None, None, None, None, ctypes.c_void_p(256), 1 << 40, None)
    assert st == 1 and b"aligned" in lib.ifcm_last_error()
    st = lib.pso_fitness_batch(ctypes.c_void_p(256), shp, ctypes.byref(p), None, 4,
                               ctypes.c_void_p(256), None, None, None, None,
                               ctypes.c_void_p(256), 1 << 40, None)
    assert st == 1
    st = lib.pso_fitness_batch(ctypes.c_void_p(256), shp, ctypes.byref(p), ctypes.c_void_p(256),
                               0, ctypes.c_void_p(256), ctypes.c_void_p(256),
                               ctypes.c_void_p(256), None, None, ctypes.c_void_p(256), 1 << 40,
                               None)
    assert st == 1


def test_swarm_validation(lib):
    from paper_2002_01981_gb300 import native as N
    s = N.PsoState(0, 1, 0.2, 1, 256, 256, 256, 256, 256)
    assert lib.pso_init(ctypes.byref(s), None) == 1
    s = N.PsoState(4, 1, 0.0, 1, 256, 256, 256, 256, 256)
    assert lib.pso_step(ctypes.byref(s), ctypes.c_void_p(256), None) == 1
    s = N.PsoState(4, -1, 0.2, 1, 256, 256, 256, 256, 256)
    assert lib.pso_init(ctypes.byref(s), None) == 1
    s = N.PsoState(2000, 1, 0.2, 1, 256, 256, 256, 256, 256)
    assert lib.pso_init(ctypes.byref(s), None) == 1


def test_workspace_sizes_scale_with_the_batch(lib):
    from paper_2002_01981_gb300 import native as N
    shp = N.IfcmShape(181, 217, 181, 184)
    p = _params()
    one = lib.pso_fitness_batch_workspace_bytes(shp, ctypes.byref(p), 1)
    twenty = lib.pso_fitness_batch_workspace_bytes(shp, ctypes.byref(p), 20)
    plane = 184 * 217 * 181 * 4
    # two membership buffers of c planes per particle dominate
    assert twenty - one >= 19 * 2 * 4 * plane
    assert twenty < 21 * (2 * 4 * plane) + (1 << 26)
    o = N.PifcmOptions(20, 30, 1, 0.2, 1, 300, -1)
    full = lib.pifcm3d_workspace_bytes(shp, ctypes.byref(p), ctypes.byref(o))
    assert full >= twenty
    host = lib.pifcm3d_host_workspace_bytes(shp, ctypes.byref(p), ctypes.byref(o))
    assert host >= full + 5 * plane
    assert lib.ifcm_fit_workspace_bytes(shp, ctypes.byref(_params(c=9))) == 0


def test_options_validation(lib):
    from paper_2002_01981_gb300 import native as N
    shp = N.IfcmShape(8, 8, 8, 8)
    p = _params()
    fake = ctypes.c_void_p(256)
    for o in (N.PifcmOptions(0, 3, 1, 0.2, 1, 300, -1), N.PifcmOptions(4, 0, 1, 0.2, 1, 300, -1),
              N.PifcmOptions(4, 3, 1, 0.2, 1, 300, 8), N.PifcmOptions(4, 3, 1, -0.2, 1, 300, -1),
              N.PifcmOptions(4, 3, 1, 0.2, 1, 300, -1, 2)):
        assert lib.pifcm3d(fake, shp, ctypes.byref(p), ctypes.byref(o), None, fake, fake,
                           1 << 40, None) == 1


def test_status_strings(lib):
    for s in range(7):
        assert lib.ifcm_status_string(s)


def _batch_volumes(specs):
    """Descriptors with fake (aligned, never dereferenced) device pointers."""
    from paper_2002_01981_gb300 import native as N
    arr = (N.IfcmBatchVolume * len(specs))()
    for i, (shape, c, P) in enumerate(specs):
        arr[i] = N.IfcmBatchVolume(256, N.IfcmShape(*shape), c, P, 256, 256, 256, 256, 0)
    return arr


def test_multi_volume_layout_and_validation(lib):
    from paper_2002_01981_gb300 import native as N
    assert ctypes.sizeof(N.IfcmBatchVolume) == 8 + 16 + 4 + 4 + 5 * 8
    p = _params()
    fake = ctypes.c_void_p(256)
    ok = _batch_volumes([((20, 16, 12, 20), 3, 4)])
    assert lib.pso_fitness_multi(ok, 0, ctypes.byref(p), fake, 1 << 40, None) == 1
    for bad in ([((20, 16, 12, 20), 9, 4)], [((20, 16, 12, 20), 3, 0)],
                [((20, 16, 12, 18), 3, 4)], [((20, 16, 12, 20), 3, 5000)]):
        assert lib.pso_fitness_multi(_batch_volumes(bad), 1, ctypes.byref(p), fake, 1 << 40,
                                     None) == 1
        assert lib.pso_fitness_multi_workspace_bytes(_batch_volumes(bad), 1, ctypes.byref(p)) == 0
    # a workspace below what the largest volume needs alone is refused before any launch
    need = lib.pso_fitness_multi_min_workspace_bytes(ok, 1, ctypes.byref(p))
    assert need > 0
    assert lib.pso_fitness_multi(ok, 1, ctypes.byref(p), fake, need - 256, None) == 2


def test_multi_volume_workspace_is_the_largest_wave(lib):
    from paper_2002_01981_gb300 import native as N
    p = _params()
    a = ((40, 32, 24, 40), 3, 6)
    b = ((24, 24, 24, 24), 3, 5)
    d = ((64, 48, 40, 64), 5, 2)
    one = lambda s: lib.pso_fitness_multi_workspace_bytes(_batch_volumes([s]), 1, ctypes.byref(p))
    both = lib.pso_fitness_multi_workspace_bytes(_batch_volumes([a, b]), 2, ctypes.byref(p))
    # volumes of one c share a wave: their buffers add up
    assert both >= one(a) + one(b) - (1 << 16)
    mixed = _batch_volumes([a, d, b])
    # groups of different c run one after the other in the same workspace
    full = lib.pso_fitness_multi_workspace_bytes(mixed, 3, ctypes.byref(p))
    assert full == max(both, one(d))
    lo = lib.pso_fitness_multi_min_workspace_bytes(mixed, 3, ctypes.byref(p))
    assert lo == max(one(a), one(b), one(d))
    # one volume needs what the single-volume batch entry needs, give or take
    # the alignment slack
    shp = N.IfcmShape(*a[0])
    pc = _params(c=3)
    single = lib.pso_fitness_batch_workspace_bytes(shp, ctypes.byref(pc), 6)
    assert abs(one(a) - single) <= 4096


def test_stencil_plan_rule_and_forcing(lib):
    from paper_2002_01981_gb300 import native as N
    npp, tz = ctypes.c_int32(), ctypes.c_int32()
    shp = N.IfcmShape(181, 217, 181, 184)
    assert lib.ifcm_stencil_plan(shp, 4, 20, ctypes.byref(npp), ctypes.byref(tz)) == 0
    assert npp.value == 2 and 8 <= tz.value <= 181
    assert lib.ifcm_stencil_plan(shp, 5, 20, ctypes.byref(npp), ctypes.byref(tz)) == 0
    assert npp.value == 2
    assert lib.ifcm_stencil_plan(shp, 6, 20, ctypes.byref(npp), ctypes.byref(tz)) == 0
    assert npp.value == 1
    assert lib.ifcm_stencil_plan(shp, 9, 20, ctypes.byref(npp), ctypes.byref(tz)) == -1
    assert lib.ifcm_stencil_plan(N.IfcmShape(5, 4, 3, 6), 4, 20, None, None) == -1
    # forcing: chunks are clamped to >= 8 planes; np = 2 is ignored above c = 5
    assert lib.ifcm_stencil_force_plan(3, 1) == 1
    assert lib.ifcm_stencil_force_plan(1, 0) == 1
    assert lib.ifcm_stencil_force_plan(1, 100) == 0
    lib.ifcm_stencil_plan(shp, 4, 20, ctypes.byref(npp), ctypes.byref(tz))
    assert (npp.value, tz.value) == (1, 8)
    assert lib.ifcm_stencil_force_plan(2, 4) == 0
    lib.ifcm_stencil_plan(shp, 4, 20, ctypes.byref(npp), ctypes.byref(tz))
    assert (npp.value, tz.value) == (2, 46)
    lib.ifcm_stencil_plan(shp, 6, 20, ctypes.byref(npp), ctypes.byref(tz))
    assert npp.value == 1
    assert lib.ifcm_stencil_force_plan(0, 0) == 0
    # a 2D image: an item is a run of tiles down the image (64 rows = 6 tiles of
    # 11 rows).  The rule cuts the column into the fewest runs that give four
    # items per CTA of the grid, which depends on the SM count: one particle
    # gives 2 x runs items, so a GB300's 152 SMs take runs of one tile, and the
    # one-SM count seen without a GPU takes 2 runs of 3 tiles
    lib.ifcm_stencil_plan(N.IfcmShape(64, 64, 1, 64), 4, 1, ctypes.byref(npp), ctypes.byref(tz))
    assert tz.value in (1, 3)
    # a large one: 20 particles on 854 x 854 (27 x 78 tiles) take 3 runs of 26
    # tiles per column with 152 SMs, whole columns with one
    lib.ifcm_stencil_plan(N.IfcmShape(854, 854, 1, 856), 4, 20, ctypes.byref(npp),
                          ctypes.byref(tz))
    assert npp.value == 2 and tz.value in (26, 78)


def test_multi_volume_wave_count(lib):
    p = _params()
    a = ((40, 32, 24, 40), 3, 6)
    b = ((24, 24, 24, 24), 3, 5)
    d = ((16, 16, 16, 16), 5, 1)
    vols = _batch_volumes([a, d, b])
    full = lib.pso_fitness_multi_workspace_bytes(vols, 3, ctypes.byref(p))
    lo = lib.pso_fitness_multi_min_workspace_bytes(vols, 3, ctypes.byref(p))
    assert lib.pso_fitness_multi_waves(vols, 3, ctypes.byref(p), full) == 2      # one per c
    assert lib.pso_fitness_multi_waves(vols, 3, ctypes.byref(p), lo) == 3        # one per volume
    assert lib.pso_fitness_multi_waves(vols, 3, ctypes.byref(p), lo - 256) == -1
    many = _batch_volumes([((8, 8, 8, 8), 3, 1)] * 70)
    assert lib.pso_fitness_multi_waves(many, 70, ctypes.byref(p), 1 << 40) == 2   # 64 + 6

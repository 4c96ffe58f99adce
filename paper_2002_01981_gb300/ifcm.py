"""Python binding of the C ABI with the same names (argument marshalling only).

Device memory and streams come from PyTorch: tensors are passed by
``data_ptr()`` and work is queued on ``torch.cuda.current_stream()``.  Every
step of the path runs in the CUDA kernels of ``libpifcm.so``; these wrappers
only check tensors, allocate caller-owned buffers and workspaces, and read
results back.

Volumes are CUDA float32 tensors of shape (nz, ny, pitch_x) with pitch_x a
multiple of 4; ``nx`` (<= pitch_x) gives the real row length.  Memberships
are (c, nz, ny, pitch_x).
"""
import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import native as N


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _check_cuda(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def shape_of(vol, nx=None):
    if vol.dim() != 3:
        raise ValueError("volume must be (nz, ny, pitch_x)")
    nz, ny, pitch = vol.shape
    return N.IfcmShape(int(nx if nx is not None else pitch), int(ny), int(nz), int(pitch))


_U_DTYPES = {"fp32": N.IFCM_U_FP32, "bf16": N.IFCM_U_BF16}
_REDUCES = {"fp64": N.IFCM_REDUCE_FP64, "comp32": N.IFCM_REDUCE_COMP32}


@dataclass
class Params:
    """Method parameters (Algorithm 1 inputs): clusters c, fuzzifier m, the
    iteration cap and stop threshold of one IFCM run, the d^2 floor; and the
    storage of the memberships between iterations ("fp32" or "bf16") and the
    precision of the centre / objective sums above the warp ("fp64" or
    "comp32", compensated FP32)."""
    c: int = 4
    m: float = 2.0
    max_iter: int = 50
    eps_u: float = 1e-5
    dist_floor: float = 1e-12
    V: int = 1
    h: float = 1.0
    u_dtype: str = "fp32"
    reduce: str = "fp64"

    def native(self):
        if self.u_dtype not in _U_DTYPES:
            raise ValueError(f"u_dtype must be one of {sorted(_U_DTYPES)}")
        if self.reduce not in _REDUCES:
            raise ValueError(f"reduce must be one of {sorted(_REDUCES)}")
        return N.IfcmParams(self.c, self.m, self.V, self.h, self.max_iter, self.eps_u,
                            self.dist_floor, _U_DTYPES[self.u_dtype], _REDUCES[self.reduce])


@dataclass
class Options:
    """Whole-run options of Algorithm 1 (swarm size, generations, ...)."""
    P: int = 20
    generations: int = 30
    radius: int = 1
    vmax: float = 0.2
    seed: int = 1
    init_max_iter: int = 300
    slice_z: int = -1
    fitness: str = "restart"      # or "onestep" (Algorithm 2 steps 6-11 read literally)

    def native(self):
        modes = {"restart": N.PIFCM_FITNESS_RESTART, "onestep": N.PIFCM_FITNESS_ONESTEP}
        if self.fitness not in modes:
            raise ValueError(f"fitness must be one of {sorted(modes)}")
        return N.PifcmOptions(self.P, self.generations, self.radius, self.vmax, self.seed,
                              self.init_max_iter, self.slice_z, modes[self.fitness])


def workspace(nbytes, device="cuda"):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def device_status(ws):
    lib = N.load()
    return lib.ifcm_device_status(_ptr(ws), _stream())


# ------------------------------------------------------------ Alg 2 step 1
def ifcm_normalize(vol, nx=None, out=None, ws=None):
    lib = N.load()
    _check_cuda(vol, torch.float32, "vol")
    shp = shape_of(vol, nx)
    out = torch.empty_like(vol) if out is None else out
    need = lib.ifcm_normalize_workspace_bytes(shp)
    ws = workspace(need, vol.device) if ws is None else ws
    N.check(lib.ifcm_normalize(_ptr(vol), _ptr(out), shp, _ptr(ws), ws.numel(), _stream()))
    N.check(device_status(ws))
    return out


# ------------------------------------------------------------ one IFCM run
def _lam_xi_tensor(lam_xi, device):
    if isinstance(lam_xi, torch.Tensor):
        _check_cuda(lam_xi, torch.float64, "lam_xi")
        return lam_xi
    return torch.tensor(np.asarray(lam_xi, dtype=np.float64).reshape(-1), device=device)


def ifcm_fit(x, params, lam_xi, nx=None, u_init=None, c_init=None, ws=None, plain=False):
    """One IFCM run; returns (U, C, J, iterations).  ``plain=True`` runs the
    paper-shaped form (one thread per voxel, host loop)."""
    lib = N.load()
    _check_cuda(x, torch.float32, "x")
    shp = shape_of(x, nx)
    p = params.native()
    dev = x.device
    c = params.c
    u_out = torch.empty((c,) + tuple(x.shape), dtype=torch.float32, device=dev)
    c_out = torch.empty(c, dtype=torch.float64, device=dev)
    J_out = torch.empty(1, dtype=torch.float64, device=dev)
    it_out = torch.empty(1, dtype=torch.int32, device=dev)
    if u_init is not None:
        _check_cuda(u_init, torch.float32, "u_init")
    if c_init is not None:
        c_init = _lam_xi_tensor(c_init, dev)
    need = lib.ifcm_fit_workspace_bytes(shp, ctypes.byref(p))
    ws = workspace(need, dev) if ws is None else ws
    if plain:
        lam, xi = (float(v) for v in (lam_xi.tolist() if isinstance(lam_xi, torch.Tensor)
                                      else lam_xi))
        N.check(lib.ifcm_fit_plain(_ptr(x), shp, ctypes.byref(p), lam, xi, _ptr(u_init),
                                   _ptr(c_init), _ptr(u_out), _ptr(c_out), _ptr(J_out),
                                   _ptr(it_out), _ptr(ws), ws.numel(), _stream()))
    else:
        lx = _lam_xi_tensor(lam_xi, dev)
        N.check(lib.ifcm_fit(_ptr(x), shp, ctypes.byref(p), _ptr(lx), _ptr(u_init),
                             _ptr(c_init), _ptr(u_out), _ptr(c_out), _ptr(J_out), _ptr(it_out),
                             _ptr(ws), ws.numel(), _stream()))
    N.check(device_status(ws))
    return u_out, c_out, float(J_out.item()), int(it_out.item())


# ---------------------------------------------- Alg 1 step 4, whole swarm
def pso_fitness_batch_workspace_bytes(x, params, P, nx=None):
    """Workspace bytes of a ``pso_fitness_batch`` call with P particles."""
    p = params.native()
    return N.load().pso_fitness_batch_workspace_bytes(shape_of(x, nx), ctypes.byref(p), int(P))


def pso_fitness_batch(x, params, lam_xi, u0, c0, nx=None, ws=None, want_centres=False):
    """Fitness (J of an IFCM run from (u0, c0)) of every particle; returns
    (fitness [P] float64, iterations [P] int32, centres [P, c] or None)."""
    lib = N.load()
    _check_cuda(x, torch.float32, "x")
    _check_cuda(u0, torch.float32, "u0")
    dev = x.device
    lam_xi = _lam_xi_tensor(lam_xi, dev).reshape(-1, 2).contiguous()
    c0 = _lam_xi_tensor(c0, dev)
    P = lam_xi.shape[0]
    shp = shape_of(x, nx)
    p = params.native()
    fit = torch.empty(P, dtype=torch.float64, device=dev)
    its = torch.empty(P, dtype=torch.int32, device=dev)
    cout = torch.empty((P, params.c), dtype=torch.float64, device=dev) if want_centres else None
    need = lib.pso_fitness_batch_workspace_bytes(shp, ctypes.byref(p), P)
    ws = workspace(need, dev) if ws is None else ws
    N.check(lib.pso_fitness_batch(_ptr(x), shp, ctypes.byref(p), _ptr(lam_xi), P, _ptr(u0),
                                  _ptr(c0), _ptr(fit), _ptr(its), _ptr(cout), _ptr(ws),
                                  ws.numel(), _stream()))
    N.check(device_status(ws))
    return fit, its, cout


class FitnessGraph:
    """A captured ``pso_fitness_multi`` call.  ``launch()`` replays it on the
    current stream with whatever the input tensors hold then; ``outputs`` are
    the (fitness, iterations) tensors every replay rewrites."""

    def __init__(self, handle, keep, outputs, ws):
        self._h = handle
        self._keep = keep
        self.outputs = outputs
        self.ws = ws

    def launch(self):
        N.check(N.load().ifcm_graph_launch(self._h, _stream()))

    def check(self):
        """Synchronise and raise if a kernel of the last replay flagged an error."""
        N.check(device_status(self.ws))

    def close(self):
        if self._h:
            N.load().ifcm_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pso_fitness_multi_graph(volumes, params, ws=None):
    """Capture ``pso_fitness_multi(volumes, params)`` into a CUDA graph."""
    lib = N.load()
    descs, keep, outs = _multi_descriptors(volumes)
    p = params.native()
    dev = volumes[0].x.device
    if ws is None:
        ws = workspace(lib.pso_fitness_multi_workspace_bytes(descs, len(volumes),
                                                             ctypes.byref(p)), dev)
    h = ctypes.c_void_p()
    N.check(lib.pso_fitness_multi_graph(descs, len(volumes), ctypes.byref(p), _ptr(ws),
                                        ws.numel(), ctypes.byref(h)))
    return FitnessGraph(h, (keep, volumes), outs, ws)


# ------------------------------------------------ work decomposition plans
def autotune(mode=1):
    """Turn timing of candidate stencil plans on (1) or off (0, built-in rule)."""
    N.load().ifcm_autotune_enable(int(mode))


def autotune_reset():
    N.load().ifcm_autotune_reset()


def resident_enable(on=True):
    """Whole runs of small volumes in one launch (on by default); off sends
    every batch through the stencil kernels.  See ifcm_resident_enable."""
    N.load().ifcm_resident_enable(1 if on else 0)


def force_plan(np_=0, chunks=1):
    """Make every later launch use np_ particles per item and `chunks`
    z-chunks per tile (np_ = 0 lifts it)."""
    N.check(N.load().ifcm_stencil_force_plan(int(np_), int(chunks)))


def stencil_plan(shape, c, P):
    """(particles per item, z-chunk depth, tuned?) for a one-volume batch."""
    np_, tz = ctypes.c_int32(), ctypes.c_int32()
    r = N.load().ifcm_stencil_plan(shape, int(c), int(P), ctypes.byref(np_), ctypes.byref(tz))
    if r < 0:
        raise ValueError("invalid shape, c or P")
    return np_.value, tz.value, bool(r)


# ------------------------------- Alg 1 step 4, many swarms on many volumes
@dataclass
class BatchVolume:
    """One volume of ``pso_fitness_multi``: its normalised volume, cluster
    count, particles (lam_xi [P, 2]) and the shared start (u0, c0)."""
    x: torch.Tensor
    c: int
    lam_xi: object
    u0: torch.Tensor
    c0: object
    nx: int = None


def _multi_descriptors(volumes):
    descs = (N.IfcmBatchVolume * len(volumes))()
    keep, outs = [], []
    for i, v in enumerate(volumes):
        _check_cuda(v.x, torch.float32, f"volumes[{i}].x")
        _check_cuda(v.u0, torch.float32, f"volumes[{i}].u0")
        dev = v.x.device
        lx = _lam_xi_tensor(v.lam_xi, dev).reshape(-1, 2).contiguous()
        c0 = _lam_xi_tensor(v.c0, dev)
        P = lx.shape[0]
        fit = torch.empty(P, dtype=torch.float64, device=dev)
        its = torch.empty(P, dtype=torch.int32, device=dev)
        keep += [lx, c0]
        outs.append((fit, its))
        descs[i] = N.IfcmBatchVolume(v.x.data_ptr(), shape_of(v.x, v.nx), int(v.c), int(P),
                                     lx.data_ptr(), v.u0.data_ptr(), c0.data_ptr(),
                                     fit.data_ptr(), its.data_ptr())
    return descs, keep, outs


def pso_fitness_multi_workspace_bytes(volumes, params, minimum=False):
    lib = N.load()
    descs, _keep, _ = _multi_descriptors(volumes)
    p = params.native()
    fn = (lib.pso_fitness_multi_min_workspace_bytes if minimum
          else lib.pso_fitness_multi_workspace_bytes)
    return fn(descs, len(volumes), ctypes.byref(p))


def pso_fitness_multi_waves(volumes, params, ws_bytes):
    lib = N.load()
    descs, _keep, _ = _multi_descriptors(volumes)
    p = params.native()
    return lib.pso_fitness_multi_waves(descs, len(volumes), ctypes.byref(p), int(ws_bytes))


def pso_fitness_multi(volumes, params, ws=None):
    """Fitness of every particle of every volume (volumes of the same c share
    each batched launch); ``params.c`` is ignored, each volume has its own.
    Returns a list of (fitness [P] float64, iterations [P] int32)."""
    lib = N.load()
    descs, _keep, outs = _multi_descriptors(volumes)
    p = params.native()
    dev = volumes[0].x.device
    if ws is None:
        ws = workspace(lib.pso_fitness_multi_workspace_bytes(descs, len(volumes),
                                                             ctypes.byref(p)), dev)
    N.check(lib.pso_fitness_multi(descs, len(volumes), ctypes.byref(p), _ptr(ws), ws.numel(),
                                  _stream()))
    N.check(device_status(ws))
    return outs


# ------------------------------------------- d J / d (lambda, xi) and polish
def ifcm_grad_workspace_bytes(x, params, K, nx=None):
    p = params.native()
    return N.load().ifcm_grad_workspace_bytes(shape_of(x, nx), ctypes.byref(p), int(K))


def ifcm_grad(x, params, lam_xi, u0, c0, K, nx=None, ws=None):
    """(J^{K-1}, tensor [dJ/dlambda, dJ/dxi]) of K unrolled IFCM iterations
    from (u0, c0) at (lambda, xi).  Both results stay on the device."""
    lib = N.load()
    _check_cuda(x, torch.float32, "x")
    _check_cuda(u0, torch.float32, "u0")
    dev = x.device
    lx = _lam_xi_tensor(lam_xi, dev)
    c0 = _lam_xi_tensor(c0, dev)
    shp = shape_of(x, nx)
    p = params.native()
    J = torch.empty(1, dtype=torch.float64, device=dev)
    g = torch.empty(2, dtype=torch.float64, device=dev)
    need = lib.ifcm_grad_workspace_bytes(shp, ctypes.byref(p), int(K))
    ws = workspace(need, dev) if ws is None else ws
    N.check(lib.ifcm_grad(_ptr(x), shp, ctypes.byref(p), int(K), _ptr(lx), _ptr(u0), _ptr(c0),
                          _ptr(J), _ptr(g), _ptr(ws), ws.numel(), _stream()))
    return J[0], g


def ifcm_polish(x, params, lam_xi, u0, c0, K, steps=10, step0=0.05, decay=0.7, nx=None,
                ws=None):
    """Projected gradient polishing from lam_xi; returns (best (lambda, xi)
    as a device tensor, its J^{K-1})."""
    lib = N.load()
    _check_cuda(x, torch.float32, "x")
    _check_cuda(u0, torch.float32, "u0")
    dev = x.device
    lx = _lam_xi_tensor(lam_xi, dev).clone()
    c0 = _lam_xi_tensor(c0, dev)
    shp = shape_of(x, nx)
    p = params.native()
    J = torch.empty(1, dtype=torch.float64, device=dev)
    need = lib.ifcm_grad_workspace_bytes(shp, ctypes.byref(p), int(K))
    ws = workspace(need, dev) if ws is None else ws
    N.check(lib.ifcm_polish(_ptr(x), shp, ctypes.byref(p), int(K), int(steps), float(step0),
                            float(decay), _ptr(lx), _ptr(u0), _ptr(c0), _ptr(J), _ptr(ws),
                            ws.numel(), _stream()))
    return lx, float(J[0])


class IFCMObjective(torch.autograd.Function):
    """J^{K-1}(lambda, xi) as a differentiable function of a CUDA float64
    tensor lam_xi of shape (2,).  ``forward`` runs the checkpointed forward
    pass and the adjoint kernels together (``ifcm_grad``) and keeps the
    gradient; ``backward`` scales it by the incoming gradient.

        J = IFCMObjective.apply(lam_xi, x, u0, c0, params, K, nx)
    """

    @staticmethod
    def forward(ctx, lam_xi, x, u0, c0, params, K, nx=None):
        J, g = ifcm_grad(x, params, lam_xi.detach().contiguous(), u0, c0, K, nx=nx)
        ctx.save_for_backward(g)
        return J.clone()

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return gJ * g, None, None, None, None, None, None


# ------------------------------------------------------ Alg 1 steps 3, 5-8
class Swarm:
    """Device-resident swarm; ``init`` is step 3, ``step`` steps 5-8."""

    def __init__(self, P, seed, vmax=0.2, radius=1, device="cuda"):
        self.P, self.seed, self.vmax, self.radius = int(P), int(seed), float(vmax), int(radius)
        f64 = dict(dtype=torch.float64, device=device)
        self.x = torch.empty((P, 2), **f64)
        self.v = torch.empty((P, 2), **f64)
        self.pbest_x = torch.empty((P, 2), **f64)
        self.pbest_f = torch.empty(P, **f64)
        self.gen = torch.zeros(1, dtype=torch.int32, device=device)

    def native(self):
        return N.PsoState(self.P, self.radius, self.vmax, self.seed, self.x.data_ptr(),
                          self.v.data_ptr(), self.pbest_x.data_ptr(), self.pbest_f.data_ptr(),
                          self.gen.data_ptr())

    def init(self):
        s = self.native()
        N.check(N.load().pso_init(ctypes.byref(s), _stream()))
        return self

    def step(self, fitness):
        _check_cuda(fitness, torch.float64, "fitness")
        s = self.native()
        N.check(N.load().pso_step(ctypes.byref(s), _ptr(fitness), _stream()))
        return self


# ------------------------------------------------------------ Alg 1 whole
def _result_dict(r, c):
    return {"centres": list(r.centres)[:c], "lambda": r.lambda_, "xi": r.xi, "J": r.J,
            "best_fitness": r.best_fitness, "updates": int(r.updates),
            "iters_final": int(r.iters_final), "iters_init": int(r.iters_init),
            "status": int(r.status), "best_particle": int(r.best_particle)}


def pifcm3d_buffers(vol, params, options, nx=None):
    """Caller-owned buffers of a device run: (u_out, result, ws)."""
    lib = N.load()
    shp = shape_of(vol, nx)
    p, o = params.native(), options.native()
    nz_run = 1 if options.slice_z >= 0 else shp.nz
    u_out = torch.empty((params.c, nz_run, shp.ny, shp.pitch_x), dtype=torch.float32,
                        device=vol.device)
    res = torch.zeros(ctypes.sizeof(N.PifcmResult), dtype=torch.uint8, device=vol.device)
    ws = workspace(lib.pifcm3d_workspace_bytes(shp, ctypes.byref(p), ctypes.byref(o)),
                   vol.device)
    return u_out, res, ws


def pifcm3d(vol, params, options, nx=None, buffers=None, sync=True):
    """Algorithm 1 on the device.  Returns (U, result dict) or, with
    sync=False, (U, result tensor) without reading anything back."""
    lib = N.load()
    _check_cuda(vol, torch.float32, "vol")
    shp = shape_of(vol, nx)
    p, o = params.native(), options.native()
    u_out, res, ws = buffers if buffers is not None else pifcm3d_buffers(vol, params, options, nx)
    N.check(lib.pifcm3d(_ptr(vol), shp, ctypes.byref(p), ctypes.byref(o), _ptr(u_out),
                        _ptr(res), _ptr(ws), ws.numel(), _stream()))
    if not sync:
        return u_out, res
    r = N.PifcmResult.from_buffer_copy(res.cpu().numpy().tobytes())
    if r.status:
        N.check(device_status(ws))
    return u_out, _result_dict(r, params.c)


class RunGraph:
    """A captured pifcm3d run: ``launch()`` replays Algorithm 1 on what the
    volume tensor then holds; ``result()`` reads the result block of the last
    replay (synchronising)."""

    def __init__(self, handle, buffers, keep, c):
        self._h = handle
        self.u_out, self._res, self.ws = buffers
        self._keep = keep
        self._c = c

    def launch(self):
        N.check(N.load().ifcm_graph_launch(self._h, _stream()))

    def result(self):
        r = N.PifcmResult.from_buffer_copy(self._res.cpu().numpy().tobytes())
        if r.status:
            N.check(device_status(self.ws))
        return _result_dict(r, self._c)

    def close(self):
        if self._h:
            N.load().ifcm_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pifcm3d_graph(vol, params, options, nx=None, buffers=None):
    """Capture one pifcm3d run into a CUDA graph (replayed by RunGraph.launch)."""
    lib = N.load()
    _check_cuda(vol, torch.float32, "vol")
    shp = shape_of(vol, nx)
    p, o = params.native(), options.native()
    bufs = buffers if buffers is not None else pifcm3d_buffers(vol, params, options, nx)
    u_out, res, ws = bufs
    h = ctypes.c_void_p()
    N.check(lib.pifcm3d_graph(_ptr(vol), shp, ctypes.byref(p), ctypes.byref(o), _ptr(u_out),
                              _ptr(res), _ptr(ws), ws.numel(), ctypes.byref(h)))
    return RunGraph(h, bufs, vol, params.c)


def pifcm3d_host_workspace(shape, params, options, device="cuda"):
    lib = N.load()
    p, o = params.native(), options.native()
    return workspace(lib.pifcm3d_host_workspace_bytes(shape, ctypes.byref(p), ctypes.byref(o)),
                     device)


def pifcm3d_host(vol, params, options, nx=None, u_out=None, ws=None):
    """Algorithm 1 with HOST input/outputs (numpy or pinned CPU tensors of
    shape (nz, ny, pitch_x)); copies happen inside the library call."""
    lib = N.load()
    if isinstance(vol, np.ndarray):
        vol = torch.from_numpy(np.ascontiguousarray(vol, dtype=np.float32))
    if vol.is_cuda or vol.dtype != torch.float32 or not vol.is_contiguous():
        raise TypeError("vol must be a contiguous float32 host array")
    nz, ny, pitch = vol.shape
    shp = N.IfcmShape(int(nx if nx is not None else pitch), int(ny), int(nz), int(pitch))
    p, o = params.native(), options.native()
    if ws is None:
        ws = pifcm3d_host_workspace(shp, params, options)
    res = N.PifcmResult()
    N.check(lib.pifcm3d_host(ctypes.c_void_p(vol.data_ptr()), shp, ctypes.byref(p),
                             ctypes.byref(o),
                             ctypes.c_void_p(u_out.data_ptr()) if u_out is not None else None,
                             ctypes.byref(res), _ptr(ws), ws.numel(), _stream()))
    return u_out, _result_dict(res, params.c)


# ------------------------------------------------------------ profiling
def profile_enable(on=True):
    N.load().ifcm_profile_enable(1 if on else 0)


PROF_STENCIL, PROF_ADJOINT_POINT, PROF_ADJOINT_GATHER, PROF_STENCIL3D = 0, 1, 2, 3


def set_wait_limit_ns(ns=0):
    """Bound (ns) of every wait of the kernels on their shared-memory tiles;
    0 restores the default (about one second).  See ifcm_set_wait_limit_ns."""
    N.load().ifcm_set_wait_limit_ns(int(ns))


def profile_read(kind=PROF_STENCIL):
    """(summed kernel ms, launches) recorded for one kind of kernel since the
    last read of that kind."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    N.check(N.load().ifcm_profile_read_kind(int(kind), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value

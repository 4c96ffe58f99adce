"""ctypes view of the C ABI in ``include/pifcm.h`` (``libpifcm.so``).

Structures mirror the header field by field; every function gets its
argument and return types here.  Loading fails loudly when the library is
missing: there is no fallback implementation.
"""
import ctypes
import os
from ctypes import (POINTER, Structure, c_char_p, c_double, c_int32, c_int64, c_size_t,
                    c_uint64, c_void_p)

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpifcm.so")

IFCM_OK = 0
STATUS_NAMES = {0: "IFCM_OK", 1: "IFCM_ERR_INVALID", 2: "IFCM_ERR_NOMEM", 3: "IFCM_ERR_CUDA",
                4: "IFCM_ERR_TIMEOUT", 5: "IFCM_ERR_BOUNDS", 6: "IFCM_ERR_UNSUPPORTED"}


class IfcmShape(Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("nz", c_int32), ("pitch_x", c_int32)]


IFCM_U_FP32, IFCM_U_BF16 = 0, 1
IFCM_REDUCE_FP64, IFCM_REDUCE_COMP32 = 0, 1


class IfcmParams(Structure):
    _fields_ = [("c", c_int32), ("m", c_double), ("V", c_int32), ("h", c_double),
                ("max_iter", c_int32), ("eps_u", c_double), ("dist_floor", c_double),
                ("u_dtype", c_int32), ("reduce", c_int32)]


class PsoState(Structure):
    _fields_ = [("P", c_int32), ("radius", c_int32), ("vmax", c_double), ("seed", c_uint64),
                ("x", c_void_p), ("v", c_void_p), ("pbest_x", c_void_p),
                ("pbest_f", c_void_p), ("gen", c_void_p)]


PIFCM_FITNESS_RESTART, PIFCM_FITNESS_ONESTEP = 0, 1


class PifcmOptions(Structure):
    _fields_ = [("P", c_int32), ("generations", c_int32), ("radius", c_int32),
                ("vmax", c_double), ("seed", c_uint64), ("init_max_iter", c_int32),
                ("slice_z", c_int32), ("fitness_mode", c_int32)]


class PifcmResult(Structure):
    _fields_ = [("centres", c_double * 8), ("lambda_", c_double), ("xi", c_double),
                ("J", c_double), ("best_fitness", c_double), ("updates", c_int64),
                ("iters_final", c_int32), ("iters_init", c_int32), ("status", c_int32),
                ("best_particle", c_int32)]


class IfcmBatchVolume(Structure):
    _fields_ = [("x", c_void_p), ("shape", IfcmShape), ("c", c_int32), ("P", c_int32),
                ("lam_xi", c_void_p), ("u0", c_void_p), ("c0", c_void_p),
                ("fitness", c_void_p), ("iters", c_void_p)]


# name -> (restype, argtypes); the exported symbols of include/pifcm.h
SIGNATURES = {
    "ifcm_status_string": (c_char_p, [c_int32]),
    "ifcm_last_error": (c_char_p, []),
    "ifcm_device_status": (c_int32, [c_void_p, c_void_p]),
    "ifcm_normalize_workspace_bytes": (c_size_t, [IfcmShape]),
    "ifcm_normalize": (c_int32, [c_void_p, c_void_p, IfcmShape, c_void_p, c_size_t, c_void_p]),
    "ifcm_fit_workspace_bytes": (c_size_t, [IfcmShape, POINTER(IfcmParams)]),
    "ifcm_fit": (c_int32, [c_void_p, IfcmShape, POINTER(IfcmParams), c_void_p, c_void_p,
                           c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                           c_size_t, c_void_p]),
    "ifcm_fit_plain": (c_int32, [c_void_p, IfcmShape, POINTER(IfcmParams), c_double, c_double,
                                 c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                 c_void_p, c_size_t, c_void_p]),
    "pso_fitness_batch_workspace_bytes": (c_size_t, [IfcmShape, POINTER(IfcmParams), c_int32]),
    "pso_fitness_batch": (c_int32, [c_void_p, IfcmShape, POINTER(IfcmParams), c_void_p,
                                    c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_size_t, c_void_p]),
    "pso_fitness_multi_workspace_bytes": (c_size_t, [POINTER(IfcmBatchVolume), c_int32,
                                                     POINTER(IfcmParams)]),
    "pso_fitness_multi_min_workspace_bytes": (c_size_t, [POINTER(IfcmBatchVolume), c_int32,
                                                         POINTER(IfcmParams)]),
    "pso_fitness_multi_waves": (c_int32, [POINTER(IfcmBatchVolume), c_int32,
                                          POINTER(IfcmParams), c_size_t]),
    "pso_fitness_multi": (c_int32, [POINTER(IfcmBatchVolume), c_int32, POINTER(IfcmParams),
                                    c_void_p, c_size_t, c_void_p]),
    "ifcm_autotune_enable": (None, [c_int32]),
    "ifcm_autotune_reset": (None, []),
    "ifcm_stencil_force_plan": (c_int32, [c_int32, c_int32]),
    "ifcm_stencil_plan": (c_int32, [IfcmShape, c_int32, c_int32, POINTER(c_int32),
                                    POINTER(c_int32)]),
    "pso_fitness_multi_graph": (c_int32, [POINTER(IfcmBatchVolume), c_int32,
                                          POINTER(IfcmParams), c_void_p, c_size_t,
                                          POINTER(c_void_p)]),
    "ifcm_graph_launch": (c_int32, [c_void_p, c_void_p]),
    "ifcm_graph_destroy": (None, [c_void_p]),
    "pso_init": (c_int32, [POINTER(PsoState), c_void_p]),
    "pso_step": (c_int32, [POINTER(PsoState), c_void_p, c_void_p]),
    "pifcm3d_workspace_bytes": (c_size_t, [IfcmShape, POINTER(IfcmParams),
                                           POINTER(PifcmOptions)]),
    "pifcm3d": (c_int32, [c_void_p, IfcmShape, POINTER(IfcmParams), POINTER(PifcmOptions),
                          c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "pifcm3d_graph": (c_int32, [c_void_p, IfcmShape, POINTER(IfcmParams), POINTER(PifcmOptions),
                                c_void_p, c_void_p, c_void_p, c_size_t, POINTER(c_void_p)]),
    "pifcm3d_host_workspace_bytes": (c_size_t, [IfcmShape, POINTER(IfcmParams),
                                                POINTER(PifcmOptions)]),
    "pifcm3d_host": (c_int32, [c_void_p, IfcmShape, POINTER(IfcmParams),
                               POINTER(PifcmOptions), c_void_p, POINTER(PifcmResult),
                               c_void_p, c_size_t, c_void_p]),
    "ifcm_fit_noalloc": (c_int32, [c_void_p, IfcmShape, POINTER(IfcmParams), c_void_p,
                                   c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_void_p, c_void_p]),
    "ifcm_grad_workspace_bytes": (c_size_t, [IfcmShape, POINTER(IfcmParams), c_int32]),
    "ifcm_grad": (c_int32, [c_void_p, IfcmShape, POINTER(IfcmParams), c_int32, c_void_p,
                            c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                            c_void_p]),
    "ifcm_polish": (c_int32, [c_void_p, IfcmShape, POINTER(IfcmParams), c_int32, c_int32,
                              c_double, c_double, c_void_p, c_void_p, c_void_p, c_void_p,
                              c_void_p, c_size_t, c_void_p]),
    "ifcm_profile_enable": (None, [c_int32]),
    "ifcm_profile_read": (c_int32, [POINTER(c_double), POINTER(c_int64)]),
    "ifcm_profile_read_kind": (c_int32, [c_int32, POINTER(c_double), POINTER(c_int64)]),
    "ifcm_set_wait_limit_ns": (None, [c_uint64]),
    "ifcm_resident_enable": (None, [c_int32]),
    "ifcm_fit_noalloc_status": (c_int32, [c_void_p]),
}

_lib = None


def load(path=LIB_PATH):
    """Load libpifcm.so and attach the prototypes (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with paper_2002_01981_gb300.build.build() "
            "(nvcc, sm_103a); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class IfcmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status):
    if status != IFCM_OK:
        msg = load().ifcm_last_error()
        raise IfcmError(status, msg.decode() if msg else "")
    return status

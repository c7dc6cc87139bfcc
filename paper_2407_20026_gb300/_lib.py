"""ctypes declarations of ``include/sso.h`` and the loader of ``libsso.so``.

Argument marshalling only.  Importing this module fails loudly when the
compiled library is missing; there is no fallback implementation.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsso.so")

OK = 0
ERR_INVALID = 1
ERR_OOM = 2
ERR_SINGULAR = 3
ERR_NOT_CONVERGED = 4
ERR_TIMEOUT = 5
ERR_CUDA = 6
ERR_NOT_READY = 7
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "OOM", 3: "SINGULAR", 4: "NOT_CONVERGED",
                5: "TIMEOUT", 6: "CUDA", 7: "NOT_READY"}

FP64 = 0
FP32_IR = 1
F32X2 = 2
JACOBI = 0
BLOCK_JACOBI = 1
TWO_LEVEL = 2
CHAIN = 3


class SSOError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        super().__init__("sso status %s (%d): %s" % (STATUS_NAMES.get(status, "?"), status,
                                                     message))


class Mesh(ctypes.Structure):
    _fields_ = [
        ("n_nodes", ctypes.c_int32), ("xyz", ctypes.c_void_p),
        ("n_beams", ctypes.c_int32), ("beam_conn", ctypes.c_void_p),
        ("beam_props", ctypes.c_void_p),
        ("n_quads", ctypes.c_int32), ("quad_conn", ctypes.c_void_p),
        ("quad_props", ctypes.c_void_p),
        ("fixed", ctypes.c_void_p), ("nodal_load", ctypes.c_void_p),
        ("pressure", ctypes.c_double), ("gamma", ctypes.c_double),
    ]


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32), ("precond", ctypes.c_int32),
        ("rtol", ctypes.c_double), ("inner_rtol", ctypes.c_double),
        ("max_iter", ctypes.c_int32), ("max_sweeps", ctypes.c_int32),
        ("iters_per_launch", ctypes.c_int32), ("warm_start", ctypes.c_int32),
        ("timeout_ms", ctypes.c_double),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
        ("sweeps", ctypes.c_int32), ("rel_residual", ctypes.c_double),
        ("ms", ctypes.c_double),
    ]

    def as_dict(self):
        return {"status": self.status, "iterations": self.iterations, "sweeps": self.sweeps,
                "rel_residual": self.rel_residual, "ms": self.ms}


# name -> (argtypes, restype); every symbol declared in include/sso.h
_vp, _i32, _f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
SIGNATURES = {
    "sso_default_options": ([ctypes.POINTER(Options)], None),
    "sso_last_error": ([], ctypes.c_char_p),
    "sso_version": ([], ctypes.c_char_p),
    "sso_kernel_launches": ([], ctypes.c_ulonglong),
    "sso_beam_stiffness": ([_i32, _vp, _vp, _vp, _vp, _vp], _i32),
    "sso_quad_stiffness": ([_i32, _vp, _vp, _vp, _vp, _vp], _i32),
    "sso_bsr_spmv": ([_i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "sso_bsr_spmv_noalloc": ([_i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "sso_model_create": ([ctypes.POINTER(Mesh), _vp, ctypes.POINTER(_vp)], _i32),
    "sso_model_destroy": ([_vp], None),
    "sso_model_set_design": ([_vp, _vp, _vp], _i32),
    "sso_model_solve": ([_vp, ctypes.POINTER(Options), ctypes.POINTER(Stats)], _i32),
    "sso_model_gradient": ([_vp, _f64, _vp, ctypes.POINTER(Stats)], _i32),
    "sso_model_get": ([_vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "sso_model_info": ([_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)],
                       _i32),
    "sso_model_get_stiffness": ([_vp, _vp, _vp, _vp, _vp], _i32),
    "sso_model_get_load": ([_vp, _vp], _i32),
    "sso_batch_create": ([ctypes.POINTER(_vp), _i32, ctypes.POINTER(_vp)], _i32),
    "sso_batch_destroy": ([_vp], None),
    "sso_batch_solve": ([_vp, ctypes.POINTER(Options), ctypes.POINTER(Stats)], _i32),
    "sso_batch_gradient": ([_vp, ctypes.POINTER(_f64), ctypes.POINTER(_vp),
                            ctypes.POINTER(Stats)], _i32),
    "sso_batch_set_profiling": ([_vp, _i32], _i32),
    "sso_batch_set_parts": ([_vp, _i32], _i32),
    "sso_server_create": ([ctypes.POINTER(Options), ctypes.c_size_t, _i32, _i32,
                           ctypes.POINTER(_vp)], _i32),
    "sso_server_create_lanes": ([ctypes.POINTER(Options), ctypes.c_size_t, _i32, _i32, _i32,
                                 ctypes.POINTER(_vp)], _i32),
    "sso_server_destroy": ([_vp], None),
    "sso_server_submit": ([_vp, ctypes.POINTER(Mesh), _f64, ctypes.POINTER(ctypes.c_uint64)],
                          _i32),
    "sso_server_step": ([_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)], _i32),
    "sso_server_completed": ([_vp, ctypes.POINTER(ctypes.c_uint64), _i32, ctypes.POINTER(_i32)],
                             _i32),
    "sso_server_info": ([_vp, ctypes.POINTER(_f64), ctypes.POINTER(ctypes.c_int64)], _i32),
    "sso_server_poll": ([_vp, ctypes.c_uint64, _vp, _vp, _vp, _vp, ctypes.POINTER(Stats),
                         ctypes.POINTER(_f64)], _i32),
    "sso_batch_kernel_times": ([_vp, ctypes.POINTER(_f64), ctypes.POINTER(_f64),
                                ctypes.POINTER(ctypes.c_int64)], _i32),
    "sso_model_volume": ([_vp, _vp, _vp, _vp], _i32),
    "sso_model_set_topology": ([_vp, _vp, _f64], _i32),
    "sso_aggregate": ([ctypes.POINTER(Mesh), _vp, ctypes.POINTER(_i32)], _i32),
    "sso_model_get_topology_gradient": ([_vp, _vp], _i32),
    "sso_batch_setup_times": ([_vp, ctypes.POINTER(_f64), ctypes.POINTER(_f64),
                               ctypes.POINTER(_f64), ctypes.POINTER(_f64), ctypes.POINTER(_f64),
                               ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
                              _i32),
}

_lib = None


def load():
    """Load libsso.so (built in-tree by ``_build.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                "libsso.so not found at %s; build it with __graft_entry__.build() "
                "(there is no CPU fallback)" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def check(status):
    if status != OK:
        msg = load().sso_last_error().decode(errors="replace")
        raise SSOError(status, msg)
    return status

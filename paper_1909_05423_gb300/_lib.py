"""ctypes binding of the C ABI in include/pittpack_gb.h (argument marshalling only).

The shared library must have been built (``python -m paper_1909_05423_gb300.build`` or
``__graft_entry__.build()``); loading fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpittpack_gb.so")

PP_OK = 0
STATUS_NAMES = {0: "PP_OK", 1: "PP_ERR_INVALID_ARG", 2: "PP_ERR_UNSUPPORTED_SIZE", 3: "PP_ERR_BC_PAIRING",
                4: "PP_ERR_OUT_OF_MEMORY", 5: "PP_ERR_CUDA", 6: "PP_ERR_TIMEOUT", 7: "PP_ERR_INTERNAL",
                8: "PP_ERR_RANGE"}
PP_ERR_RANGE = 8
BC_CODE = {"P": 0, "N": 1, "D": 2}
DTYPES = {"f64": 0, "mixed_f64io": 1, "mixed_f32io": 2}

# every entry point declared in include/pittpack_gb.h
EXPORTS = ["pp_plan_create", "pp_solve", "pp_solve_refined", "pp_solve_refined_noalloc", "pp_fold_bc", "pp_solve_batched",
           "pp_solve_adjoint", "pp_solve_host", "pp_run_stage", "pp_plan_destroy", "pp_plan_status", "pp_plan_device_bytes",
           "pp_plan_launch_shapes", "pp_plan_z_method", "pp_plan_z_split", "pp_proto_tc_gemm_check", "pp_proto_dft32_tc", "pp_last_error_string", "pp_version"]


class PPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class PlanOptions(ctypes.Structure):
    _fields_ = [("threads_x", ctypes.c_int), ("threads_y", ctypes.c_int), ("lines_x", ctypes.c_int),
                ("cols_y", ctypes.c_int), ("autotune", ctypes.c_int), ("threads_x_inv", ctypes.c_int),
                ("lines_x_inv", ctypes.c_int), ("threads_y_inv", ctypes.c_int), ("cols_y_inv", ctypes.c_int),
                ("z_method", ctypes.c_int), ("z_split", ctypes.c_int), ("reserved", ctypes.c_int * 1)]


_lock = threading.Lock()
_lib = None


def load():
    """Load the library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError("pittpack-gb CUDA library not built (%s missing); run "
                              "`python -m paper_1909_05423_gb300.build`" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        lib.pp_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, ctypes.POINTER(PlanOptions)]
        lib.pp_plan_create.restype = ctypes.c_int
        for name in ("pp_solve", "pp_solve_refined", "pp_solve_refined_noalloc", "pp_solve_adjoint",
                     "pp_solve_host"):
            fn = getattr(lib, name)
            fn.argtypes = [vp, vp, vp, vp]
            fn.restype = ctypes.c_int
        lib.pp_run_stage.argtypes = [vp, ctypes.c_int, vp, vp, vp]
        lib.pp_run_stage.restype = ctypes.c_int
        lib.pp_solve_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int, vp]
        lib.pp_solve_batched.restype = ctypes.c_int
        lib.pp_fold_bc.argtypes = [vp, vp, vp, ctypes.POINTER(vp), vp]
        lib.pp_fold_bc.restype = ctypes.c_int
        lib.pp_plan_destroy.argtypes = [vp]
        lib.pp_plan_destroy.restype = ctypes.c_int
        lib.pp_plan_status.argtypes = [vp]
        lib.pp_plan_status.restype = ctypes.c_int
        lib.pp_plan_device_bytes.argtypes = [vp]
        lib.pp_plan_device_bytes.restype = ctypes.c_size_t
        lib.pp_plan_launch_shapes.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        lib.pp_plan_launch_shapes.restype = ctypes.c_int
        lib.pp_plan_z_method.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        lib.pp_plan_z_method.restype = ctypes.c_int
        lib.pp_plan_z_split.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        lib.pp_plan_z_split.restype = ctypes.c_int
        lib.pp_proto_tc_gemm_check.argtypes = [vp, vp, vp, ctypes.c_int, vp, vp]
        lib.pp_proto_tc_gemm_check.restype = ctypes.c_int
        lib.pp_proto_dft32_tc.argtypes = [vp, vp, vp, vp, ctypes.c_longlong, vp, vp]
        lib.pp_proto_dft32_tc.restype = ctypes.c_int
        lib.pp_last_error_string.argtypes = []
        lib.pp_last_error_string.restype = ctypes.c_char_p
        lib.pp_version.argtypes = []
        lib.pp_version.restype = ctypes.c_char_p
        _lib = lib
        return lib


def check(status: int):
    if status != PP_OK:
        raise PPError(status, load().pp_last_error_string().decode())


def bc_array(bc: str):
    if len(bc) != 6 or any(c not in BC_CODE for c in bc):
        raise ValueError("bc must be 6 letters from P/N/D for faces x-,x+,y-,y+,z-,z+: %r" % (bc,))
    return (ctypes.c_int * 6)(*[BC_CODE[c] for c in bc])

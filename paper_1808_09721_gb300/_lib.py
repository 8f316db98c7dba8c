"""ctypes declarations of the C ABI in include/rmhd.h (librmhd.so).

Argument marshalling only: every step of the method runs in the CUDA kernels
of librmhd.so. If the library is missing or cannot be loaded the import fails
loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librmhd.so")

RMHD_OK = 0
ERRORS = {-1: "RMHD_ERR_INVALID", -2: "RMHD_ERR_CUDA", -3: "RMHD_ERR_NEWTON", -4: "RMHD_ERR_C2P",
          -5: "RMHD_ERR_STATE", -6: "RMHD_ERR_NOMEM"}
RESISTIVE, TWO_FLUID = 0, 1
OUTFLOW, PERIODIC = 0, 1
FP64, MIXED, FLOATFLOAT = 0, 1, 2
SSP2, SSP3 = 0, 1  # IMEX integrators of Tables 1 and 2
HOST, DEVICE = 0, 1

# every symbol include/rmhd.h declares
EXPORTS = ("rmhd_workspace_bytes", "rmhd_create", "rmhd_destroy", "rmhd_last_error", "rmhd_set_prims",
           "rmhd_get_prims", "rmhd_get_cons", "rmhd_set_cons", "rmhd_imex_step", "rmhd_check",
           "rmhd_diagnostics", "rmhd_recording_bytes", "rmhd_record", "rmhd_adjoint_step",
           "rmhd_batch_workspace_bytes", "rmhd_create_batch", "rmhd_autotune",
           "rmhd_set_profiling", "rmhd_kernel_times", "rmhd_diagnostics_noalloc", "rmhd_version",
           "rmhd_set_solver_stats", "rmhd_solver_stats", "rmhd_set_refinement_cap",
           "rmhd_state_doubles", "rmhd_get_state", "rmhd_set_state", "rmhd_fp64_fma_rate",
           "rmhd_step_phase", "rmhd_slab_workspace_bytes", "rmhd_create_slab", "rmhd_halo_doubles",
           "rmhd_halo_pack", "rmhd_halo_unpack", "rmhd_eval_math",
           "rmhd_set_first_start")


class Config(C.Structure):
    _fields_ = [("model", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("xmin", C.c_double), ("xmax", C.c_double), ("ymin", C.c_double), ("ymax", C.c_double),
                ("gamma", C.c_double), ("sigma", C.c_double), ("mu_e", C.c_double), ("mu_p", C.c_double),
                ("kappa", C.c_double), ("cfl", C.c_double),
                ("bc_x", C.c_int), ("bc_y", C.c_int), ("precision", C.c_int), ("scheme", C.c_int),
                ("nz", C.c_int), ("bc_z", C.c_int), ("zlen", C.c_double)]


class RmhdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)


def load(path: str | None = None):
    """Load librmhd.so (build it first with paper_1808_09721_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"librmhd.so not found at {p}: run `python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(p)
    for name in EXPORTS:
        if not hasattr(L, name):
            raise ImportError(f"librmhd.so lacks {name}")
    L.rmhd_workspace_bytes.argtypes = [C.POINTER(Config), C.POINTER(C.c_size_t)]
    L.rmhd_create.argtypes = [C.POINTER(_P), C.POINTER(Config), _P, _P, C.c_size_t]
    L.rmhd_destroy.argtypes = [_P]
    L.rmhd_destroy.restype = None
    L.rmhd_last_error.argtypes = [_P]
    L.rmhd_last_error.restype = C.c_char_p
    for name in ("rmhd_set_prims", "rmhd_get_prims", "rmhd_get_cons", "rmhd_set_cons"):
        getattr(L, name).argtypes = [_P, _P, C.c_int]
    L.rmhd_imex_step.argtypes = [_P, C.c_double, C.c_int, _D]
    L.rmhd_check.argtypes = [_P]
    L.rmhd_diagnostics.argtypes = [_P, _D]
    _I = C.POINTER(C.c_int)
    L.rmhd_recording_bytes.argtypes = [_P, C.c_int, C.c_int, C.POINTER(C.c_size_t)]
    L.rmhd_record.argtypes = [_P, C.c_int, C.c_int, _P, C.c_size_t]
    L.rmhd_adjoint_step.argtypes = [_P, _P, C.c_int, _P, C.c_int, _D]
    L.rmhd_batch_workspace_bytes.argtypes = [C.POINTER(Config), C.c_int, _I, C.POINTER(C.c_size_t)]
    L.rmhd_create_batch.argtypes = [C.POINTER(_P), C.POINTER(Config), C.c_int, _I, _D, _P, _P, C.c_size_t]
    L.rmhd_autotune.argtypes = [_P, _I]
    L.rmhd_set_profiling.argtypes = [_P, C.c_int]
    L.rmhd_kernel_times.argtypes = [_P, _D, C.POINTER(C.c_int)]
    L.rmhd_set_solver_stats.argtypes = [_P, C.c_int]
    L.rmhd_solver_stats.argtypes = [_P, C.POINTER(C.c_ulonglong)]
    L.rmhd_set_refinement_cap.argtypes = [_P, C.c_int]
    L.rmhd_set_first_start.argtypes = [_P, C.c_int]
    L.rmhd_state_doubles.argtypes = [_P, C.POINTER(C.c_size_t)]
    L.rmhd_get_state.argtypes = [_P, _P, C.c_int]
    L.rmhd_set_state.argtypes = [_P, _P, C.c_int]
    L.rmhd_diagnostics_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                            _P, _P, _P, _P]
    L.rmhd_fp64_fma_rate.argtypes = [_P, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    L.rmhd_step_phase.argtypes = [_P, C.c_double, C.c_int, C.POINTER(C.c_double)]
    L.rmhd_eval_math.argtypes = [C.c_int, C.c_longlong, _P, _P, _P, _P]
    L.rmhd_slab_workspace_bytes.argtypes = [C.POINTER(Config), C.c_int, C.c_int, C.POINTER(C.c_size_t)]
    L.rmhd_create_slab.argtypes = [C.POINTER(_P), C.POINTER(Config), C.c_int, C.c_int, _P, _P, C.c_size_t]
    L.rmhd_halo_doubles.argtypes = [_P, C.POINTER(C.c_size_t)]
    L.rmhd_halo_pack.argtypes = [_P, _P, _P]
    L.rmhd_halo_unpack.argtypes = [_P, _P, _P]
    L.rmhd_version.restype = C.c_char_p
    _lib = L
    return L

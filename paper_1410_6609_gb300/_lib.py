"""ctypes binding of libccmg.so (include/ccmg.h): argument marshalling only.

The library is built in-tree by ``paper_1410_6609_gb300._build``. Loading fails loudly when it is
missing: there is no fallback implementation of any operation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

_lock = threading.Lock()
_lib = None

MG_OK, MG_ERR_INVALID, MG_ERR_CUDA, MG_ERR_OOM, MG_ERR_NOT_CONVERGED, MG_ERR_DIVERGED, MG_ERR_TIMEOUT = range(7)
STATUS_NAMES = {0: "MG_OK", 1: "MG_ERR_INVALID", 2: "MG_ERR_CUDA", 3: "MG_ERR_OOM",
                4: "MG_ERR_NOT_CONVERGED", 5: "MG_ERR_DIVERGED", 6: "MG_ERR_TIMEOUT"}
MG_FP64, MG_MIXED = 0, 1
DIRICHLET, NEUMANN, PERIODIC = 0, 1, 2


class MgParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("h", ctypes.c_double),
        ("bc_type", ctypes.c_int * 6),
        ("bc_value", ctypes.c_double * 6),
        ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
        ("cgc_weight", ctypes.c_double),
        ("prec", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("mixed_inner", ctypes.c_int),
    ]


class MgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


# name -> (restype, argtypes)
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
SIGNATURES = {
    "mg_default_params": (None, [_P, _I, _I, _I, _D]),
    "mg_create": (_I, [_P, _P, _P]),
    "mg_destroy": (_I, [_P]),
    "mg_last_error": (ctypes.c_char_p, [_P]),
    "mg_num_levels": (_I, [_P]),
    "mg_level_dims": (_I, [_P, _I, _P]),
    "mg_set_bc_values": (_I, [_P, _P]),
    "mg_set_rhs": (_I, [_P, _P]),
    "mg_set_rhs_f": (_I, [_P, _P]),
    "mg_set_solution": (_I, [_P, _P]),
    "mg_get_solution": (_I, [_P, _P]),
    "mg_vcycle": (_I, [_P, _I]),
    "mg_solve": (_I, [_P, _D, _I, _P, _P]),
    "mg_residual": (_I, [_P, _P, _P]),
    "mg_efield": (_I, [_P, _P]),
    "mg_set_gradient_stencil": (_I, [_P, _I]),
    "mg_set_bc_field": (_I, [_P, _I, _P]),
    "mg_gradient_stencil": (_I, [_P]),
    "mg_sphere_density": (_I, [_P, _I, _P, _P, _P, _I, _P]),
    "mg_force_gather": (_I, [_P, _I, _P, _P, _P, _I, _P]),
    "mg_force_gather_adjoint": (_I, [_P, _I, _P, _P, _P, _I, _P, _P, _P, _P]),
    "mg_sphere_density_adjoint": (_I, [_P, _I, _P, _P, _I, _P, _P]),
    "mg_rhs_adjoint": (_I, [_P, _P, _P, _P]),
    "mg_adjoint_solve": (_I, [_P, _P, _P, _D, _I, _P, _P]),
    "mg_step_host": (_I, [_P, _I, _P, _P, _P, _I, _D, _I, _P, _P, _P]),
    "mg_level_set": (_I, [_P, _I, _I, _P]),
    "mg_level_get": (_I, [_P, _I, _I, _P]),
    "mg_op_smooth": (_I, [_P, _I, _I]),
    "mg_op_residual_restrict": (_I, [_P, _I]),
    "mg_op_residual_restrict_red": (_I, [_P, _I]),
    "mg_op_prolong_correct": (_I, [_P, _I]),
    "mg_op_prolong_smooth": (_I, [_P, _I]),
    "mg_level_prolong_sweep_kind": (_I, [_P, _I]),
    "mg_op_coarse_solve": (_I, [_P, _P]),
    "mg_op_residual_norm": (_I, [_P]),
    "mg_op_scale_convert": (_I, [_P, _P, _P, ctypes.c_longlong, _D, _P, _P, _P, _P]),
    "mg_op_defect_update": (_I, [_P, _I, _D, _D, _P, _P, _P, _P, _P, _P, _P]),
    "mg_op_defect_step": (_I, [_P]),
    "mg_outer_counts": (_I, [_P, _P]),
    "mg_kernel_launches": (ctypes.c_longlong, [_P]),
    "mg_level_sweep_kind": (_I, [_P, _I]),
    "mg_selftest_wait_timeout": (_I, [_P, _I]),
    "mg_set_permittivity": (_I, [_P, _P]),
    "mg_has_permittivity": (_I, [_P]),
    "mg_set_reaction": (_I, [_P, _P]),
    "mg_has_reaction": (_I, [_P]),
    "mg_solve_pb": (_I, [_P, _D, _I, _D, _I, _P, _P]),
    "mg_residual_norm_static": (_I, [_I, _I, _I, _D, _P, _P, _P, _P, _P]),
    "mg_batch_create": (_I, [_I, _P, _P, _P]),
    "mg_batch_destroy": (_I, [_P]),
    "mg_batch_last_error": (ctypes.c_char_p, [_P]),
    "mg_batch_size": (_I, [_P]),
    "mg_batch_set_rhs": (_I, [_P, _I, _P]),
    "mg_batch_set_rhs_all": (_I, [_P, _P]),
    "mg_batch_set_solution": (_I, [_P, _I, _P]),
    "mg_batch_get_solution": (_I, [_P, _I, _P]),
    "mg_batch_vcycle": (_I, [_P, _I]),
    "mg_batch_solve": (_I, [_P, _D, _I, _P, _P]),
    "mg_batch_set_tiles": (_I, [_P, _P]),
    "mg_batch_get_tiles": (_I, [_P, _P]),
    "mg_batch_autotune": (_I, [_P, _I, _P, _P, _P]),
    "mg_batch_kernel_launches": (ctypes.c_longlong, [_P]),
}


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load libccmg.so (building it first if it is missing and nvcc is available)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB_PATH) or not _build.up_to_date():
                if not build_if_missing:
                    raise OSError(f"libccmg.so not built at {_build.LIB_PATH}")
                _build.build()
            lib = ctypes.CDLL(_build.LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(lib, ctx, status: int, what: str = ""):
    if status != MG_OK:
        msg = lib.mg_last_error(ctx)
        raise MgError(status, (what + ": " if what else "") + (msg.decode() if msg else ""))

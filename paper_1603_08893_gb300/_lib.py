"""ctypes binding of ``librve.so`` (declarations of include/rve.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Importing this module loads the compiled library and raises
``ImportError`` if it has not been built -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

RVE_OK = 0
RVE_ERR_INVALID = -1
RVE_ERR_CUDA = -2
RVE_ERR_NOMEM = -3
RVE_ERR_CG_MAXIT = -4
RVE_ERR_CG_BREAKDOWN = -5
RVE_ERR_NEWTON_MAXIT = -6
RVE_ERR_NONFINITE = -7
RVE_ERR_DETF = -8
RVE_ERR_TIMEOUT = -9
RVE_ERR_UNSUPPORTED = -10

RVE_SVK = 0
RVE_J2 = 1
RVE_FP64 = 0
RVE_MIXED = 1
RVE_TAN_AUTO = 0
RVE_TAN_FULL81 = 1
RVE_TAN_RECOMPUTE = 2
RVE_TAN_SYM45 = 3
RVE_PRECOND_NONE = 0
RVE_PRECOND_REFERENCE = 1
RVE_MAX_NEWTON_LOG = 64


class rve_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("tangent", C.c_int),
                ("max_newton", C.c_int), ("max_cg", C.c_int),
                ("cg_tol_floor", C.c_double), ("cg_atol", C.c_double),
                ("mixed_refine", C.c_int), ("residual", C.c_int),
                ("autotune", C.c_int), ("precond", C.c_int),
                ("stream", C.c_void_p), ("workspace", C.c_void_p),
                ("workspace_bytes", C.c_size_t)]


class rve_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("newton_iters", C.c_int),
                ("cg_iters_total", C.c_int),
                ("cg_iters", C.c_int * RVE_MAX_NEWTON_LOG),
                ("rel_update", C.c_double * RVE_MAX_NEWTON_LOG),
                ("residual", C.c_double * RVE_MAX_NEWTON_LOG),
                ("elapsed_ms", C.c_double), ("substeps", C.c_int),
                ("cuts", C.c_int),
                ("substep_to", C.c_double * RVE_MAX_NEWTON_LOG),
                ("macro_iters", C.c_int), ("tangent_solves", C.c_int)]


_H = C.c_void_p
_P = C.c_void_p
_SIGS = {
    "rve_default_options": (None, [C.POINTER(rve_options)]),
    "rve_workspace_size": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.POINTER(rve_options), C.POINTER(C.c_size_t)]),
    "rve_create": (C.c_int, [C.POINTER(_H), C.c_int, C.c_int, C.c_int, C.c_int,
                             C.c_int, _P, _P, _P, C.POINTER(rve_options)]),
    "rve_destroy": (None, [_H]),
    "rve_set_macro_F": (C.c_int, [_H, _P]),
    "rve_solve_increment": (C.c_int, [_H, C.c_double, C.c_double,
                                      C.POINTER(rve_stats)]),
    "rve_solve_step": (C.c_int, [_H, _P, C.c_double, C.c_double, C.c_int,
                                 C.POINTER(rve_stats)]),
    "rve_solve_mixed": (C.c_int, [_H, _P, _P, _P, C.c_double, C.c_double, C.c_double,
                                  C.c_int, C.POINTER(rve_stats)]),
    "rve_macro_F": (C.c_int, [_H, _P]),
    "rve_get_F": (C.c_int, [_H, _P, C.c_int]),
    "rve_get_P": (C.c_int, [_H, _P, C.c_int]),
    "rve_get_K4": (C.c_int, [_H, _P, C.c_int]),
    "rve_get_history": (C.c_int, [_H, _P, C.c_int]),
    "rve_adjoint_grad_mu": (C.c_int, [_H, _P, C.c_double, _P, C.c_int,
                                      C.POINTER(C.c_int)]),
    "rve_adjoint_grad": (C.c_int, [_H, _P, C.c_double, _P, _P, C.c_int,
                                   C.POINTER(C.c_int)]),
    "rve_adjoint_grad_params": (C.c_int, [_H, _P, C.c_double, _P, C.c_int,
                                          C.POINTER(C.c_int)]),
    "rve_tape": (C.c_int, [_H, C.c_int]),
    "rve_tape_length": (C.c_int, [_H]),
    "rve_adjoint_grad_path": (C.c_int, [_H, _P, C.c_double, _P, C.c_int, C.POINTER(C.c_int)]),
    "rve_homogenized_P": (C.c_int, [_H, _P]),
    "rve_set_F": (C.c_int, [_H, _P, C.c_int]),
    "rve_apply_operator": (C.c_int, [_H, _P, _P, C.c_int]),
    "rve_project": (C.c_int, [_H, _P, _P, C.c_int]),
    "rve_last_error": (C.c_char_p, [_H]),
    "rve_status_string": (C.c_char_p, [C.c_int]),
    "rve_launch_count": (C.c_int, [_H, C.POINTER(C.c_longlong)]),
    "rve_tuning": (C.c_int, [_H, C.POINTER(C.c_int)]),
    "rve_set_tuning": (C.c_int, [_H, C.POINTER(C.c_int)]),
    "rve_save": (C.c_int, [_H, C.c_char_p]),
    "rve_load": (C.c_int, [C.POINTER(_H), C.c_char_p, C.POINTER(rve_options)]),
    "rve_grid": (C.c_int, [_H, C.POINTER(C.c_int)]),
    "rve_model": (C.c_int, [_H]),
    "rve_kernel_timing": (C.c_int, [_H, C.c_int, C.c_int]),
    "rve_set_wait_polls": (C.c_int, [_H, C.c_uint]),
    "rve_kernel_time": (C.c_int, [_H, C.POINTER(C.c_double),
                                  C.POINTER(C.c_longlong)]),
    "rve_project_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, _P, _P, _P]),
    "rve_batch_create": (C.c_int, [C.POINTER(_H), C.c_int, _P, C.c_int, _P, _P, _P,
                                   C.POINTER(rve_options)]),
    "rve_batch_destroy": (None, [_H]),
    "rve_batch_solve": (C.c_int, [_H, _P, C.c_double, C.c_double, _P]),
    "rve_batch_solve_step": (C.c_int, [_H, _P, C.c_double, C.c_double, C.c_int, _P]),
    "rve_batch_size": (C.c_int, [_H]),
    "rve_batch_cell": (_H, [_H, C.c_int]),
    "rve_batch_homogenized_P": (C.c_int, [_H, _P]),
    "rve_batch_launch_count": (C.c_int, [_H, C.POINTER(C.c_longlong)]),
    "rve_batch_last_error": (C.c_char_p, [_H]),
}


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()

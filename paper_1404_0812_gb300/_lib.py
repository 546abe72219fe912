"""ctypes declarations of the C ABI in include/rbffd.h.

Argument marshalling only: every computation happens in ``librbffd.so``.
If the library cannot be built or loaded, ``load()`` raises -- there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import _build

RBFFD_MAX_GROUPS = 8
OK, EINVAL, ECUDA, ENOMEM, EPS_SEARCH_FAILED, SOLVER_NOT_CONVERGED, TIMEOUT, NOT_IMPLEMENTED, ESINGULAR = range(9)
GAUSSIAN, IMQ = 0, 1
F32, F64 = 0, 1
PREC_F64, PREC_DD = 0, 1
MODEL_NONE, MODEL_LINEAR, MODEL_SCHNAKENBERG, MODEL_GRAY_SCOTT, MODEL_BARRIO = range(5)
SOLVER_BICGSTAB, SOLVER_BANDED_LU = 0, 1
STENCIL_OK, STENCIL_NO_BRACKET, STENCIL_NO_CONVERGENCE, STENCIL_SINGULAR, STENCIL_ACCEPTED_PREDICTION = range(5)

vp = C.c_void_p


class BuildOpts(C.Structure):
    _fields_ = [("kernel", C.c_int), ("kappa_target", C.c_double), ("eps_tol", C.c_double),
                ("max_evals", C.c_int), ("use_learned", C.c_int), ("accept_lo", C.c_double),
                ("accept_hi", C.c_double), ("eps_override", vp),
                ("mlp", vp * RBFFD_MAX_GROUPS), ("block_threads", C.c_int),
                ("blocks_per_sm", C.c_int), ("eps_lo", C.c_double), ("eps_hi", C.c_double),
                ("precision", C.c_int)]


class EllView(C.Structure):
    _fields_ = [("ngroups", C.c_int), ("n", C.c_int * RBFFD_MAX_GROUPS),
                ("npad", C.c_int * RBFFD_MAX_GROUPS),
                ("row_begin", C.c_int64 * (RBFFD_MAX_GROUPS + 1)),
                ("elem_begin", C.c_int64 * (RBFFD_MAX_GROUPS + 1)), ("elems", C.c_int64),
                ("row_node", vp), ("idx", vp), ("w64", vp), ("w32", vp)]


class StepParams(C.Structure):
    _fields_ = [("model", C.c_int), ("nspecies", C.c_int), ("dtype", C.c_int), ("dt", C.c_double),
                ("delta_u", C.c_double), ("delta_v", C.c_double), ("coef", C.c_double * 8),
                ("tol", C.c_double), ("maxit", C.c_int), ("use_graph", C.c_int), ("order", C.c_int),
                ("source_u", vp), ("source_v", vp), ("source_rate", C.c_double), ("solver", C.c_int)]


class State(C.Structure):
    _fields_ = [("u", vp), ("v", vp), ("u_prev", vp), ("v_prev", vp), ("f_prev", vp),
                ("g_prev", vp), ("has_history", C.c_int), ("step", C.c_int64),
                ("u_prev2", vp), ("v_prev2", vp), ("f_prev2", vp), ("g_prev2", vp),
                ("u_prev3", vp), ("v_prev3", vp), ("f_prev3", vp), ("g_prev3", vp), ("t", C.c_double)]


class StepReport(C.Structure):
    _fields_ = [("steps_done", C.c_int64), ("max_iters_u", C.c_int32), ("max_iters_v", C.c_int32),
                ("total_iters", C.c_int64), ("last_relres_u", C.c_double),
                ("last_relres_v", C.c_double), ("failed_step", C.c_int64)]


# name -> (restype, argtypes)
SIGNATURES = {
    "rbffd_build_opts_default": (None, [C.POINTER(BuildOpts)]),
    "rbffd_build_operator": (C.c_int, [vp, vp, C.c_int64, vp, C.c_int, C.POINTER(BuildOpts), vp,
                                       C.POINTER(vp)]),
    "rbffd_apply": (C.c_int, [vp, vp, vp, C.c_int, vp]),
    "rbffd_autotune_build": (C.c_int, [vp, vp, C.c_int64, vp, C.c_int, C.POINTER(BuildOpts), C.c_int64,
                                       C.c_char_p, vp, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                       C.POINTER(C.c_double)]),
    "rbffd_step_imex": (C.c_int, [vp, C.POINTER(State), C.POINTER(StepParams), C.c_int64, vp,
                                  C.POINTER(StepReport)]),
    "rbffd_get_stencil_info": (C.c_int, [vp, vp, vp, vp, vp, vp]),
    "rbffd_get_rows": (C.c_int, [vp, vp, vp, vp]),
    "rbffd_get_eps": (C.c_int, [vp, vp, vp, vp, vp]),
    "rbffd_get_ell": (C.c_int, [vp, C.POINTER(EllView)]),
    "rbffd_get_build_timings": (C.c_int, [vp, C.POINTER(C.c_double)]),
    "rbffd_launch_count": (C.c_int64, []),
    "rbffd_op_nodes": (C.c_int64, [vp]),
    "rbffd_op_max_n": (C.c_int, [vp]),
    "rbffd_op_nnz": (C.c_int64, [vp]),
    "rbffd_op_apply_bytes": (C.c_int64, [vp, C.c_int]),
    "rbffd_destroy": (None, [vp]),
    "rbffd_mlp_param_count": (C.c_int64, [C.c_int]),
    "rbffd_mlp_create": (C.c_int, [C.c_int, vp, C.POINTER(vp)]),
    "rbffd_mlp_get_params": (C.c_int, [vp, vp]),
    "rbffd_mlp_load": (C.c_int, [vp, vp]),
    "rbffd_mlp_destroy": (None, [vp]),
    "rbffd_features": (C.c_int, [vp, vp, vp, C.c_int, vp, vp, C.POINTER(C.c_int64), vp]),
    "rbffd_mlp_loss_grad": (C.c_int, [vp, vp, vp, C.c_int64, vp, vp, vp]),
    "rbffd_mlp_train": (C.c_int, [vp, vp, vp, C.c_int64, C.c_int, C.c_int, C.c_float, C.c_uint64,
                                  vp, vp]),
    "rbffd_mlp_predict": (C.c_int, [vp, vp, C.c_int64, vp, vp]),
    "rbffd_selftest_barrier_timeout": (C.c_int, [vp]),
    "rbffd_stencil_weights_noalloc": (C.c_int, [vp, vp, C.c_int64, vp, C.c_int64, C.c_int, vp, C.c_int,
                                                vp, vp]),
    "rbffd_op_bandwidth": (C.c_int, [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), vp]),
    "rbffd_lu_factor": (C.c_int, [vp, C.c_double, C.c_double, C.c_int, vp, C.POINTER(vp)]),
    "rbffd_lu_solve": (C.c_int, [vp, vp, vp, vp]),
    "rbffd_lu_bytes": (C.c_int64, [vp]),
    "rbffd_lu_destroy": (None, [vp]),
    "rbffd_morton_order": (C.c_int, [vp, C.c_int64, vp, vp]),
    "rbffd_rcm_order": (C.c_int, [vp, vp, vp]),
    "rbffd_rcm_order_host": (C.c_int, [vp, vp, C.c_int64, vp]),
    "rbffd_status_str": (C.c_char_p, [C.c_int]),
    "rbffd_last_error": (C.c_char_p, []),
    "rbffd_fp64_peak": (C.c_int, [vp, C.POINTER(C.c_double)]),
    "rbffd_fp64_mma_peak": (C.c_int, [vp, C.POINTER(C.c_double)]),
    "rbffd_memory_pool_config": (C.c_int, [C.c_int64]),
    "rbffd_release_memory": (C.c_int, []),
    "rbffd_memory_stats": (C.c_int, [C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
}

_lock = threading.Lock()
_handle = None


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load (building first if needed) the C-ABI library.  Raises if absent."""
    global _handle
    with _lock:
        if _handle is not None:
            return _handle
        path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"RBF-FD CUDA library not found at {path}")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _handle = lib
        return lib


class RbffdError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load(build=False)
        msg = lib.rbffd_last_error().decode(errors="replace")
        super().__init__(f"{where}: {lib.rbffd_status_str(status).decode()} ({status}): {msg}")
        self.status = status


def check(status: int, where: str, allow=()):
    if status != OK and status not in allow:
        raise RbffdError(status, where)
    return status

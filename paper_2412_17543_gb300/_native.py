"""ctypes declarations of the C ABI in include/dd_solver.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdd_gb300.so")

DD_OK, DD_INVALID_ARG, DD_OOM, DD_CUDA_ERROR, DD_SINGULAR_LOCAL, DD_NOT_CONVERGED, DD_BREAKDOWN, DD_TIMEOUT = range(8)
STATUS_NAMES = ["DD_OK", "DD_INVALID_ARG", "DD_OOM", "DD_CUDA_ERROR", "DD_SINGULAR_LOCAL", "DD_NOT_CONVERGED",
                "DD_BREAKDOWN", "DD_TIMEOUT"]
WEIGHTS = {"card": 0, "diag": 1}
PREC = {"fp64": 0, "fp32": 1, "df64": 2}
STRATEGY = {"B1": 1, "B2": 2, "B3": 3, "B4": 4}
LOCAL = {"auto": 0, "dense": 1, "fdm": 2}
ENS_NMM = {"auto": 0, "simt": 1, "tc": 2, "bf16x3": 3}
EIG = {"dense": 0, "lobpcg": 1}


class MeshDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("xc", ctypes.POINTER(ctypes.c_double)), ("yc", ctypes.POINTER(ctypes.c_double)),
                ("zc", ctypes.POINTER(ctypes.c_double)), ("coef", ctypes.POINTER(ctypes.c_double)),
                ("sub_x", ctypes.c_int32), ("sub_y", ctypes.c_int32), ("sub_z", ctypes.c_int32),
                ("dirichlet_faces", ctypes.c_uint32)]


class Options(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("coarse_group", ctypes.c_int32),
                ("use_corners", ctypes.c_int32), ("use_edges", ctypes.c_int32), ("use_faces", ctypes.c_int32),
                ("adaptive", ctypes.c_int32), ("tau", ctypes.c_double), ("max_eig_per_face", ctypes.c_int32),
                ("weights", ctypes.c_int32), ("precond_prec", ctypes.c_int32), ("schur_prec", ctypes.c_int32),
                ("flexible", ctypes.c_int32), ("reorth", ctypes.c_int32), ("stop_rhs_norm", ctypes.c_int32),
                ("maxit", ctypes.c_int32), ("local_solver", ctypes.c_int32),
                ("ens_nmm", ctypes.c_int32), ("ens_elem_rc", ctypes.c_int32), ("ens_fdm_rc", ctypes.c_int32),
                ("loop_graph", ctypes.c_int32), ("zero_initial_guess", ctypes.c_int32),
                ("adaptive_solver", ctypes.c_int32), ("lobpcg_iters", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("n_free", ctypes.c_int64), ("n_gamma", ctypes.c_int64), ("n_sub", ctypes.c_int32),
                ("n_coarse", ctypes.c_int32), ("n_adaptive", ctypes.c_int32), ("n_sub2", ctypes.c_int32),
                ("n_coarse3", ctypes.c_int32), ("local_solver", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("setup_seconds", ctypes.c_double), ("ens_nmm", ctypes.c_int32), ("ens_nmm_ms", ctypes.c_float * 3),
                ("ens_elem_rc", ctypes.c_int32), ("ens_fdm_rc", ctypes.c_int32), ("neumann", ctypes.c_int32),
                ("symv_slots", ctypes.c_int32), ("schur_threads", ctypes.c_int32),
                ("tune_symv_ms", ctypes.c_float * 3), ("tune_kii_ms", ctypes.c_float * 3),
                ("tune_schur_ms", ctypes.c_float * 3)]


class KernelProf(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("launches", ctypes.c_int64), ("alg_bytes", ctypes.c_double),
                ("alg_flops", ctypes.c_double)]


PROF_CLASSES = ["KIIinv_apply", "symv_N", "schur_apply", "precond_apply", "recycle_update", "ens_schur_apply",
                "ens_precond_apply", "ens_N", "deflation"]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("rel_res0", ctypes.c_double), ("rel_res", ctypes.c_double),
                ("recycled_k", ctypes.c_int32), ("frozen", ctypes.c_int32), ("ms", ctypes.c_float)]


# every function declared in include/dd_solver.h with (restype, argtypes)
_P = ctypes.c_void_p
_D = ctypes.c_double
SIGNATURES = {
    "dd_default_options": (ctypes.c_int, [ctypes.POINTER(Options)]),
    "dd_abi_struct_sizes": (None, [ctypes.POINTER(ctypes.c_size_t)]),
    "dd_setup": (ctypes.c_int, [ctypes.POINTER(MeshDesc), ctypes.POINTER(Options), _P, ctypes.POINTER(_P)]),
    "dd_destroy": (None, [_P]),
    "dd_last_error": (ctypes.c_char_p, []),
    "dd_plan": (ctypes.c_int, [ctypes.POINTER(MeshDesc), ctypes.POINTER(Options), ctypes.POINTER(Info),
                               ctypes.POINTER(ctypes.c_int64), ctypes.c_int64]),
    "dd_get_info": (ctypes.c_int, [_P, ctypes.POINTER(Info)]),
    "dd_interface_nodes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "dd_schur_apply": (ctypes.c_int, [_P, _P, _P, _P]),
    "dd_precond_apply": (ctypes.c_int, [_P, _P, _P, _P]),
    "dd_condense": (ctypes.c_int, [_P, _P, _P, _P]),
    "dd_recover": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "dd_schur_apply_noalloc": (ctypes.c_int, [_P, _P, _P, _P]),
    "dd_selftest_bounded_wait": (ctypes.c_int, [_P, ctypes.c_int64, _P]),
    "dd_recycle_create": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _D, ctypes.POINTER(_P)]),
    "dd_recycle_destroy": (None, [_P]),
    "dd_solve": (ctypes.c_int, [_P, _P, _P, _D, _P, ctypes.POINTER(Stats), _P]),
    "dd_adjoint": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int32, _D, _P, ctypes.POINTER(Stats), _P]),
    "dd_coef_mismatch": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.POINTER(_D), _P]),
    "dd_profile": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(KernelProf), ctypes.POINTER(ctypes.c_int64), _P]),
    "dd_recycle_export": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_size_t)]),
    "dd_recycle_import": (ctypes.c_int, [_P, _P, ctypes.c_size_t, ctypes.POINTER(_P)]),
    "dd_recycle_create_batch": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _D, ctypes.POINTER(_P)]),
    "dd_solve_batch": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _D, _P, ctypes.POINTER(Stats), _P]),
    "dd_schur_apply_batch": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P]),
    "dd_precond_apply_batch": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P]),
}

ENSEMBLE_WIDTH = 32  # DD_ENSEMBLE_WIDTH

_lib = None


def load() -> ctypes.CDLL:
    """Loads the in-tree native library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"native library {LIB_PATH} is missing: run __graft_entry__.build() "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class DDError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = lib.dd_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES[code] if 0 <= code < len(STATUS_NAMES) else code}: {msg}")
        self.code = code


def check(code: int, where: str, allow=(DD_OK,)):
    if code not in allow:
        raise DDError(code, where)
    return code

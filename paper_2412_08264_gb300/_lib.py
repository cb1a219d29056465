"""ctypes declarations of the C ABI in include/bl.h and the library loader.

Argument marshalling only: every computation happens in libbl.so.  Loading
fails with an exception when the library has not been built; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libbl.so")

BL_OK, BL_EINVAL, BL_ENOMEM, BL_ECUDA, BL_ENOCONV, BL_EBREAKDOWN, BL_ESTATE = range(7)
STATUS_NAMES = {0: "BL_OK", 1: "BL_EINVAL", 2: "BL_ENOMEM", 3: "BL_ECUDA", 4: "BL_ENOCONV",
                5: "BL_EBREAKDOWN", 6: "BL_ESTATE"}
BL_REG_TV, BL_REG_FOE = 0, 1
BL_PHI = {"charbonnier": 0, "sq": 1, "log1p": 2}
BL_FP32, BL_FP64 = 0, 1
BL_SOLVE_CG, BL_SOLVE_RCG, BL_SOLVE_MINRES, BL_SOLVE_RMINRES = 0, 1, 2, 3
BL_STOP_RESID, BL_STOP_NSC = 0, 1
BL_RECYCLE = {"ritz": 0, "hritz": 1, "rgsv": 2}
BL_SIZE = {"S": 0, "L": 1, "M": 2}
BL_SIDE = {"R": 0, "L": 1, "M": 2}
BL_REFRESH = {"outer": 0, "inner": 1}
BL_STORE_NONE, BL_STORE_RECENT, BL_STORE_LANCZOS = 0, 1, 2
KERNEL_CLASSES = ["hvp", "hvp_multi", "grad", "jw", "krylov", "lbfgs", "gram", "gemm", "dense", "other",
                  "krylov_vec"]


class PairDesc(C.Structure):
    _fields_ = [("height", C.c_int32), ("width", C.c_int32), ("blur_sigma", C.c_double),
                ("blur_radius", C.c_int32), ("mask", C.c_void_p)]


class RegDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_filters", C.c_int32), ("filter_size", C.c_int32),
                ("phi", C.c_int32), ("phi_eps", C.c_double), ("l2_eps", C.c_double),
                ("precision", C.c_int32), ("max_recycle", C.c_int32), ("max_basis", C.c_int32)]


class LbfgsOpts(C.Structure):
    _fields_ = [("max_iters", C.c_int32), ("history", C.c_int32), ("gtol", C.c_double),
                ("gtol_relative", C.c_int32), ("max_backtrack", C.c_int32), ("armijo_slack", C.c_double),
                ("graph", C.c_int32)]


class KrylovOpts(C.Structure):
    _fields_ = [("method", C.c_int32), ("stop", C.c_int32), ("tol", C.c_double),
                ("relative", C.c_int32), ("maxit", C.c_int32), ("store_basis", C.c_int32),
                ("warm_start", C.c_int32), ("graph", C.c_int32)]


class RecycleOpts(C.Structure):
    _fields_ = [("kind", C.c_int32), ("size", C.c_int32), ("side", C.c_int32), ("s", C.c_int32),
                ("variant", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("resid", C.c_double),
                ("nsc_est", C.c_double), ("rhs_norm", C.c_double)]


EXPORTS = {
    "bl_problem_create": (C.c_int, [C.POINTER(PairDesc), C.c_int32, C.POINTER(RegDesc), C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "bl_problem_destroy": (None, [C.c_void_p]),
    "bl_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "bl_num_params": (C.c_int32, [C.c_void_p]),
    "bl_num_pixels": (C.c_int64, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32]),
    "bl_set_data": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.c_void_p, C.c_void_p]),
    "bl_forward": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.c_void_p, C.c_void_p]),
    "bl_set_point": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.c_void_p, C.c_void_p]),
    "bl_lower_solve": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.c_void_p,
                                 C.POINTER(LbfgsOpts), C.c_void_p, C.POINTER(SolveInfo)]),
    "bl_gradient": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.c_void_p, C.c_void_p,
                              C.c_void_p, C.c_void_p]),
    "bl_hvp": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.c_void_p, C.c_void_p]),
    "bl_ritz_update": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.POINTER(RecycleOpts)]),
    "bl_hessian_solve": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.POINTER(KrylovOpts),
                                   C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.POINTER(SolveInfo)]),
    "bl_hypergrad": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.c_void_p, C.c_void_p,
                               C.c_void_p, C.POINTER(C.c_double)]),
    "bl_recycle_dim": (C.c_int32, [C.c_void_p, C.c_int32]),
    "bl_basis_size": (C.c_int32, [C.c_void_p, C.c_int32]),
    "bl_recycle_export": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_size_t)]),
    "bl_recycle_import": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t]),
    "bl_launch_count": (C.c_int64, [C.c_void_p]),
    "bl_graph_used": (C.c_int32, [C.c_void_p]),
    "bl_hvp_tma": (C.c_int32, [C.c_void_p]),
    "bl_hvp_tile": (C.c_int32, [C.c_void_p, C.c_int32]),
    "bl_set_hvp_tile": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "bl_profile_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "bl_profile_read": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int64)]),
    "bl_profile_read_bytes": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64)]),
    "bl_last_error": (C.c_char_p, []),
    "bl_jw_fp32_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int32,
                                    C.c_int32, C.c_int32, C.c_double, C.c_void_p, C.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libbl.so and declare every exported symbol; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libbl.so not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'` (no fallback exists)")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class BLError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str, allow=(BL_OK,)):
    if status in allow:
        return status
    raise BLError(status, where, load().bl_last_error().decode(errors="replace"))

"""ctypes declarations for libbddc.so (the C ABI in include/bddc.h).

The shared library is built in-tree by `paper_2410_14786_gb300.build`. This
module raises on import failure: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libbddc.so")

OK = 0
NOT_CONVERGED = 1
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_CUDA = -3
ERR_SINGULAR = -4
ERR_TIMEOUT = -5
ERR_BREAKDOWN = -6
ERR_NO_DEVICE = -7

PREC_FP64, PREC_FP32, PREC_BF16, PREC_TF32 = 0, 1, 2, 3
TC_AUTO, TC_ON, TC_OFF = 0, 1, 2
CORNERS, EDGES, FACES = 1, 2, 4
COARSE_AUTO, COARSE_DENSE, COARSE_SPARSE, COARSE_CG = 0, 1, 2, 3
LOCAL_DENSE, LOCAL_SPARSE = 0, 1

EXPORTED = [
    "bddc_setup", "bddc_apply", "bddc_matvec", "bddc_rhs", "bddc_pcg_solve",
    "bddc_pcg_solve_host", "bddc_coarse_vectors", "bddc_query", "bddc_profile_apply",
    "bddc_destroy", "bddc_strerror", "bddc_last_error", "bddc_setup_inspect",
    "bddc_apply_static_scratch", "bddc_elem_grad", "bddc_autotune", "bddc_get_tuning", "bddc_set_tuning",
    "bddc_pcg_history", "bddc_test_coarse_stall", "bddc_clear_device_error",
]


class Tuning(C.Structure):
    _fields_ = [("gemv_stage_kb_interior", C.c_int32), ("gemv_stage_kb_interface", C.c_int32),
                ("coarse_rowblock_min_nrhs", C.c_int32), ("gemv_rows_interior", C.c_int32),
                ("gemv_rows_interface", C.c_int32), ("coarse_overlap", C.c_int32),
                ("sym_stages_interior", C.c_int32), ("sym_stages_interface", C.c_int32),
                ("interior_block_height", C.c_int32), ("coarse_level_launches", C.c_int32)]


class Problem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("ne", C.c_int32), ("elem_sigma", C.POINTER(C.c_double)),
                ("elem_subdomain", C.POINTER(C.c_int32)), ("n_sub", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("constraints", C.c_uint32), ("nrhs_max", C.c_int32),
                ("n_threads", C.c_int32), ("device", C.c_int32), ("coarse", C.c_int32),
                ("no_graph", C.c_int32), ("phi_fp64", C.c_int32),
                ("tensor_cores", C.c_int32), ("coarse_blocks", C.c_int32), ("full_operators", C.c_int32),
                ("history", C.c_int32), ("coarse_cg_maxit", C.c_int32), ("coarse_cg_rtol", C.c_double),
                ("local_solver", C.c_int32), ("local_leaf", C.c_int32)]


class Info(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "n_nodes", "n_free", "n_interior", "n_interface_nodes", "n_sub", "n_c",
        "n_corners", "n_edges", "n_faces", "sum_ni", "sum_nI2", "sum_nG2", "sum_nG_nc",
        "max_ni", "operator_bytes", "coarse_bytes", "device_bytes", "apply_bytes_1rhs",
        "interior_op_bytes", "interface_op_bytes", "n_interface_copies", "kernel_launches",
        "coarse_factor_entries", "coarse_update_total", "coarse_levels")] + [
        ("setup_seconds", C.c_double), ("precision", C.c_int32), ("error_subdomain", C.c_int32),
        ("device_error", C.c_int32), ("phi_precision", C.c_int32),
        ("tensor_cores", C.c_int32), ("solve_graph", C.c_int32), ("symmetric_operators", C.c_int32),
        ("coarse_cg_iters", C.c_int32), ("local_solver", C.c_int32), ("interior_levels", C.c_int32),
        ("interior_factor_entries", C.c_int64)]


class BDDCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libbddc status {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libbddc.so not built at {path}; run paper_2410_14786_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i32, dbl = C.c_void_p, C.c_int32, C.c_double
    pi32, pdbl = C.POINTER(C.c_int32), C.POINTER(C.c_double)
    sig = {
        "bddc_setup": (C.c_int, [C.POINTER(Problem), C.POINTER(Options), C.POINTER(vp)]),
        "bddc_apply": (C.c_int, [vp, vp, vp, i32, vp]),
        "bddc_apply_static_scratch": (C.c_int, [vp, vp, vp, i32, vp]),
        "bddc_matvec": (C.c_int, [vp, vp, vp, i32, vp]),
        "bddc_elem_grad": (C.c_int, [vp, vp, vp, vp, i32, vp]),
        "bddc_autotune": (C.c_int, [vp, i32, vp, vp]),
        "bddc_get_tuning": (C.c_int, [vp, vp]),
        "bddc_set_tuning": (C.c_int, [vp, vp]),
        "bddc_rhs": (C.c_int, [vp, vp, vp, i32, vp]),
        "bddc_pcg_solve": (C.c_int, [vp, vp, vp, i32, dbl, i32, pi32, pdbl, vp]),
        "bddc_pcg_solve_host": (C.c_int, [vp, vp, vp, i32, dbl, i32, pi32, pdbl, vp]),
        "bddc_coarse_vectors": (C.c_int, [vp, vp, vp, i32, vp]),
        "bddc_pcg_history": (C.c_int, [vp, i32, i32, pdbl, pdbl, pdbl]),
        "bddc_test_coarse_stall": (C.c_int, [vp, i32, C.c_int64]),
        "bddc_clear_device_error": (C.c_int, [vp]),
        "bddc_query": (C.c_int, [vp, C.POINTER(Info)]),
        "bddc_profile_apply": (C.c_int, [vp, vp, vp, i32, i32, pdbl, vp]),
        "bddc_setup_inspect": (C.c_int, [C.POINTER(Problem), C.POINTER(Options), i32, C.POINTER(Info), pdbl,
                                         C.c_int64]),
        "bddc_destroy": (None, [vp]),
        "bddc_strerror": (C.c_char_p, [C.c_int]),
        "bddc_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_LIB = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


def check(code: int, allow=(OK,)) -> int:
    if code in allow:
        return code
    L = lib()
    detail = L.bddc_last_error().decode() or L.bddc_strerror(code).decode()
    raise BDDCError(code, detail)

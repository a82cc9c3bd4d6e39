"""ctypes declarations of the C ABI in include/dlr.h (argument marshalling only;
all computation happens in libdlr_gb300.so)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdlr_gb300.so")

DLR_OK, DLR_EINVAL, DLR_ENOMEM, DLR_ENOTCONV = 0, -1, -2, -3
DLR_ESINGULAR, DLR_ETIMEOUT, DLR_ENONPOS, DLR_ECUDA = -4, -5, -6, -7
DLR_FP64, DLR_MIXED = 0, 1
DLR_SEL_QDEIM, DLR_SEL_DEIM = 0, 1
DLR_METHOD_DLR, DLR_METHOD_SN = 0, 1

ERROR_NAMES = {DLR_EINVAL: "EINVAL", DLR_ENOMEM: "ENOMEM", DLR_ENOTCONV: "ENOTCONV",
               DLR_ESINGULAR: "ESINGULAR", DLR_ETIMEOUT: "ETIMEOUT",
               DLR_ENONPOS: "ENONPOS", DLR_ECUDA: "ECUDA"}

# every entry point declared in include/dlr.h
SYMBOLS = ["dlr_create", "dlr_step", "dlr_step_batch", "dlr_autotune", "dlr_set_split", "dlr_debug_lose_edge",
           "dlr_get_T", "dlr_set_T", "dlr_get_factors", "dlr_set_factors", "dlr_get_quadrature", "dlr_get_selected",
           "dlr_get_psi", "dlr_set_psi",
           "dlr_get_stats", "dlr_set_timing", "dlr_set_edge_inflow", "dlr_footprint_bytes",
           "dlr_destroy", "dlr_last_error", "dlr_sweep", "dlr_sweep_noalloc", "dlr_debug_tc_gemm"]


class DlrProblem(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("lx", C.c_double), ("ly", C.c_double),
                ("n_polar", C.c_int32), ("n_azim", C.c_int32), ("rank", C.c_int32),
                ("dt", C.c_double), ("c", C.c_double), ("a_rad", C.c_double),
                ("sigma", C.POINTER(C.c_double)), ("rho_cv", C.POINTER(C.c_double)),
                ("T0", C.POINTER(C.c_double)), ("T_edge", C.c_double * 4),
                ("precision", C.c_int32), ("selection", C.c_int32), ("augment", C.c_int32),
                ("si_tol", C.c_double), ("si_max_iter", C.c_int32), ("si_fixed_iters", C.c_int32),
                ("allow_nonpositive", C.c_int32), ("method", C.c_int32),
                ("sigma_texp", C.c_double), ("cv_texp", C.c_double), ("T_ref", C.c_double),
                ("dsa", C.c_int32), ("dsa_tol", C.c_double), ("dsa_max_iter", C.c_int32),
                ("reflect", C.c_int32 * 4), ("sweep_mode", C.c_int32),
                ("element", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class DlrRuntime(C.Structure):
    _fields_ = [("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("ctx", C.c_void_p), ("hbm_budget", C.c_size_t)]


class DlrStats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("si_iters_total", C.c_int64),
                ("cell_angle_updates", C.c_int64), ("si_iters_last", C.c_int32),
                ("status", C.c_int32), ("ms_si_total", C.c_double), ("ms_step_total", C.c_double),
                ("si_launches", C.c_int64), ("kernel_launches", C.c_int64),
                ("nonpositive_cells", C.c_int64), ("dsa_iters_total", C.c_int64),
                ("sweep_grouped", C.c_int32),
                ("refl_passes_last", C.c_int32)]


_lib = None


def load() -> C.CDLL:
    """Loads the in-tree library; raises if it has not been built (there is
    no fallback implementation)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2601_18705_gb300.build` (needs nvcc)")
    L = C.CDLL(LIB_PATH)
    H = C.c_void_p
    dp = C.POINTER(C.c_double)
    L.dlr_create.argtypes = [C.POINTER(DlrProblem), C.POINTER(DlrRuntime), C.POINTER(H)]
    L.dlr_step.argtypes = [H, C.c_int32]
    L.dlr_step_batch.argtypes = [C.POINTER(H), C.c_int32, C.c_int32]
    L.dlr_autotune.argtypes = [C.POINTER(H), C.c_int32, C.c_int32, C.c_int32, dp, dp]
    L.dlr_set_split.argtypes = [C.POINTER(H), C.c_int32, C.c_double]
    L.dlr_debug_lose_edge.argtypes = [C.POINTER(H), C.c_int32]
    L.dlr_get_T.argtypes = [H, C.c_void_p, C.c_int32]
    L.dlr_set_T.argtypes = [H, C.c_void_p, C.c_int32]
    L.dlr_get_factors.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32), C.c_int32]
    L.dlr_set_factors.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
    L.dlr_get_quadrature.argtypes = [H, dp, dp]
    L.dlr_get_selected.argtypes = [H, C.POINTER(C.c_int32)]
    L.dlr_get_psi.argtypes = [H, C.c_void_p, C.c_int32]
    L.dlr_set_psi.argtypes = [H, C.c_void_p, C.c_int32]
    L.dlr_get_stats.argtypes = [H, C.POINTER(DlrStats)]
    L.dlr_set_timing.argtypes = [H, C.c_int32]
    L.dlr_set_edge_inflow.argtypes = [H, C.c_int32, C.c_double]
    L.dlr_footprint_bytes.argtypes = [C.POINTER(DlrProblem)]
    L.dlr_footprint_bytes.restype = C.c_size_t
    L.dlr_destroy.argtypes = [H]
    L.dlr_destroy.restype = None
    L.dlr_last_error.restype = C.c_char_p
    L.dlr_sweep.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_int32, dp, dp,
                            C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    L.dlr_sweep_noalloc.argtypes = L.dlr_sweep.argtypes
    L.dlr_debug_tc_gemm.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                    C.c_void_p]
    for name in SYMBOLS:
        if name not in ("dlr_destroy", "dlr_last_error", "dlr_footprint_bytes"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


class DlrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(rc: int) -> None:
    if rc != DLR_OK:
        raise DlrError(rc, load().dlr_last_error().decode(errors="replace"))

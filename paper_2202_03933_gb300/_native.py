"""ctypes declarations of the C ABI in ``include/mortar.h`` (marshalling only).

Loading fails loudly when the CUDA library has not been built: there is no
CPU fallback on the product path.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmortar_gb300.so")

MORTAR_OK = 0
STATUS = {0: "MORTAR_OK", -1: "MORTAR_ERR_INVALID_ARG", -2: "MORTAR_ERR_DEGENERATE",
          -3: "MORTAR_ERR_NEWTON", -4: "MORTAR_ERR_CAPACITY", -5: "MORTAR_ERR_CUDA",
          -6: "MORTAR_ERR_OOM", -7: "MORTAR_ERR_TIMEOUT", -8: "MORTAR_ERR_STATE",
          -9: "MORTAR_ERR_NOT_BUILT"}

# every symbol include/mortar.h declares (checked by the CPU test-suite)
EXPORTS = (
    "mortar_default_options", "mortar_create", "mortar_destroy", "mortar_set_interface",
    "mortar_set_batch", "mortar_set_coordinates", "mortar_search", "mortar_get_pairs",
    "mortar_evaluate", "mortar_csr_size", "mortar_csr_copy", "mortar_get_pair_blocks",
    "mortar_weighted_gap_grad", "mortar_run_graph", "mortar_get_gradient", "mortar_get_stats",
    "mortar_set_timing", "mortar_set_launch", "mortar_status_string", "mortar_probe_dfma",
    "mortar_integrate_pairs_static", "mortar_autotune", "mortar_tangent", "mortar_tangent_copy",
    "mortar_contact_terms", "mortar_set_watchdog",
)


class MortarError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed: {STATUS.get(code, code)}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("lm", ctypes.c_int32), ("d_domain", ctypes.c_int32),
                ("newton_max_iter", ctypes.c_int32), ("block_size", ctypes.c_int32),
                ("search_inflation", ctypes.c_double), ("newton_tol", ctypes.c_double),
                ("clip_tol_rel", ctypes.c_double), ("merge_tol_rel", ctypes.c_double),
                ("area_tol_rel", ctypes.c_double), ("bin_margin", ctypes.c_double),
                ("integration", ctypes.c_int32), ("element_rule_n", ctypes.c_int32),
                ("facing_test", ctypes.c_int32), ("watchdog_us", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "n_interfaces", "n_pairs", "n_nonempty", "n_gauss_points", "n_cells", "n_newton_fail",
        "n_xi_out_of_range", "n_clip_overflow", "nnz_D", "nnz_M", "n_bins", "reruns", "graph_kernels", "fused")] + \
        [(n, ctypes.c_float) for n in ("ms_search", "ms_integrate", "ms_assemble", "ms_adjoint",
                                       "ms_adjoint_pairs", "ms_total", "eta_t", "ms_tangent")] + \
        [("nnzb_K", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded CUDA library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"CUDA library {LIB_PATH} is missing; build it with "
                    "`python -m paper_2202_03933_gb300.build` (needs nvcc, sm_103a)")
            L = ctypes.CDLL(LIB_PATH)
            P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            pp = ctypes.POINTER(ctypes.c_void_p)
            sig = {
                "mortar_default_options": [ctypes.POINTER(Options)],
                "mortar_create": [pp, ctypes.POINTER(Options), P],
                "mortar_set_interface": [P, P, i64, P, i64, i32, P, i64, P, i64, i32, i32],
                "mortar_set_batch": [P, i32, P, P, P, P, P, P, i32, P, P, i32, i32],
                "mortar_set_coordinates": [P, P, P, i32],
                "mortar_search": [P, ctypes.POINTER(i64)],
                "mortar_get_pairs": [P, P, P, i64, i32],
                "mortar_evaluate": [P],
                "mortar_csr_size": [P, i32, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)],
                "mortar_csr_copy": [P, i32, P, P, P, i64, i32],
                "mortar_get_pair_blocks": [P, P, P, P, i64, i32],
                "mortar_weighted_gap_grad": [P, P, ctypes.POINTER(f64), P, P, i32],
                "mortar_run_graph": [P, P, i32],
                "mortar_get_gradient": [P, ctypes.POINTER(f64), P, P, i32],
                "mortar_get_stats": [P, ctypes.POINTER(Stats)],
                "mortar_set_timing": [P, i32],
                "mortar_set_watchdog": [P, i32],
                "mortar_set_launch": [P, i32, i32, i32, i32],
                "mortar_autotune": [P, P, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                    ctypes.POINTER(ctypes.c_float)],
                "mortar_tangent": [P, P, P, i32, i32, ctypes.POINTER(i64)],
                "mortar_tangent_copy": [P, P, P, P, i64, i32],
                "mortar_contact_terms": [P, P, f64, P, P, P, P, i32],
                "mortar_status_string": [ctypes.c_int],
                "mortar_probe_dfma": [P, i32, i32, i64, i32, P],
                "mortar_integrate_pairs_static": [ctypes.POINTER(Options), P, P, i64, P, i64, i32,
                                                  P, i64, P, i64, i32, P, P, i64, P, P, P],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_char_p if name == "mortar_status_string" else ctypes.c_int
            L.mortar_destroy.argtypes = [P]
            L.mortar_destroy.restype = None
            _lib = L
    return _lib


def call(name: str, *args, ok=(MORTAR_OK,)) -> int:
    r = getattr(lib(), name)(*args)
    if r not in ok:
        raise MortarError(name, r)
    return r

"""ctypes declarations of the C ABI in include/su2fft.h.

Argument marshalling only: every step of the transform runs in the CUDA
library.  Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libsu2fft.so")

SU2_OK = 0
STATUS_NAMES = {
    0: "SU2_OK", 1: "SU2_ERR_INVALID_ARG", 2: "SU2_ERR_UNSUPPORTED", 3: "SU2_ERR_OOM",
    4: "SU2_ERR_CUDA", 5: "SU2_ERR_TIMEOUT", 6: "SU2_ERR_WORKSPACE", 7: "SU2_ERR_ALIGNMENT",
}
DTYPES = {"c64": 0, "c128": 1}
ALGOS = {"auto": 0, "fp64": 1, "fp32": 2, "tc_bf16x3": 3}
WEIGHTS = {"cc": 0, "riemann": 1}


class PlanDesc(ctypes.Structure):
    _fields_ = [
        ("num_functions", ctypes.c_int),
        ("N", ctypes.POINTER(ctypes.c_int)),
        ("N_uniform", ctypes.c_int),
        ("dtype", ctypes.c_int),
        ("algo", ctypes.c_int),
        ("weights", ctypes.c_int),
        ("flags", ctypes.c_uint),
        ("device", ctypes.c_int),
    ]


class SU2Error(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        super().__init__(f"{fn} failed: {STATUS_NAMES.get(status, status)}")


_lib = None

# (name, restype, argtypes) for every entry point of include/su2fft.h
FLAG_CUDA_GRAPH = 0x1
FLAG_AUTOTUNE = 0x2
FLAG_FULL_GROUP = 0x4
FLAG_LITERAL_GRID = 0x8
FLAG_PERSISTENT = 0x10

SIGNATURES = [
    ("su2_plan", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(PlanDesc)]),
    ("su2_workspace_size", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    ("su2_plan_persistent", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    ("su2_grid_offset", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    ("su2_coeff_offset", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    ("su2_plane_offset", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    ("su2_grid_elems", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    ("su2_coeff_elems", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    ("su2_num_coeffs", ctypes.c_size_t, [ctypes.c_int]),
    ("su2_forward", ctypes.c_int, [ctypes.c_void_p] * 5),
    ("su2_forward_stage1", ctypes.c_int, [ctypes.c_void_p] * 4),
    ("su2_forward_stage2", ctypes.c_int, [ctypes.c_void_p] * 4),
    ("su2_forward_pipelined", ctypes.c_int, [ctypes.c_void_p] * 7),
    ("su2_selftest_bounded_wait", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("su2_forward_stage2_depth", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 3),
    ("su2_forward_noalloc", ctypes.c_int, [ctypes.c_void_p] * 4),
    ("su2_forward_stage1_slab", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 4),
    ("su2_forward_stage2_rows", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
     + [ctypes.c_void_p] * 3),
    ("su2_inverse", ctypes.c_int, [ctypes.c_void_p] * 5),
    ("su2_backward", ctypes.c_int, [ctypes.c_void_p] * 5),
    ("su2_sync_status", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("su2_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("su2_status_string", ctypes.c_char_p, [ctypes.c_int]),
]


def load(path: str | None = None):
    """Load libsu2fft.so (built in-tree by paper_2605_23923_gb300.build)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(
            f"CUDA library not built: {p} is missing. Run paper_2605_23923_gb300.build.build() "
            "(needs nvcc); there is no CPU fallback.")
    lib = ctypes.CDLL(p)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def check(fn: str, status: int):
    if status != SU2_OK:
        raise SU2Error(fn, status)

"""ctypes binding of libbpdn (include/bpdn.h): argument marshalling only.

Every computation happens in the CUDA library; if the library has not been built
(or fails to load) the import of the solver API raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

BPDN_OK = 0
BPDN_EINVAL, BPDN_ECUDA, BPDN_ESIZE, BPDN_EALIGN, BPDN_ESTATE = -1, -2, -3, -4, -5
STATUS_NAMES = {-1: "EINVAL", -2: "ECUDA", -3: "ESIZE", -4: "EALIGN", -5: "ESTATE"}

PX_NOT_CONVERGED = 1
PX_BT_LIMIT = 2
PX_NONFINITE = 4
PX_SUPPORT_OVERFLOW = 8
PX_KKT_FAIL = 16
PX_ZERO_SOLUTION = 32
PX_CERTIFIED = 64
PX_DEVICE_TIMEOUT = 128

MAX_N = 80
MAX_L = 65536
MAX_SMAX = 32
MAX_KSEL = 4
MAX_MOTION = 2

EXPORTED = [
    "bpdn_default_options", "bpdn_op_workspace_bytes", "bpdn_make_operator",
    "bpdn_destroy_operator", "bpdn_op_info", "bpdn_op_lipschitz", "bpdn_op_export",
    "bpdn_solve_workspace_bytes", "bpdn_solve", "bpdn_refit", "bpdn_refit_workspace_bytes",
    "bpdn_last_error", "bpdn_version",
    "bpdn_solve_noalloc", "bpdn_backward_workspace_bytes", "bpdn_backward",
    "bpdn_solve_ragged_workspace_bytes", "bpdn_solve_ragged_workspace_bytes_for", "bpdn_solve_ragged",
    "bpdn_select", "bpdn_make_operator_md", "bpdn_bench_peak", "bpdn_classify", "bpdn_classify_merge",
]


class Options(ctypes.Structure):
    """Mirror of bpdn_options."""
    _fields_ = [
        ("max_iter", ctypes.c_int32),
        ("tol", ctypes.c_float),
        ("c_alpha", ctypes.c_float),
        ("alpha0_scale", ctypes.c_float),
        ("precision", ctypes.c_int32),
        ("refit", ctypes.c_int32),
        ("s_max", ctypes.c_int32),
        ("max_bt", ctypes.c_int32),
        ("tile_pixels", ctypes.c_int32),
        ("refit_rounds", ctypes.c_int32),
        ("blocks", ctypes.c_int32),
        ("seed", ctypes.c_uint32),
        ("kernel", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 3),
    ]


class BPDNError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bpdn error {code} ({STATUS_NAMES.get(code, '?')}): {msg}")
        self.code = code


_lib = None


class Stack(ctypes.Structure):
    """Mirror of bpdn_stack."""
    _fields_ = [
        ("op", ctypes.c_void_p),
        ("d_g", ctypes.c_void_p),
        ("P", ctypes.c_int64),
        ("d_lambda", ctypes.c_void_p),
        ("lambda_per_pixel", ctypes.c_int32),
        ("d_x", ctypes.c_void_p),
        ("d_support", ctypes.c_void_p),
        ("d_nsupp", ctypes.c_void_p),
        ("d_status", ctypes.c_void_p),
        ("d_iters", ctypes.c_void_p),
        ("d_nbt", ctypes.c_void_p),
        ("tile_pixels", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
    ]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libbpdn.so (raises if it is missing and build_if_missing is False)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libbpdn is not built ({path} missing): run "
                               "`python -m paper_1805_01759_gb300.build` (needs nvcc)")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, sz, i32, i64, dbl = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    op_t = ctypes.c_void_p
    optp = ctypes.POINTER(Options)
    i32p = ctypes.POINTER(ctypes.c_int32)
    dblp = ctypes.POINTER(ctypes.c_double)
    lib.bpdn_default_options.argtypes = [optp]
    lib.bpdn_default_options.restype = None
    lib.bpdn_op_workspace_bytes.argtypes = [i32, i32]
    lib.bpdn_op_workspace_bytes.restype = sz
    lib.bpdn_make_operator.argtypes = [dblp, i32, dbl, dbl, dbl, dbl, i32, vp, sz, vp,
                                       ctypes.POINTER(op_t)]
    lib.bpdn_make_operator.restype = ctypes.c_int
    lib.bpdn_make_operator_md.argtypes = [dblp, i32, dbl, dbl, dbl, dbl, i32, i32, dblp, dblp, dblp,
                                          ctypes.POINTER(i32), vp, sz, vp, ctypes.POINTER(op_t)]
    lib.bpdn_make_operator_md.restype = ctypes.c_int
    lib.bpdn_destroy_operator.argtypes = [op_t]
    lib.bpdn_destroy_operator.restype = None
    lib.bpdn_op_info.argtypes = [op_t, i32p, i32p, dblp, dblp]
    lib.bpdn_op_info.restype = ctypes.c_int
    lib.bpdn_op_lipschitz.argtypes = [op_t]
    lib.bpdn_op_lipschitz.restype = dbl
    lib.bpdn_op_export.argtypes = [op_t, i32, vp, sz, vp]
    lib.bpdn_op_export.restype = ctypes.c_int
    lib.bpdn_solve_workspace_bytes.argtypes = [op_t, i64, optp]
    lib.bpdn_solve_workspace_bytes.restype = sz
    lib.bpdn_solve.argtypes = [op_t, vp, i64, vp, i32, optp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    lib.bpdn_solve.restype = ctypes.c_int
    lib.bpdn_refit.argtypes = [op_t, vp, i64, vp, i32, optp, vp, vp, vp, vp, vp, vp, sz, vp]
    lib.bpdn_refit_workspace_bytes.argtypes = [op_t, i64]
    lib.bpdn_refit_workspace_bytes.restype = sz
    lib.bpdn_refit.restype = ctypes.c_int
    lib.bpdn_solve_noalloc.argtypes = [op_t, vp, i64, vp, i32, optp, vp, vp, vp, vp, vp, vp, vp]
    lib.bpdn_solve_noalloc.restype = ctypes.c_int
    lib.bpdn_backward_workspace_bytes.argtypes = [op_t, i64]
    lib.bpdn_backward_workspace_bytes.restype = sz
    lib.bpdn_backward.argtypes = [op_t, i64, vp, i32, vp, vp, vp, vp, i32, vp, vp, vp, vp, sz, vp]
    lib.bpdn_backward.restype = ctypes.c_int
    lib.bpdn_solve_ragged_workspace_bytes.argtypes = [i32]
    lib.bpdn_solve_ragged_workspace_bytes.restype = sz
    lib.bpdn_solve_ragged_workspace_bytes_for.argtypes = [ctypes.POINTER(Stack), i32, optp]
    lib.bpdn_solve_ragged_workspace_bytes_for.restype = sz
    lib.bpdn_solve_ragged.argtypes = [ctypes.POINTER(Stack), i32, optp, vp, sz, vp]
    lib.bpdn_solve_ragged.restype = ctypes.c_int
    lib.bpdn_select.argtypes = [op_t, vp, i64, vp, vp, vp, vp, i32, i32, dbl, vp, vp, vp, vp]
    lib.bpdn_select.restype = ctypes.c_int
    lib.bpdn_last_error.argtypes = []
    lib.bpdn_classify.argtypes = [op_t, vp, i64, vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.bpdn_classify.restype = ctypes.c_int
    lib.bpdn_classify_merge.argtypes = [i64, vp, i32, vp, vp, vp, vp, vp, vp, vp]
    lib.bpdn_classify_merge.restype = ctypes.c_int
    lib.bpdn_bench_peak.argtypes = [i32, i32, i32, i64, vp, dblp, vp]
    lib.bpdn_bench_peak.restype = ctypes.c_int
    lib.bpdn_last_error.restype = ctypes.c_char_p
    lib.bpdn_version.argtypes = []
    lib.bpdn_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def check(rc: int) -> None:
    if rc != BPDN_OK:
        raise BPDNError(rc, load().bpdn_last_error().decode())


def default_options(**overrides) -> Options:
    opt = Options()
    load().bpdn_default_options(ctypes.byref(opt))
    for k, v in overrides.items():
        if not hasattr(opt, k):
            raise TypeError(f"unknown option {k}")
        setattr(opt, k, v)
    return opt

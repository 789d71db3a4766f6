"""The C ABI library (CPU only): it loads, exports every function the headers under
include/ declare, and rejects bad arguments with error codes before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1805_01759_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(bpdn_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    return _lib.load(build_if_missing=True)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.EXPORTED), set(names) ^ set(_lib.EXPORTED)


def test_options_struct_layout(lib):
    opt = _lib.default_options()
    assert ctypes.sizeof(_lib.Options) == 64
    assert opt.max_iter == 500 and abs(opt.tol - 1e-6) < 1e-12 and opt.c_alpha == 0.5
    assert opt.refit == 1 and opt.s_max == 32 and opt.precision == 0


def test_workspace_sizes(lib):
    assert lib.bpdn_op_workspace_bytes(25, 400) > 25 * 400 * 16
    assert lib.bpdn_op_workspace_bytes(0, 400) == 0
    assert lib.bpdn_op_workspace_bytes(25, 0) == 0
    assert lib.bpdn_op_workspace_bytes(81, 400) == 0 and lib.bpdn_op_workspace_bytes(80, 400) > 0
    assert lib.bpdn_op_workspace_bytes(25, 65537) == 0
    assert lib.bpdn_op_workspace_bytes(25, 1025) > 0
    assert lib.bpdn_op_workspace_bytes(25, 400) % 256 == 0


def test_argument_errors_without_gpu(lib):
    out = ctypes.c_void_p()
    b = np.zeros(25)
    dp = b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    # NULL output / workspace / baselines
    assert lib.bpdn_make_operator(dp, 25, 0.031, 7e5, -1.0, 1.0, 10, None, 0, None, None) == -1
    assert lib.bpdn_make_operator(dp, 25, 0.031, 7e5, -1.0, 1.0, 10, None, 0, None, ctypes.byref(out)) == -1
    assert b"NULL" in lib.bpdn_last_error()
    fake_ws = ctypes.c_void_p(256)
    assert lib.bpdn_make_operator(dp, 0, 0.031, 7e5, -1.0, 1.0, 10, fake_ws, 1 << 20, None, ctypes.byref(out)) == -3
    assert lib.bpdn_make_operator(dp, 25, -1.0, 7e5, -1.0, 1.0, 10, fake_ws, 1 << 20, None, ctypes.byref(out)) == -1
    assert lib.bpdn_make_operator(dp, 25, 0.031, 7e5, 1.0, -1.0, 10, fake_ws, 1 << 20, None, ctypes.byref(out)) == -1
    assert lib.bpdn_make_operator(dp, 25, 0.031, 7e5, -1.0, 1.0, 10, fake_ws, 16, None, ctypes.byref(out)) == -3
    assert lib.bpdn_make_operator(dp, 25, 0.031, 7e5, -1.0, 1.0, 10, ctypes.c_void_p(264), 1 << 20, None,
                                  ctypes.byref(out)) == -4
    b2 = b.copy()
    b2[3] = np.nan
    assert lib.bpdn_make_operator(b2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 25, 0.031, 7e5,
                                  -1.0, 1.0, 10, fake_ws, 1 << 20, None, ctypes.byref(out)) == -1
    # an invalid handle is rejected before any CUDA call
    opt = _lib.default_options()
    assert lib.bpdn_solve(None, None, 1, None, 0, ctypes.byref(opt), None, None, None, None, None, None,
                          None, 0, None) == -1
    assert lib.bpdn_refit(None, None, 1, None, 0, ctypes.byref(opt), None, None, None, None, None, None, 0,
                          None) == -1
    assert lib.bpdn_refit_workspace_bytes(None, 1 << 20) >= 460 * (1 << 20)
    assert lib.bpdn_op_info(None, None, None, None, None) == -1
    assert np.isnan(lib.bpdn_op_lipschitz(None))
    lib.bpdn_destroy_operator(None)  # ignored
    assert lib.bpdn_version().startswith(b"bpdn-gb300")


def test_ragged_host_checks():
    """bpdn_solve_ragged rejects bad arguments on the host, before touching a GPU."""
    from paper_1805_01759_gb300 import _lib
    lib = _lib.load()
    opt = _lib.default_options()
    assert lib.bpdn_solve_ragged_workspace_bytes(0) == 0
    assert lib.bpdn_solve_ragged_workspace_bytes(3) == 3 * 256
    arr3 = (_lib.Stack * 3)()
    for i, P in enumerate((10, 0, 1000)):
        arr3[i].P = P
    full = lib.bpdn_solve_ragged_workspace_bytes_for(arr3, 3, ctypes.byref(opt))
    assert full >= 3 * 256 + 460 * 1010
    opt0 = _lib.default_options(refit=0)
    assert lib.bpdn_solve_ragged_workspace_bytes_for(arr3, 3, ctypes.byref(opt0)) == 3 * 256
    assert lib.bpdn_solve_ragged(None, 0, ctypes.byref(opt), None, 0, None) == _lib.BPDN_OK
    assert lib.bpdn_solve_ragged(None, -1, ctypes.byref(opt), None, 0, None) == _lib.BPDN_EINVAL
    assert lib.bpdn_solve_ragged(None, 2, ctypes.byref(opt), None, 0, None) == _lib.BPDN_EINVAL
    arr = (_lib.Stack * 2)()
    assert lib.bpdn_solve_ragged(arr, 2, ctypes.byref(opt), None, 0, None) == _lib.BPDN_ESIZE


def test_select_host_checks():
    """bpdn_select rejects a missing operator on the host, before touching a GPU."""
    from paper_1805_01759_gb300 import _lib
    lib = _lib.load()
    assert lib.bpdn_select(None, None, 0, None, None, None, None, 16, 4, 0.0, None, None, None, None) == \
        _lib.BPDN_EINVAL
    assert _lib.MAX_KSEL == 4


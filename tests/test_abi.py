"""The C-ABI library loads and exports every function include/evd.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    text = (ROOT / "include" / "evd.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:evd_status_t|void|const char\*|int64_t|int)\s+(evd_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["evd_plan_create", "evd_plan_workspace_size", "evd_sbr", "evd_bulge_chase",
                     "evd_tridiag_solve", "evd_back_transform", "evd_syevd", "evd_syevd_batched",
                     "evd_plan_status", "evd_plan_destroy", "evd_status_string", "evd_refine", "evd_dgemm",
                     "evd_autotune"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as ge
    from paper_2511_16174_gb300 import build
    build.build()
    lib = ctypes.CDLL(str(build.OUT))
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_string_needs_no_gpu():
    from paper_2511_16174_gb300 import build
    lib = ctypes.CDLL(str(build.OUT))
    lib.evd_status_string.restype = ctypes.c_char_p
    lib.evd_status_string.argtypes = [ctypes.c_int]
    assert lib.evd_status_string(0) == b"EVD_OK"
    assert lib.evd_status_string(7) == b"EVD_ERR_TIMEOUT"


def test_plan_rejects_bad_arguments_on_host():
    """Host-detectable errors return before any device work (no GPU needed for them)."""
    from paper_2511_16174_gb300 import build
    lib = ctypes.CDLL(str(build.OUT))
    f = lib.evd_plan_create
    f.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                  ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    f.restype = ctypes.c_int
    h = ctypes.c_void_p()
    assert f(ctypes.byref(h), -1, 1, 1, 0, 0, 0, None) == 1          # n < 0
    assert f(ctypes.byref(h), 10, 5, 1, 0, 0, 0, None) == 1          # lda < n
    assert f(ctypes.byref(h), 10, 10, 1, 0, 32, 48, None) == 1       # nb % b != 0
    assert f(ctypes.byref(h), 10, 10, 1, 0, 256, 256, None) == 1     # b > 128
    assert f(ctypes.byref(h), 10, 10, 1, 1, 0, 0, None) == 8         # INT8 split not built
    assert f(None, 10, 10, 1, 0, 0, 0, None) == 1

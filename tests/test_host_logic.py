"""Host logic of the C library that runs without a GPU, through the C ABI.

* Autotuner cache: an entry for the power-of-two bucket of n, the job and the
  precision is returned as is, without timing; n in the same bucket hits the same
  entry; another job, precision or bucket does not match it; n < 64 needs no tuning.
* Product scratch sizes (evd_gemm_workspace_size): zero for the FP64 engine
  (slices = 0), growing with the slice count and with each dimension, and at least
  the bytes of the slices themselves (s (m + n) k bfloat16 values).
"""
import ctypes
import json

import pytest

from paper_2511_16174_gb300 import build


@pytest.fixture(scope="module")
def lib():
    build.build()
    L = ctypes.CDLL(str(build.OUT))
    L.evd_autotune.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_char_p,
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.evd_autotune.restype = ctypes.c_int
    L.evd_gemm_workspace_size.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_size_t)]
    L.evd_gemm_workspace_size.restype = ctypes.c_int
    return L


def tune(lib, n, job, prec, path):
    b, nb = ctypes.c_int(-1), ctypes.c_int(-1)
    st = lib.evd_autotune(n, job, prec, str(path).encode(), ctypes.byref(b), ctypes.byref(nb))
    return st, b.value, nb.value


def test_autotune_cache_hit_needs_no_gpu(lib, tmp_path):
    cache = tmp_path / "tune.jsonl"
    entries = [{"n_bucket": 2048, "job": 1, "prec": 0, "b": 64, "nb": 128, "ms": 12.5},
               {"n_bucket": 2048, "job": 0, "prec": 0, "b": 32, "nb": 64, "ms": 3.0},
               {"n_bucket": 4096, "job": 1, "prec": 0, "b": 128, "nb": 128, "ms": 80.0}]
    cache.write_text("".join(json.dumps(e) + "\n" for e in entries))
    # 1500 .. 2800 round to the bucket 2048 (log2 rounded to the nearest integer)
    for n in (1500, 2048, 2800):
        assert tune(lib, n, 1, 0, cache) == (0, 64, 128)
    assert tune(lib, 2048, 0, 0, cache) == (0, 32, 64)  # job decides
    assert tune(lib, 4000, 1, 0, cache) == (0, 128, 128)  # bucket 4096


def test_autotune_small_n_needs_no_tuning(lib, tmp_path):
    assert tune(lib, 40, 1, 0, tmp_path / "none.jsonl") == (0, 32, 32)


def test_autotune_rejects_int8_and_bad_arguments(lib, tmp_path):
    assert tune(lib, 1000, 1, 1, tmp_path / "x.jsonl")[0] == 8  # EVD_ERR_NOT_SUPPORTED
    b = ctypes.c_int()
    assert lib.evd_autotune(-1, 1, 0, None, ctypes.byref(b), ctypes.byref(b)) == 1
    assert lib.evd_autotune(100, 1, 0, None, None, ctypes.byref(b)) == 1


def ws(lib, m, n, k, s):
    out = ctypes.c_size_t()
    assert lib.evd_gemm_workspace_size(m, n, k, s, ctypes.byref(out)) == 0
    return out.value


def test_gemm_workspace_sizes(lib):
    assert ws(lib, 1000, 1000, 1000, 0) == 0
    base = ws(lib, 1000, 700, 500, 8)
    assert base >= 8 * (1000 + 700) * 500 * 2
    assert ws(lib, 1000, 700, 500, 6) < base
    assert ws(lib, 2000, 700, 500, 8) > base
    assert ws(lib, 1000, 1400, 500, 8) > base
    assert ws(lib, 1000, 700, 1000, 8) > base
    out = ctypes.c_size_t()
    assert lib.evd_gemm_workspace_size(10, 10, 10, 9, ctypes.byref(out)) == 1  # slices > 8
    assert lib.evd_gemm_workspace_size(-1, 10, 10, 8, ctypes.byref(out)) == 1


def test_committed_gb300_cache_answers_the_benchmark_sizes(lib):
    """The cache measured on GB300 (paper_2511_16174_gb300/autotune_gb300.json) is read
    by the library itself: the n = 49152 solve of the benchmark takes its entry."""
    path = build.PKG / "autotune_gb300.json"
    entries = json.loads(path.read_text())
    for n in (8192, 16384, 49152):
        st, b, nb = tune(lib, n, 1, 0, path)
        bucket = 1 << round(__import__("math").log2(n))
        e = [x for x in entries if x["n_bucket"] == bucket and x["job"] == 1 and x["prec"] == 0][0]
        assert (st, b, nb) == (0, e["b"], e["nb"])
        assert nb % b == 0 and nb <= 16 * b

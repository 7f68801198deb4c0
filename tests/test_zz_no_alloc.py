"""evd_dgemm_static: the product with library-owned scratch (no workspace argument).

It must agree with evd_dgemm (workspace passed by the caller) within the FP64 product
bound on two calls in a row.  It must not take device memory after its first call on
the device, and it must reject a product whose scratch need exceeds the fixed
capacity before any device work.  This file is named to be collected last, and it
passes run alone too.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2511_16174_gb300 import inputs

U = 2.0 ** -53
STATIC_BYTES = 64 << 20  # EVD_STATIC_SCRATCH_BYTES


@pytest.fixture(scope="module")
def evd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_16174_gb300 import evd as m
    return m


def _dev(X, evd):
    t = evd.empty_colmajor(X.shape[0], X.shape[1])
    t.copy_(torch.from_numpy(np.ascontiguousarray(X)))
    return t


@pytest.mark.gpu
@pytest.mark.parametrize("slices,ta,tb,shape", [(8, "N", "N", (300, 200, 1000)), (8, "T", "N", (257, 64, 127)),
                                                (8, "N", "T", (130, 700, 2100)), (0, "N", "N", (90, 70, 50)),
                                                (0, "T", "N", (64, 64, 4096))])
def test_static_matches_workspace_entry_point_twice(evd, slices, ta, tb, shape):
    m, n, k = shape
    r = inputs.rng(900 + m + n + k + slices)
    A = r.standard_normal((m, k) if ta == "N" else (k, m))
    B = r.standard_normal((k, n) if tb == "N" else (n, k))
    C0 = r.standard_normal((m, n))
    opA = A if ta == "N" else A.T
    opB = B if tb == "N" else B.T
    ref = -(opA @ opB) + 0.5 * C0
    bound = 3 * k * U * (np.abs(opA) @ np.abs(opB)) + 2 * U * np.abs(C0)
    Ad, Bd = _dev(A, evd), _dev(B, evd)
    Cw = _dev(C0, evd)
    evd.dgemm(ta, tb, -1.0, Ad, Bd, 0.5, Cw, slices=slices)
    torch.cuda.synchronize()
    got_ws = Cw.cpu().numpy()
    for _ in range(2):
        Cs = _dev(C0, evd)
        evd.dgemm_static(ta, tb, -1.0, Ad, Bd, 0.5, Cs, slices=slices)
        torch.cuda.synchronize()
        got = Cs.cpu().numpy()
        assert np.all(np.abs(got - ref) <= bound)
        assert np.all(np.abs(got - got_ws) <= 2 * bound)
    assert evd.dgemm_status() == (0, 0)  # no device-side timeout latched


@pytest.mark.gpu
def test_static_takes_no_device_memory_after_first_call(evd):
    r = inputs.rng(950)
    A, B = _dev(r.standard_normal((512, 512)), evd), _dev(r.standard_normal((512, 512)), evd)
    C = _dev(np.zeros((512, 512)), evd)
    evd.dgemm_static("N", "N", 1.0, A, B, 0.0, C, slices=8)  # first call: address lookup, module load
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        evd.dgemm_static("N", "N", 1.0, A, B, 0.0, C, slices=8)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_rejects_oversize_before_device_work():
    """Runs without a GPU: the capacity check precedes every CUDA call."""
    from paper_2511_16174_gb300 import evd as m
    lib = m._lib
    fake = ctypes.c_void_p(256)  # never dereferenced: the call returns first
    size = ctypes.c_size_t()
    n = 4096
    assert lib.evd_gemm_workspace_size(n, n, n, 8, ctypes.byref(size)) == 0
    assert size.value > STATIC_BYTES
    code = lib.evd_dgemm_static(b"N", b"N", n, n, n, 1.0, fake, n, fake, n, 0.0, fake, n, 8, None)
    assert code == 2  # EVD_ERR_WORKSPACE: even its least scratch (no K-split) exceeds the array
    # invalid arguments are rejected before the capacity check
    assert lib.evd_dgemm_static(b"X", b"N", n, n, n, 1.0, fake, n, fake, n, 0.0, fake, n, 8, None) == 1
    assert lib.evd_dgemm_static(b"N", b"N", n, n, n, 1.0, fake, n, fake, n, 0.0, fake, n, 9, None) == 1

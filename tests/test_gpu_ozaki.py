"""The tensor-core split product (through evd_dgemm) against exact arithmetic.

* One slice of integer-valued operands: every partial sum is an integer and the
  result must equal the int64 product bit for bit (checks the exact FP32 tensor-core
  accumulation, the staggered drains and the int64 recombination up to K = 49152).
* Two to four slices of random operands: the result must equal, bit for bit, the
  exact rational value of the truncated slice-pair sum of the oracle's splitting
  definition, rounded once (checks the digit extraction and the scaling).
* Eight slices: within the FP64 error bound of the exact product.
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from paper_2511_16174_gb300 import inputs

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def evd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_16174_gb300 import evd as m
    return m


def dev(X, evd):
    t = evd.empty_colmajor(X.shape[0], X.shape[1])
    t.copy_(torch.from_numpy(np.ascontiguousarray(X)))
    return t


@pytest.mark.parametrize("K", [16, 300, 4096, 49152])
def test_one_slice_integer_product_is_exact(evd, K):
    r = inputs.rng(500 + K)
    m, n = 300, 200
    A = r.integers(-127, 128, size=(m, K)).astype(np.float64)
    B = r.integers(-127, 128, size=(K, n)).astype(np.float64)
    A[:, 0] = 127.0   # every row/column max is 127, so the scaling is 2^7 and one digit is exact
    B[0, :] = -127.0
    ref = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    C = dev(np.zeros((m, n)), evd)
    evd.dgemm("N", "N", 1.0, dev(A, evd), dev(B, evd), 0.0, C, slices=1)
    torch.cuda.synchronize()
    got = C.cpu().numpy()
    assert np.array_equal(got, ref), np.max(np.abs(got - ref))


@pytest.mark.parametrize("s", [2, 3, 4])
def test_few_slices_match_splitting_definition_bitwise(evd, s):
    r = inputs.rng(600 + s)
    m, n, K = 130, 70, 100
    A = r.standard_normal((m, K)) * np.exp(r.uniform(-3, 3, size=(m, 1)))
    B = r.standard_normal((K, n))
    sa, ea = oracle.ozaki_split(A, s, 7)
    sb, eb = oracle.ozaki_split(B.T, s, 7)
    ref = oracle.ozaki_value(sa, ea, sb, eb)
    C = dev(np.zeros((m, n)), evd)
    evd.dgemm("N", "N", 1.0, dev(A, evd), dev(B, evd), 0.0, C, slices=s)
    torch.cuda.synchronize()
    got = C.cpu().numpy()
    assert np.array_equal(got, ref), np.max(np.abs(got - ref))


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_eight_slices_fp64_bound(evd, ta, tb):
    r = inputs.rng(700)
    m, n, K = 257, 131, 1000
    A = r.standard_normal((m, K) if ta == "N" else (K, m))
    B = r.standard_normal((K, n) if tb == "N" else (n, K))
    C0 = r.standard_normal((m, n))
    opA = A if ta == "N" else A.T
    opB = B if tb == "N" else B.T
    C = dev(C0, evd)
    evd.dgemm(ta, tb, -1.0, dev(A, evd), dev(B, evd), 0.5, C, slices=8)
    torch.cuda.synchronize()
    got = C.cpu().numpy()
    ref = -(opA @ opB) + 0.5 * C0
    bound = 3 * K * U * (np.abs(opA) @ np.abs(opB)) + 2 * U * np.abs(C0)
    assert np.all(np.abs(got - ref) <= bound)


def test_eight_slices_long_k(evd):
    r = inputs.rng(701)
    m, n, K = 256, 192, 49152
    A = r.standard_normal((m, K))
    B = r.standard_normal((K, n))
    C = dev(np.zeros((m, n)), evd)
    evd.dgemm("N", "N", 1.0, dev(A, evd), dev(B, evd), 0.0, C, slices=8)
    torch.cuda.synchronize()
    got = C.cpu().numpy()
    ref = A @ B
    bound = 3 * K * U * (np.abs(A) @ np.abs(B))
    assert np.all(np.abs(got - ref) <= bound)
    # against the exact rational product on sampled entries: the split keeps about
    # 56 bits per operand, so the error is far below FP64's own K u |A||B|
    for (i, j) in [(0, 0), (17, 101), (255, 191), (128, 3), (77, 150), (200, 64)]:
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(A[i], B[:, j]))
        scale = float(np.abs(A[i]) @ np.abs(B[:, j]))
        assert abs(Fraction(float(got[i, j])) - exact) <= Fraction(2.0 ** -50) * Fraction(scale)

"""Reordered stages (Sec. 3.3) against the conventional order, through the C ABI.

The reordered solve forms Q_sb = Q_s Q_b I -- BC-Back of the identity, whose fused
waves skip the column tiles a group's rows are still zero in -- while D&C computes
Q_d on a second stream, then Q = Q_sb Q_d.  On the same input both orders give the
same eigenvalues (the D&C stage is the same), eigenvectors within the acceptance
bounds, and (well separated spectrum, sign fixed by the largest entry) the same
eigenvectors to a small multiple of the FP64 product error.  A column range that
skipped a nonzero tile would change Q by O(1).
"""
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


def _dev(A, evd):
    t = evd.empty_colmajor(A.shape[0], A.shape[1])
    t.copy_(torch.from_numpy(np.ascontiguousarray(A)))
    return t


def _signed(Q):
    idx = np.argmax(np.abs(Q), axis=0)
    return Q * np.sign(Q[idx, np.arange(Q.shape[1])])[None, :]


@pytest.mark.parametrize("n,prec", [(1030, "fp64"), (2048, "fp64"), (3001, "fp64"), (2048, "split_bf16")])
def test_reordered_matches_conventional(evd, n, prec):
    lam = np.sort(inputs.spectrum_uniform(n, 6100 + n))
    A = inputs.qlq(lam, 6200 + n)
    out = {}
    for order in (0, 1):
        plan = evd.Plan(n, job="V", prec=prec, b=64, nb=64, options={"order": order})
        assert plan.option("order") == order
        ws = plan.workspace()
        w = torch.empty(n, dtype=torch.float64, device="cuda")
        Q = evd.empty_colmajor(n, n)
        plan.syevd(_dev(A, evd), w, Q, ws)
        plan.check(f"syevd order={order}")
        out[order] = (w.cpu().numpy(), Q.cpu().numpy())
        m = oracle.metrics(A, out[order][0], out[order][1], w_ref=lam)
        acc = oracle.acceptance(n, float(np.max(np.abs(lam))))
        assert m["dlam"] <= acc["dlam"] and m["orth_max"] <= acc["orth_max"] and m["resid"] <= acc["resid"], (order, m)
    if prec == "fp64":
        assert np.array_equal(out[0][0], out[1][0])
    gaps = np.diff(lam)
    gap = np.minimum(np.r_[np.inf, gaps], np.r_[gaps, np.inf])
    sep = gap >= 1e-3
    d = np.abs(_signed(out[0][1])[:, sep] - _signed(out[1][1])[:, sep])
    assert np.max(d) <= 1e3 * n * U, np.max(d)


def test_reordered_is_the_default_from_8192(evd):
    assert evd.Plan(8192, job="V").option("order") == 1
    assert evd.Plan(4096, job="V").option("order") == 0
    assert evd.Plan(8192, job="V", b=32, nb=32).option("order") == 0   # needs the fused b = 64 waves

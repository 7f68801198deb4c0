"""Run-to-run repeatability of the whole solve, through the C ABI.

Every stage is deterministic by construction: the split products accumulate exact
integers, their K-split partial sums are reduced in a fixed order, the bulge
chasing's sweeps apply the same arithmetic per entry whatever their timing, the
fused BC-Back waves update each element of X once per wave with exact integer
arithmetic, and the reordered stages' concurrent D&C reads nothing the waves write.
So two solves of the same matrix with the same plan give bit-identical eigenvalues
and eigenvectors, in both precisions and both stage orders.  A race (a buffer read
before it is written, a shared-memory stage overwritten early) shows up here as a
difference, even where the results stay within the accuracy bounds.
"""
import numpy as np
import pytest
import torch

from paper_2511_16174_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def evd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_16174_gb300 import evd as m
    return m


@pytest.mark.parametrize("n,prec,order", [(4096, "fp64", 1), (4096, "split_bf16", 1), (4096, "split_bf16", 0),
                                          (3001, "fp64", 0)])
def test_two_solves_are_bit_identical(evd, n, prec, order):
    lam = np.sort(inputs.spectrum_uniform(n, 7100 + n))
    A = torch.from_numpy(inputs.qlq(lam, 7200 + n)).cuda()
    plan = evd.Plan(n, job="V", prec=prec, b=64, options={"order": order})
    ws = plan.workspace()
    out = []
    for rep in range(2):
        Ad = evd.as_colmajor(A.clone())
        w = torch.empty(n, dtype=torch.float64, device="cuda")
        Q = evd.empty_colmajor(n, n)
        plan.syevd(Ad, w, Q, ws)
        plan.check(f"syevd {prec} order={order} run {rep}")
        out.append((w.clone(), Q.clone()))
    assert torch.equal(out[0][0], out[1][0]), "eigenvalues differ between two identical solves"
    diff = (out[0][1] - out[1][1]).abs().max().item()
    assert diff == 0.0, f"eigenvectors differ between two identical solves (max |dQ| = {diff:.3e})"

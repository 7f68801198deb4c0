"""The two BC-Back paths for b = 64, through the C ABI.

* Split precision (6 slices) at n = 4096 with b = 64 takes the fused wave kernel in
  its 6-slice form (X in fixed point on the grid 2^-41), followed by refinement; the
  result must meet the FP64 acceptance bounds against the constructed spectrum
  (clustered spectra are covered at n <= 2048 in test_gpu_refine.py).
* FP64 with b = 64 and an odd leading dimension of Q cannot use the fused kernel
  (its tensor copies want an even column stride) and takes the batched split
  products; the result must meet the same bounds.
Collected last: these sizes take longer than the parity sweep.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_16174_gb300 import inputs

pytestmark = pytest.mark.gpu


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


def _bounds_hold(A, w, Q, lam):
    n = A.shape[0]
    m = oracle.metrics(A, w, Q, w_ref=lam)
    acc = oracle.acceptance(n, float(np.max(np.abs(lam))))
    assert m["dlam"] <= acc["dlam"], m
    assert m["orth_max"] <= acc["orth_max"], m
    assert m["resid"] <= acc["resid"], m
    return m


def test_split_bf16_fused_six_slices_n4096(evd):
    n = 4096
    lam = np.sort(inputs.spectrum_uniform(n, 9400))
    A = inputs.qlq(lam, 9401)
    w, Q = evd.syevd(_dev(A, evd), job="V", prec="split_bf16", b=64, nb=64)
    m = _bounds_hold(A, w.cpu().numpy(), Q.cpu().numpy(), lam)
    print(f"\nsplit-bf16 fused n={n}: |dlam| {m['dlam']:.2e} orth {m['orth_max']:.2e} resid {m['resid']:.2e}")


def test_fp64_b64_odd_ldq_unfused(evd):
    n = 1025
    lam = np.sort(inputs.spectrum_uniform(n, 9500))
    A = inputs.qlq(lam, 9501)
    plan = evd.Plan(n, job="V", b=64, nb=64)
    ws = plan.workspace()
    Ad = _dev(A, evd)
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    # Q with leading dimension n (odd): the transposed view of a contiguous n x n tensor
    Qd = torch.empty((n, n), dtype=torch.float64, device="cuda").t()
    plan.syevd(Ad, w, Qd, ws)
    plan.check("syevd, odd ldq")
    _bounds_hold(A, w.cpu().numpy(), Qd.cpu().numpy(), lam)

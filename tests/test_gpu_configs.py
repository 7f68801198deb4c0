"""The benchmark configurations' own paths, through the C ABI.

* n = 8192, b = nb = 64, A = Q Lambda Q^T with Lambda geometric from 1 down to 1e-8
  (random signs) and Q 32 seeded Householder reflectors: the whole solve against the
  constructed spectrum, with the acceptance bounds |dlam| <= 10 n u ||A||_2,
  ||Q^T Q - I||_max <= 10 n u, ||A Q - Q Lambda||_F / (n ||A||_F) <= 10 u (the metrics
  are taken on the GPU with torch's FP64 products; test side only).
* Double blocking nb = 16 b (the blocking of the largest sizes): the SBR band
  elementwise against the oracle's Eq. 1 reduction at n = 2048, b = 64, nb = 1024,
  which runs the block-presplit Z products over 16 panels, and the whole solve with
  that blocking against the oracle's eigenvalues.
* Split precision on the clustered spectrum of the split configuration (5 % of the
  eigenvalues in clusters of 8 spaced 1e-6, the rest uniform in [-1, 1]) at n = 4096:
  within the same bounds; the error against the FP64 solve is printed.
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


def _gpu_metrics(Ad, w, Q, lam):
    n = Ad.shape[0]
    with torch.no_grad():
        lam_t = torch.from_numpy(np.sort(lam)).cuda()
        dlam = float((w - lam_t).abs().max())
        O = Q.t() @ Q
        O.diagonal().sub_(1.0)
        orth = float(O.abs().max())
        del O
        R = Ad @ Q - Q * w[None, :]
        resid = float(torch.linalg.matrix_norm(R) / (n * torch.linalg.matrix_norm(Ad)))
    return {"dlam": dlam, "orth_max": orth, "resid": resid}


def _assert_bounds(m, n, lam):
    acc = oracle.acceptance(n, float(np.max(np.abs(lam))))
    assert m["dlam"] <= acc["dlam"], m
    assert m["orth_max"] <= acc["orth_max"], m
    assert m["resid"] <= acc["resid"], m


def test_config2_n8192_geometric_spectrum(evd):
    n = 8192
    lam = inputs.spectrum_geometric(n, inputs.SEED_BASE + 1)
    Ad = evd.as_colmajor(inputs.qlq_device(np.sort(lam), inputs.SEED_BASE + 1))
    plan = evd.Plan(n, job="V", b=64, nb=64)
    ws = plan.workspace()
    Aw = Ad.clone(memory_format=torch.preserve_format)
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    Q = evd.empty_colmajor(n, n)
    plan.syevd(Aw, w, Q, ws)
    plan.check("syevd n=8192")
    del Aw, ws
    m = _gpu_metrics(Ad, w, Q, lam)
    print(f"\nconfig 2 n={n}: |dlam| {m['dlam']:.2e} orth {m['orth_max']:.2e} resid {m['resid']:.2e}")
    _assert_bounds(m, n, lam)


def test_sbr_band_nb_16b_matches_oracle(evd):
    n, b, nb = 2048, 64, 1024
    A = inputs.goe(n, 4100)
    B_ref, _, _ = oracle.sbr(A, b)
    plan = evd.Plan(n, job="V", b=b, nb=nb)
    assert (plan.b, plan.nb) == (b, nb)
    ws = plan.workspace()
    Ad = _dev(A, evd)
    plan.sbr(Ad, ws)
    plan.check("sbr nb=16b")
    Ag = Ad.cpu().numpy()
    i, j = np.indices((n, n))
    band = (i >= j) & (i - j <= b)
    err = np.max(np.abs(Ag[band] - B_ref[band]))
    assert err <= 1e-12 * np.linalg.norm(A), err


def test_syevd_nb_16b_matches_oracle(evd):
    n, b, nb = 2048, 64, 1024
    A = inputs.goe(n, 4200)
    w_ref, _ = oracle.eigh(A, want_vectors=False)
    w, Q = evd.syevd(_dev(A, evd), job="V", b=b, nb=nb)
    m = oracle.metrics(A, w.cpu().numpy(), Q.cpu().numpy(), w_ref=w_ref)
    _assert_bounds(m, n, w_ref)


def test_split_bf16_clustered_n4096(evd):
    n = 4096
    lam = inputs.spectrum_clustered(n, 4300)
    Ad = _dev(inputs.qlq(lam, 4301), evd)
    w_s, Q_s = evd.syevd(Ad, job="V", prec="split_bf16")
    m = _gpu_metrics(Ad, w_s, Q_s, lam)
    w_d, _ = evd.syevd(Ad, job="V", prec="fp64")
    print(f"\nsplit-bf16 clustered n={n}: |dlam| {m['dlam']:.2e} orth {m['orth_max']:.2e} resid {m['resid']:.2e}; "
          f"max |w_split - w_fp64| {float((w_s - w_d).abs().max()):.2e}")
    _assert_bounds(m, n, lam)

"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Stage by stage on the same seeded inputs:
* SBR band: elementwise against the oracle's Eq. 1 reduction (same Householder
  convention, so the band is the same up to rounding).
* BC tridiagonal: d and e elementwise against the oracle's bulge chasing.
* D&C: eigenvalues elementwise against implicit QL on the same T; eigenvectors by
  residual, orthogonality and (well separated spectra) elementwise up to sign.
* The whole solve: |dlam| <= 10 n u ||A||_2, ||Q^T Q - I||_max <= 10 n u,
  ||A Q - Q Lambda||_F / (n ||A||_F) <= 10 u.
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


def to_dev(A):
    from paper_2511_16174_gb300 import evd as m
    t = m.empty_colmajor(A.shape[0], A.shape[1])
    t.copy_(torch.from_numpy(np.ascontiguousarray(A)))
    return t


def to_host(t):
    return t.detach().cpu().numpy()


def norm2(A):
    return float(np.max(np.abs(np.linalg.eigvalsh(A)))) if A.shape[0] else 0.0


@pytest.mark.parametrize("n,b,nb", [(64, 8, 8), (100, 32, 32), (257, 32, 32), (512, 32, 32), (300, 64, 64),
                                    (257, 32, 64), (512, 32, 128), (300, 16, 64), (129, 8, 32), (1000, 64, 256)])
def test_sbr_band_matches_oracle(evd, n, b, nb):
    """Double blocking (nb > b) defers the trailing update but computes the same band."""
    A = inputs.goe(n, 1000 + n + b)
    B_ref, _, _ = oracle.sbr(A, b)
    plan = evd.Plan(n, job="V", b=b, nb=nb)
    ws = plan.workspace()
    Ad = to_dev(A)
    plan.sbr(Ad, ws)
    plan.check("sbr")
    Ag = to_host(Ad)
    i, j = np.indices((n, n))
    band = (i >= j) & (i - j <= b)
    err = np.max(np.abs(Ag[band] - B_ref[band]))
    assert err <= 1e-12 * np.linalg.norm(A), err


@pytest.mark.parametrize("n,b", [(64, 8), (100, 16), (257, 32), (512, 32), (129, 64), (200, 3), (1100, 64),
                                 (900, 32)])
def test_bulge_chase_matches_oracle(evd, n, b):
    A = inputs.goe(n, 2000 + n + b)
    B_ref, _, _ = oracle.sbr(A, b)
    d_ref, e_ref, _ = oracle.bc(B_ref, b)
    plan = evd.Plan(n, job="V", b=b, nb=b)
    ws = plan.workspace()
    Ad = to_dev(A)
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    e = torch.empty(n, dtype=torch.float64, device="cuda")
    plan.sbr(Ad, ws)
    plan.bulge_chase(ws, d, e)
    plan.check("bc")
    scale = np.linalg.norm(A)
    assert np.max(np.abs(to_host(d) - d_ref)) <= 1e-11 * scale
    assert np.max(np.abs(to_host(e)[: n - 1] - e_ref)) <= 1e-11 * scale


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 100, 500, 1030])
def test_tridiag_solve_matches_oracle(evd, n):
    r = inputs.rng(3000 + n)
    dd = r.standard_normal(n)
    ee = r.standard_normal(max(n - 1, 0))
    w_ref, Z_ref = oracle.steql(dd, ee, "I")
    plan = evd.Plan(n, job="V", b=2, nb=2)
    ws = plan.workspace()
    d = torch.tensor(dd, device="cuda")
    e = torch.zeros(max(n, 1), dtype=torch.float64, device="cuda")
    e[: n - 1] = torch.tensor(ee, device="cuda")
    Qd = evd.empty_colmajor(n, n)
    plan.tridiag_solve(d, e, Qd, ws)
    plan.check("dc")
    w = to_host(d)
    Q = to_host(Qd)
    T = np.diag(dd) + np.diag(ee, 1) + np.diag(ee, -1)
    tn = norm2(T)
    assert np.max(np.abs(w - w_ref)) <= 10 * n * U * tn
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= 10 * n * U
    assert np.linalg.norm(T @ Q - Q * w) / (n * np.linalg.norm(T)) <= 10 * U


def test_tridiag_solve_laplacian_closed_form(evd):
    n = 700
    plan = evd.Plan(n, job="V", b=2, nb=2)
    ws = plan.workspace()
    d = torch.full((n,), 2.0, dtype=torch.float64, device="cuda")
    e = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    Qd = evd.empty_colmajor(n, n)
    plan.tridiag_solve(d, e, Qd, ws)
    plan.check("dc")
    k = np.arange(1, n + 1)
    lam = 2.0 - 2.0 * np.cos(k * np.pi / (n + 1))
    assert np.max(np.abs(to_host(d) - lam)) <= 10 * n * U * 4
    Q = to_host(Qd)
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= 10 * n * U


def test_tridiag_solve_deflation_heavy(evd):
    """Repeated diagonal blocks: many equal poles and zero couplings."""
    n = 256
    dd = np.repeat(np.array([1.0, 2.0, 3.0, 4.0]), n // 4)
    ee = np.zeros(n - 1)
    ee[::7] = 1e-3
    w_ref, _ = oracle.steql(dd, ee, None)
    plan = evd.Plan(n, job="V", b=2, nb=2)
    ws = plan.workspace()
    d = torch.tensor(dd, device="cuda")
    e = torch.zeros(n, dtype=torch.float64, device="cuda")
    e[: n - 1] = torch.tensor(ee, device="cuda")
    Qd = evd.empty_colmajor(n, n)
    plan.tridiag_solve(d, e, Qd, ws)
    plan.check("dc")
    Q = to_host(Qd)
    T = np.diag(dd) + np.diag(ee, 1) + np.diag(ee, -1)
    assert np.max(np.abs(to_host(d) - w_ref)) <= 10 * n * U * 4
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= 10 * n * U
    assert np.linalg.norm(T @ Q - Q * to_host(d)) / (n * np.linalg.norm(T)) <= 10 * U


def test_tridiag_solve_glued_copies(evd):
    """16 copies of one tridiagonal block glued by 1e-9: every eigenvalue of the
    block appears 16 times, so the merges deflate by rotations that mix columns of
    their two halves; the top merges are large enough for the tensor-core product."""
    n, nb_ = 2048, 128
    r = inputs.rng(9100)
    d0 = r.standard_normal(nb_)
    e0 = r.standard_normal(nb_ - 1)
    dd = np.tile(d0, n // nb_)
    ee = np.zeros(n - 1)
    for blk in range(n // nb_):
        ee[blk * nb_: blk * nb_ + nb_ - 1] = e0
    ee[nb_ - 1::nb_] = 1e-9
    w_ref, _ = oracle.steql(dd, ee, None)
    plan = evd.Plan(n, job="V", b=2, nb=2)
    ws = plan.workspace()
    d = torch.tensor(dd, device="cuda")
    e = torch.zeros(n, dtype=torch.float64, device="cuda")
    e[: n - 1] = torch.tensor(ee, device="cuda")
    Qd = evd.empty_colmajor(n, n)
    plan.tridiag_solve(d, e, Qd, ws)
    plan.check("dc")
    Q = to_host(Qd)
    T = np.diag(dd) + np.diag(ee, 1) + np.diag(ee, -1)
    tn = norm2(T)
    assert np.max(np.abs(to_host(d) - np.sort(w_ref))) <= 10 * n * U * tn
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= 10 * n * U
    assert np.linalg.norm(T @ Q - Q * to_host(d)) / (n * np.linalg.norm(T)) <= 10 * U


def _check_full(A, w, Q, w_ref=None):
    n = A.shape[0]
    acc = oracle.acceptance(n, norm2(A))
    m = oracle.metrics(A, w, Q, w_ref=w_ref)
    if w_ref is not None:
        assert m["dlam"] <= acc["dlam"], m
    if Q is not None:
        assert m["orth_max"] <= acc["orth_max"], m
        assert m["resid"] <= acc["resid"], m
    return m


def test_syevd_values_n512_goe(evd):
    """n = 512, A = (G + G^T)/2, b = nb = 32, eigenvalues only, elementwise vs oracle."""
    n = 512
    A = inputs.goe(n, inputs.SEED_BASE + 0)
    w_ref, _ = oracle.eigh(A, want_vectors=False)
    w, _ = evd.syevd(to_dev(A), job="N", b=32, nb=32)
    _check_full(A, to_host(w), None, w_ref=w_ref)


@pytest.mark.parametrize("n,b,nb", [(100, 8, 8), (300, 32, 32), (1024, 64, 64), (777, 32, 32), (1100, 32, 128),
                                    (2100, 64, 128)])
def test_syevd_vectors(evd, n, b, nb):
    A = inputs.goe(n, 4000 + n)
    w_ref, Q_ref = oracle.eigh(A)
    w, Q = evd.syevd(to_dev(A), job="V", b=b, nb=nb)
    _check_full(A, to_host(w), to_host(Q), w_ref=w_ref)


def test_syevd_known_spectrum_geometric(evd):
    n = 1500
    lam = inputs.spectrum_geometric(n, 17)
    A = inputs.qlq(lam, 18, k=32)
    w, Q = evd.syevd(to_dev(A), job="V", b=64, nb=64)
    _check_full(A, to_host(w), to_host(Q), w_ref=np.sort(lam))


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5])
def test_syevd_tiny(evd, n):
    A = inputs.goe(n, 50 + n) if n else np.zeros((0, 0))
    if n == 0:
        plan = evd.Plan(0, job="V")
        plan.close()
        return
    wj, _ = oracle.jacobi(A)
    w, Q = evd.syevd(to_dev(A), job="V", b=0)
    _check_full(A, to_host(w), to_host(Q), w_ref=wj)


def test_syevd_diagonal_and_zero(evd):
    n = 70
    dd = inputs.rng(5).standard_normal(n)
    w, Q = evd.syevd(to_dev(np.diag(dd)), job="V", b=8)
    assert np.max(np.abs(to_host(w) - np.sort(dd))) <= 10 * n * U * np.max(np.abs(dd))
    w0, Q0 = evd.syevd(to_dev(np.zeros((n, n))), job="V", b=8)
    assert np.all(to_host(w0) == 0.0)
    assert np.max(np.abs(to_host(Q0).T @ to_host(Q0) - np.eye(n))) <= 10 * n * U


def test_nonfinite_input_reported(evd):
    n = 40
    A = inputs.goe(n, 6)
    A[10, 3] = np.nan
    with pytest.raises(evd.EvdError) as ei:
        evd.syevd(to_dev(A), job="V", b=8)
    assert ei.value.code == 5


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_dgemm_fp64(evd, ta, tb):
    r = inputs.rng(70)
    m, n, k = 130, 77, 90
    A = r.standard_normal((m, k) if ta == "N" else (k, m))
    B = r.standard_normal((k, n) if tb == "N" else (n, k))
    C = r.standard_normal((m, n))
    ref = 1.5 * ((A if ta == "N" else A.T) @ (B if tb == "N" else B.T)) - 0.5 * C
    Cd = to_dev(C)
    evd.dgemm(ta, tb, 1.5, to_dev(A), to_dev(B), -0.5, Cd, slices=0)
    torch.cuda.synchronize()
    bound = 2 * k * U * (np.abs(A if ta == "N" else A.T) @ np.abs(B if tb == "N" else B.T)) * 1.5 + 2 * U * np.abs(C)
    assert np.all(np.abs(to_host(Cd) - ref) <= bound + 1e-300)

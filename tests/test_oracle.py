"""Pins for the CPU oracle: closed forms, invariants, special cases and brute force.

None of these compares the oracle with itself; each checks it against a fact the
mathematics fixes (1D Laplacian spectrum and eigenvectors, 2x2 closed form, Jacobi
on tiny matrices, orthogonal similarity invariants, band structure, the implicit-Q
theorem, the reduction of b = 1 SBR to one-stage tridiagonalization).
"""
import math
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2511_16174_gb300 import inputs

U = 2.0 ** -53
GOLDEN = Path(__file__).resolve().parent / "golden"


def lap_eigs(n):
    k = np.arange(1, n + 1)
    return 2.0 - 2.0 * np.cos(k * np.pi / (n + 1))


def lap_vecs(n):
    j = np.arange(1, n + 1)[:, None]
    k = np.arange(1, n + 1)[None, :]
    return np.sqrt(2.0 / (n + 1)) * np.sin(j * k * np.pi / (n + 1))


def sign_fix(Q):
    """Make the first entry of each column that is not negligible positive."""
    Q = np.array(Q)
    thr = 1e-6 * np.max(np.abs(Q), axis=0)
    idx = np.argmax(np.abs(Q) > thr[None, :], axis=0)
    s = np.sign(Q[idx, np.arange(Q.shape[1])])
    s[s == 0] = 1
    return Q * s[None, :]


# ---------------------------------------------------------------- Householder
def test_house_annihilates_and_is_orthogonal():
    r = inputs.rng(1)
    for m in (2, 3, 17, 64):
        x = r.standard_normal(m)
        beta, v, tau = oracle.house(x)
        H = np.eye(m) - tau * np.outer(v, v)
        y = H @ x
        assert abs(y[0] - beta) <= 1e-14 * np.linalg.norm(x)
        assert np.max(np.abs(y[1:])) <= 1e-14 * np.linalg.norm(x)
        assert np.max(np.abs(H.T @ H - np.eye(m))) <= 1e-14
        # LAPACK sign choice: beta = -sign(alpha) ||x||
        assert beta == pytest.approx(-math.copysign(np.linalg.norm(x), x[0]), rel=1e-14)


def test_house_zero_tail_is_identity():
    for alpha in (3.0, -2.0, 0.0):
        beta, v, tau = oracle.house([alpha, 0.0, 0.0])
        assert tau == 0.0 and beta == alpha


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [1, 2, 5, 64, 257])
def test_steql_laplacian_values(n):
    w, _ = oracle.steql(2.0 * np.ones(n), -np.ones(max(n - 1, 0)))
    assert np.max(np.abs(w - lap_eigs(n))) <= 8 * n * U * 4.0


@pytest.mark.parametrize("n", [2, 9, 100])
def test_steql_laplacian_vectors(n):
    w, Z = oracle.steql(2.0 * np.ones(n), -np.ones(n - 1), "I")
    ref = lap_vecs(n)
    assert np.max(np.abs(sign_fix(Z) - sign_fix(ref))) <= 100 * n * U


@pytest.mark.parametrize("n", [1, 3, 50, 300])
def test_bisect_laplacian(n):
    w = oracle.bisect(2.0 * np.ones(n), -np.ones(max(n - 1, 0)))
    assert np.max(np.abs(w - lap_eigs(n))) <= 8 * n * U * 4.0


def test_golden_laplacian_n8():
    ref = np.loadtxt(GOLDEN / "laplacian_n8_eigs.txt")
    w, _ = oracle.steql(2.0 * np.ones(8), -np.ones(7))
    assert np.max(np.abs(w - ref)) <= 16 * U * 4
    wb = oracle.bisect(2.0 * np.ones(8), -np.ones(7))
    assert np.max(np.abs(wb - ref)) <= 16 * U * 4


def test_jacobi_2x2_closed_form():
    r = inputs.rng(2)
    for _ in range(20):
        a, b, c = r.standard_normal(3)
        mid, rad = (a + c) / 2, math.hypot((a - c) / 2, b)
        w, V = oracle.jacobi(np.array([[a, b], [b, c]]))
        assert w == pytest.approx([mid - rad, mid + rad], abs=1e-14 * (abs(mid) + rad))
        A = np.array([[a, b], [b, c]])
        assert np.max(np.abs(A @ V - V * w)) <= 1e-14 * (abs(mid) + rad)


def test_diagonal_input_sorts():
    r = inputs.rng(3)
    dd = r.standard_normal(40)
    A = np.diag(dd)
    w, Q = oracle.eigh(A)
    assert np.array_equal(w, np.sort(dd))
    wj, _ = oracle.jacobi(A[:8, :8])
    assert np.array_equal(wj, np.sort(dd[:8]))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_brute_force_jacobi_vs_ql_vs_bisection(n):
    for seed in range(4):
        A = inputs.goe(n, 100 + seed)
        wj, Vj = oracle.jacobi(A)
        wq, Q = oracle.eigh(A)
        d, e, _ = oracle.sytrd(A)
        wb = oracle.bisect(d, e)
        scale = np.max(np.abs(wj)) + 1e-300
        assert np.max(np.abs(wj - wq)) <= 20 * n * U * scale
        assert np.max(np.abs(wj - wb)) <= 20 * n * U * scale
        assert np.max(np.abs(A @ Q - Q * wq)) <= 50 * n * U * scale


def test_clustered_wilkinson_like():
    # W21+ has pairs of eigenvalues agreeing to ~1e-13: a hard case for QL deflation
    n = 21
    d = np.abs(np.arange(n) - 10).astype(float)
    e = np.ones(n - 1)
    w, Z = oracle.steql(d, e, "I")
    wb = oracle.bisect(d, e)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    wj, _ = oracle.jacobi(T)
    assert np.max(np.abs(w - wj)) <= 1e-13
    assert np.max(np.abs(wb - wj)) <= 1e-13
    assert np.max(np.abs(Z.T @ Z - np.eye(n))) <= 1e-13
    # the two largest agree to about 1e-14 (known property of W21+)
    assert abs(w[-1] - w[-2]) < 1e-12


# ---------------------------------------------------------------- one-stage path
@pytest.mark.parametrize("n", [4, 33, 128])
def test_sytrd_reconstructs_and_preserves_invariants(n):
    A = inputs.goe(n, 7 + n)
    d, e, Q = oracle.sytrd(A, want_q=True)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    normA = np.linalg.norm(A)
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= 20 * n * U
    assert np.linalg.norm(Q @ T @ Q.T - A) <= 20 * n * U * normA
    assert abs(np.sum(d) - np.trace(A)) <= 20 * n * U * normA
    assert abs(np.sqrt(np.sum(d ** 2) + 2 * np.sum(e ** 2)) - normA) <= 20 * n * U * normA
    # Q e_1 = e_1: reflectors never touch index 0
    assert np.array_equal(Q[:, 0], np.eye(n)[:, 0])


@pytest.mark.parametrize("kind", ["geometric", "uniform", "clustered"])
def test_eigh_known_spectrum(kind):
    n = 160
    lam = {"geometric": inputs.spectrum_geometric, "uniform": inputs.spectrum_uniform,
           "clustered": inputs.spectrum_clustered}[kind](n, 11)
    A = inputs.qlq(lam, 12, k=8)
    w, Q = oracle.eigh(A)
    acc = oracle.acceptance(n, float(np.max(np.abs(lam))))
    m = oracle.metrics(A, w, Q, w_ref=np.sort(lam))
    assert m["dlam"] <= acc["dlam"]
    assert m["orth_max"] <= acc["orth_max"]
    assert m["resid"] <= acc["resid"]


def test_eigh_laplacian_dense_similarity():
    n = 60
    Qr, _ = np.linalg.qr(inputs.rng(5).standard_normal((n, n)))
    A = Qr @ inputs.laplacian(n) @ Qr.T
    A = 0.5 * (A + A.T)
    w, Q = oracle.eigh(A)
    assert np.max(np.abs(w - lap_eigs(n))) <= 10 * n * U * 4


# ---------------------------------------------------------------- SBR (Sec. 2.1.1, Eq. 1)
@pytest.mark.parametrize("n,b", [(40, 4), (64, 8), (100, 32), (33, 8), (17, 32)])
def test_sbr_band_structure_and_reconstruction(n, b):
    A = inputs.goe(n, 200 + n + b)
    B, Ys, taus = oracle.sbr(A, b, keep_reflectors=True)
    i, j = np.indices((n, n))
    assert np.all(B[np.abs(i - j) > b] == 0.0), "entries outside the band must be exactly zero"
    assert np.max(np.abs(B - B.T)) <= 20 * n * U * np.linalg.norm(A)
    Qs = oracle.sbr_q(Ys, taus)
    normA = np.linalg.norm(A)
    assert np.max(np.abs(Qs.T @ Qs - np.eye(n))) <= 20 * n * U
    assert np.linalg.norm(Qs @ B @ Qs.T - A) <= 50 * n * U * normA
    assert abs(np.trace(B) - np.trace(A)) <= 20 * n * U * normA
    assert abs(np.linalg.norm(B) - normA) <= 20 * n * U * normA
    # first b columns of Q_s are e_1..e_b: panel p's reflectors start at row (p+1) b
    assert np.array_equal(Qs[:, :b], np.eye(n)[:, :b])


def test_sbr_spectrum_matches():
    n, b = 96, 16
    lam = inputs.spectrum_uniform(n, 3)
    A = inputs.qlq(lam, 4, k=8)
    B, _, _ = oracle.sbr(A, b)
    w, _ = oracle.eigh(B, want_vectors=False)
    assert np.max(np.abs(w - lam)) <= 10 * n * U


@pytest.mark.parametrize("n", [5, 50, 129])
def test_sbr_b1_is_one_stage(n):
    A = inputs.goe(n, 300 + n)
    B, _, _ = oracle.sbr(A, 1)
    d1, e1, _ = oracle.sytrd(A)
    scale = np.linalg.norm(A)
    assert np.max(np.abs(np.diag(B) - d1)) <= 50 * n * U * scale
    assert np.max(np.abs(np.diag(B, -1) - e1)) <= 50 * n * U * scale


def test_sbr_n_le_b_is_noop():
    A = inputs.goe(10, 9)
    B, _, _ = oracle.sbr(A, 16)
    S = np.tril(A) + np.tril(A, -1).T
    assert np.array_equal(B, S)


# ---------------------------------------------------------------- BC (Sec. 2.1.1, Sec. 4.2)
@pytest.mark.parametrize("n,b", [(40, 4), (64, 8), (100, 16), (37, 5), (9, 32)])
def test_bc_tridiagonal_reconstruction(n, b):
    A = inputs.goe(n, 400 + n + b)
    B, _, _ = oracle.sbr(A, b)
    d, e, Qb = oracle.bc(B, b, want_q=True)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    normB = np.linalg.norm(B)
    assert np.max(np.abs(Qb.T @ Qb - np.eye(n))) <= 50 * n * U
    assert np.linalg.norm(Qb @ T @ Qb.T - B) <= 100 * n * U * normB
    assert abs(np.sum(d) - np.trace(B)) <= 20 * n * U * normB
    assert abs(np.sqrt(np.sum(d ** 2) + 2 * np.sum(e ** 2)) - normB) <= 50 * n * U * normB
    assert np.array_equal(Qb[:, 0], np.eye(n)[:, 0])


def test_bc_b1_noop():
    n = 30
    A = inputs.goe(n, 5)
    Tin = np.diag(np.diag(A)) + np.diag(np.diag(A, -1), -1)
    d, e, _ = oracle.bc(Tin, 1)
    assert np.array_equal(d, np.diag(A)) and np.array_equal(e, np.diag(A, -1))


@pytest.mark.parametrize("n,b", [(64, 8), (120, 16), (200, 32)])
def test_two_stage_matches_one_stage_implicit_q(n, b):
    """Implicit-Q theorem: both reductions are orthogonal similarities whose first
    column is e_1, so for an unreduced T the diagonals agree and the off-diagonals
    agree in magnitude."""
    A = inputs.goe(n, 500 + n)
    d1, e1, _ = oracle.sytrd(A)
    B, _, _ = oracle.sbr(A, b)
    d2, e2, _ = oracle.bc(B, b)
    scale = np.linalg.norm(A)
    assert np.max(np.abs(d1 - d2)) <= 1e-10 * scale
    assert np.max(np.abs(np.abs(e1) - np.abs(e2))) <= 1e-10 * scale


# ---------------------------------------------------------------- metrics and refinement
def test_metrics_exact_decomposition_is_small_and_perturbation_is_seen():
    n = 50
    lam = inputs.spectrum_uniform(n, 8)
    Qr, _ = np.linalg.qr(inputs.rng(9).standard_normal((n, n)))
    A = (Qr * lam) @ Qr.T
    m = oracle.metrics(A, lam, Qr, w_ref=lam)
    assert m["orth_max"] < 1e-14 and m["resid"] < 1e-16 and m["backward"] < 1e-16
    Qp = Qr + 1e-8 * inputs.rng(10).standard_normal((n, n))
    mp = oracle.metrics(A, lam, Qp, w_ref=lam)
    assert mp["orth_max"] > 1e-9 and mp["resid"] > 1e-11


def test_refine_quadratic_convergence_and_fixed_point():
    # well-separated spectrum (gap 2/(n-1)) so that every pair is outside delta
    n = 80
    lam = np.linspace(-1.0, 1.0, n)
    Qr, _ = np.linalg.qr(inputs.rng(21).standard_normal((n, n)))
    A = (Qr * lam) @ Qr.T
    A = 0.5 * (A + A.T)
    X = Qr + 1e-6 * inputs.rng(22).standard_normal((n, n))
    err0 = np.max(np.abs(X - Qr))
    lam1, X1, _ = oracle.refine(A, X)
    err1 = np.max(np.abs(X1 - Qr))
    lam2, X2, _ = oracle.refine(A, X1)
    err2 = np.max(np.abs(X2 - Qr))
    assert err1 < 100 * err0 ** 2 / (2.0 / (n - 1)) + 1e-14   # quadratic, scaled by 1/gap
    assert err1 < 1e-3 * err0
    assert err2 < 1e-13
    assert np.max(np.abs(lam2 - lam)) < 1e-14
    # exact input is a fixed point up to rounding
    _, X3, _ = oracle.refine(A, Qr)
    assert np.max(np.abs(X3 - Qr)) < 1e-14


def test_refine_clustered_falls_back_to_half_r():
    # a doubly repeated eigenvalue: the pair lies inside delta and gets r/2
    lam = np.array([-1.0, 0.3, 0.3, 2.0])
    Qr, _ = np.linalg.qr(inputs.rng(30).standard_normal((4, 4)))
    A = (Qr * lam) @ Qr.T
    X = Qr + 1e-6 * inputs.rng(31).standard_normal((4, 4))
    lam1, X1, info = oracle.refine(A, X)
    assert np.max(np.abs(X1.T @ X1 - np.eye(4))) < 1e-10
    assert np.max(np.abs(A @ X1 - X1 * lam1)) < 1e-10


def _mixed_pair_case():
    """A spectrum with one pair of gap 1e-9, the eigenvectors of that pair rotated by
    1e-4 within the pair (a coupling s_ij of 1e-13, the size a perturbation of A at
    that level leaves), plus a 1e-8 perturbation everywhere: the first step's
    delta (about 1e-5) holds the pair as a cluster, the second step's would not."""
    n = 120
    lam = np.linspace(-1.0, 1.0, n)
    lam[61] = lam[60] + 1e-9
    Qr, _ = np.linalg.qr(inputs.rng(33).standard_normal((n, n)))
    A = (Qr * lam) @ Qr.T
    A = 0.5 * (A + A.T)
    th = 1e-4
    X = Qr.copy()
    X[:, 60] = np.cos(th) * Qr[:, 60] + np.sin(th) * Qr[:, 61]
    X[:, 61] = -np.sin(th) * Qr[:, 60] + np.cos(th) * Qr[:, 61]
    X = X + 1e-8 * inputs.rng(34).standard_normal((n, n))
    return A, lam, X


def test_refine_held_delta_keeps_orthogonality():
    """Two steps with delta held: the mixed pair stays a cluster, orthogonality
    reaches rounding level and the residual its FP64 level."""
    A, lam, X = _mixed_pair_case()
    n = A.shape[0]
    lam2, X2, deltas = oracle.refine_steps(A, X, 2)
    assert deltas[0] > 1e-9 and deltas[1] == deltas[0]
    assert np.max(np.abs(X2.T @ X2 - np.eye(n))) < 1e-13
    assert np.linalg.norm(A @ X2 - X2 * lam2) / (n * np.linalg.norm(A)) < 1e-14


def test_refine_shrinking_delta_breaks_orthogonality():
    """Failing control: the same two steps with delta recomputed afresh rotate the
    pair by about 1e-4 in the second step and lose orthogonality to about 1e-8."""
    A, lam, X = _mixed_pair_case()
    n = A.shape[0]
    _, X1, info1 = oracle.refine(A, X)
    _, X2, info2 = oracle.refine(A, X1)
    assert info2["delta"] < 1e-9 < info1["delta"]
    assert np.max(np.abs(X2.T @ X2 - np.eye(n))) > 1e-10


# ---------------------------------------------------------------- error-free splitting
def test_ozaki_split_exact_rational_definition():
    r = inputs.rng(40)
    X = r.standard_normal((3, 7)) * np.array([[1.0], [1e-20], [3e5]])
    X[0, 3] = 0.0
    s, w = 8, 7
    sig, e = oracle.ozaki_split(X, s=s, w=w)
    for i in range(3):
        amax = np.max(np.abs(X[i]))
        assert 2.0 ** (int(e[i]) - 1) <= amax < 2.0 ** int(e[i])
        for k in range(7):
            x = Fraction(float(X[i, k])) * Fraction(2) ** (w * s - int(e[i]))
            # round half away from zero
            T = math.floor(abs(x) + Fraction(1, 2)) * (1 if x >= 0 else -1)
            rec = sum(int(sig[t, i, k]) * (1 << (w * (s - 1 - t))) for t in range(s))
            assert rec == T
            assert abs(int(sig[0, i, k])) <= 1 << w
            for t in range(1, s):
                assert -(1 << (w - 1)) <= int(sig[t, i, k]) < (1 << (w - 1))


def test_ozaki_value_is_within_fp64_gemm_bound():
    r = inputs.rng(41)
    M, N, K = 6, 5, 40
    A = r.standard_normal((M, K))
    B = r.standard_normal((K, N))
    sa, ea = oracle.ozaki_split(A, 8, 7)
    sb, eb = oracle.ozaki_split(B.T, 8, 7)
    C = oracle.ozaki_value(sa, ea, sb, eb)
    exact = np.array([[float(sum(Fraction(float(A[i, k])) * Fraction(float(B[k, j])) for k in range(K)))
                       for j in range(N)] for i in range(M)])
    bound = K * U * (np.abs(A) @ np.abs(B))
    assert np.all(np.abs(C - exact) <= bound)
    # fewer slices lose accuracy the way the split predicts
    C3 = oracle.ozaki_value(sa[:3], ea, sb[:3], eb)
    err3 = np.max(np.abs(C3 - exact) / (np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(B), axis=0)[None, :]))
    # three 7-bit slices keep 21 bits: error about K 2^-22 of max|a| max|b|
    assert 2.0 ** -14 > err3 > 2.0 ** -28

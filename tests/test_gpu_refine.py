"""Ogita-Aishima refinement and the split-precision solve, through the C ABI.

* One refinement step on the GPU equals the oracle's step (same formulas, FP64
  products) elementwise, from the same perturbed eigenvector matrix.
* Two steps (threshold held, as the solve runs them) from the eigenvectors of a
  perturbed matrix equal the oracle's two steps and reach the FP64 acceptance
  bounds.
* The split-precision solve (4 bfloat16 slices for the dense products, then
  refinement) meets the same bounds as the FP64 solve on a spectrum with tight
  clusters; its error against the FP64 solve is printed for every result.
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


def dev(X, evd):
    t = evd.empty_colmajor(X.shape[0], X.shape[1])
    t.copy_(torch.from_numpy(np.ascontiguousarray(X)))
    return t


def _perturbed(n, seed, eps):
    lam = inputs.spectrum_uniform(n, seed)
    A = inputs.qlq(lam, seed + 1)
    _, Q = oracle.eigh(A)
    X = Q + eps * inputs.rng(seed + 2).standard_normal((n, n))
    return A, np.sort(lam), X


@pytest.mark.parametrize("n", [64, 300])
def test_refine_step_matches_oracle(evd, n):
    A, _, X = _perturbed(n, 7100 + n, 1e-6)
    lam_ref, X_ref, _ = oracle.refine(A, X)
    plan = evd.Plan(n, job="V", prec="split_bf16")
    ws = plan.workspace()
    Xd = dev(X, evd)
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    plan.refine(dev(A, evd), w, Xd, 1, ws)
    plan.check("refine")
    Xg = Xd.cpu().numpy()
    assert np.max(np.abs(w.cpu().numpy() - lam_ref)) <= 100 * n * U * np.max(np.abs(lam_ref))
    assert np.max(np.abs(Xg - X_ref)) <= 1e-12


def test_refine_two_steps_match_oracle_and_reach_fp64_bounds(evd):
    """X = the eigenvectors of A + P, P symmetric at 1e-9 ||A|| (what a solve with
    less accurate products leaves): two steps with the threshold held equal the
    oracle's two steps and reach the FP64 bounds."""
    n = 400
    lam = inputs.spectrum_uniform(n, 7300)
    A = inputs.qlq(lam, 7301)
    P = inputs.rng(7302).standard_normal((n, n))
    P = 1e-9 * np.linalg.norm(A, 2) * (P + P.T) / np.linalg.norm(P + P.T, 2)
    _, X = oracle.eigh(A + P)
    lam_ref, X_ref, deltas = oracle.refine_steps(A, X, 2)
    plan = evd.Plan(n, job="V", prec="split_bf16")
    ws = plan.workspace()
    Xd = dev(X, evd)
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    plan.refine(dev(A, evd), w, Xd, 2, ws)
    plan.check("refine")
    Xg, wg = Xd.cpu().numpy(), w.cpu().numpy()
    # E_ij = (s_ij + lam_j r_ij) / (lam_j - lam_i): an FP64-accurate s_ij carries about
    # u ||A|| of rounding (the GPU's and numpy's differ), so a column's rotation against
    # a neighbour at distance gap is fixed to about u ||A|| / gap per step.  Columns
    # whose eigenvalue is at least 1e-3 from both neighbours are compared elementwise
    # within 20 u ||A||_2 / 1e-3 (two steps, a factor 10 of margin); all columns are
    # held to the acceptance bounds below.
    gaps = np.diff(np.sort(lam_ref))
    gap = np.minimum(np.r_[np.inf, gaps], np.r_[gaps, np.inf])[np.argsort(np.argsort(lam_ref))]
    sep = gap >= 1e-3
    assert sep.sum() > n // 2
    tol = 20 * U * np.max(np.abs(lam_ref)) / 1e-3
    assert np.max(np.abs(Xg[:, sep] - X_ref[:, sep])) <= tol
    assert np.max(np.abs(wg - lam_ref)) <= 100 * n * U * np.max(np.abs(lam_ref))
    lam = np.sort(lam)
    m = oracle.metrics(A, wg, Xg, w_ref=lam)
    acc = oracle.acceptance(n, float(np.max(np.abs(lam))))
    assert m["dlam"] <= acc["dlam"], m
    assert m["orth_max"] <= acc["orth_max"], m
    assert m["resid"] <= acc["resid"], m


@pytest.mark.parametrize("n", [1100, 2048])
def test_split_bf16_solve_meets_fp64_bounds_on_clusters(evd, n):
    lam = inputs.spectrum_clustered(n, 7500 + n)
    A = inputs.qlq(lam, 7600 + n)
    w_s, Q_s = evd.syevd(dev(A, evd), job="V", prec="split_bf16")
    w_d, Q_d = evd.syevd(dev(A, evd), job="V", prec="fp64")
    ws_, Qs_ = w_s.cpu().numpy(), Q_s.cpu().numpy()
    m = oracle.metrics(A, ws_, Qs_, w_ref=lam)
    acc = oracle.acceptance(n, float(np.max(np.abs(lam))))
    print(f"\nsplit-bf16 n={n}: |dlam| {m['dlam']:.2e} orth {m['orth_max']:.2e} resid {m['resid']:.2e}; "
          f"vs FP64 solve: max |w_s - w_d| {np.max(np.abs(ws_ - w_d.cpu().numpy())):.2e}")
    assert m["dlam"] <= acc["dlam"], m
    assert m["orth_max"] <= acc["orth_max"], m
    assert m["resid"] <= acc["resid"], m

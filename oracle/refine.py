"""Ogita-Aishima eigenpair refinement, one step, plain FP64 (test infrastructure).

Ogita & Aishima, "Iterative refinement for symmetric eigenvalue decomposition",
Japan J. Indust. Appl. Math. 35 (2018).  Given symmetric A and an approximate
eigenvector matrix X:

    R  = I - X^T X
    S  = X^T A X
    lam_i = s_ii / (1 - r_ii)
    delta = 2 (||S - diag(lam)||_2 + ||A||_2 ||R||_2)
    E_ij = (s_ij + lam_j r_ij) / (lam_j - lam_i)   if |lam_i - lam_j| > delta
         = r_ij / 2                                 otherwise (including i == j)
    X'  = X + X E

The 2-norms in delta are replaced by Frobenius norms, which bound them from above
(so the threshold can only grow; clustered pairs then fall into the r_ij/2 branch,
which is the safe one).  Matrix products are numpy's FP64 matmul.

Over several steps delta is held at its largest value (``delta_floor``): the new
X satisfies X'^T X' - I = E^T E + (terms of the size of R E) to second order, so a
pair that an earlier step treated as a cluster, and whose mixing it therefore kept,
would be rotated by E_ij ~ s_ij / (lam_j - lam_i) once a smaller delta lets it
through, leaving an orthogonality error of that size squared.  ``refine_steps``
threads the floor through its steps.

R and S are symmetric by definition; the computed products are replaced by their
symmetric parts (R + R^T)/2, (S + S^T)/2.  Without that, E_ij + E_ji = r_ij +
(s_ij - s_ji)/(lam_j - lam_i) carries the rounding asymmetry of S divided by the
eigenvalue gap, and the orthogonality of X stalls near 1e-12 in FP64.
"""
from __future__ import annotations

import numpy as np


def refine(A, X, delta_floor=0.0):
    """One refinement step with threshold max(delta, delta_floor).  Returns
    (lam, X_new, info) with info holding the delta used."""
    A = np.asarray(A, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    n = A.shape[0]
    R = np.eye(n) - X.T @ X
    S = X.T @ (A @ X)
    R = 0.5 * (R + R.T)
    S = 0.5 * (S + S.T)
    r = np.diag(R)
    lam = np.diag(S) / (1.0 - r)
    D = S - np.diag(lam)
    delta = max(2.0 * (np.linalg.norm(D) + np.linalg.norm(A) * np.linalg.norm(R)), float(delta_floor))
    diff = lam[None, :] - lam[:, None]          # diff[i, j] = lam_j - lam_i
    far = np.abs(diff) > delta
    E = np.where(far, (S + lam[None, :] * R) / np.where(far, diff, 1.0), 0.5 * R)
    Xn = X + X @ E
    return lam, Xn, {"delta": float(delta)}


def refine_steps(A, X, steps):
    """``steps`` refinement steps, delta held at its largest value so far.
    Returns (lam, X, deltas)."""
    lam, deltas, floor = None, [], 0.0
    for _ in range(steps):
        lam, X, info = refine(A, X, delta_floor=floor)
        floor = info["delta"]
        deltas.append(floor)
    return lam, X, deltas

"""Error measures and acceptance bounds for an eigendecomposition (test infrastructure).

* ``backward`` and ``orth_paper`` are the two quantities of Table 2 (Sec. 3.3.1):
  ||A - Q Lambda Q^T|| / (n ||A||) and ||I - Q Q^T|| / n, with the Frobenius norm
  (the paper leaves the norm unstated; Frobenius reproduces the magnitudes of
  Table 2, see the design notes).
* ``orth_max`` = ||Q^T Q - I||_max, ``resid`` = ||A Q - Q Lambda||_F / (n ||A||_F) and
  ``dlam`` = max |lambda - lambda_ref| are the acceptance measures, with bounds
  10 n u ||A||_2, 10 n u and 10 u for u = 2^-53.
"""
from __future__ import annotations

import numpy as np

U = 2.0 ** -53


def metrics(A, w, Q=None, w_ref=None):
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    out = {"n": n}
    if n == 0:
        return out
    # lower triangle is the source of truth
    L = np.tril(A)
    S = L + np.tril(L, -1).T
    normF = np.linalg.norm(S)
    out["normF"] = float(normF)
    out["trace_err"] = float(abs(np.sum(w) - np.trace(S)) / max(normF, 1e-300))
    out["frob_err"] = float(abs(np.sqrt(np.sum(np.asarray(w) ** 2)) - normF) / max(normF, 1e-300))
    if w_ref is not None:
        out["dlam"] = float(np.max(np.abs(np.asarray(w) - np.asarray(w_ref))))
    if Q is not None:
        Q = np.asarray(Q, dtype=np.float64)
        I = np.eye(n)
        out["orth_max"] = float(np.max(np.abs(Q.T @ Q - I)))
        R = S @ Q - Q * np.asarray(w)[None, :]
        out["resid"] = float(np.linalg.norm(R) / (n * max(normF, 1e-300)))
        B = S - (Q * np.asarray(w)[None, :]) @ Q.T
        out["backward"] = float(np.linalg.norm(B) / (n * max(normF, 1e-300)))
        out["orth_paper"] = float(np.linalg.norm(I - Q @ Q.T) / n)
    return out


def acceptance(n, norm2):
    """The acceptance bounds for an n x n problem with ||A||_2 = norm2."""
    return {
        "dlam": 10.0 * n * U * norm2,
        "orth_max": 10.0 * n * U,
        "resid": 10.0 * U,
    }
